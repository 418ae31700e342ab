// Allocation-free single 1D step.
//
// Some callers cannot allocate device memory at the point where they want to advance a
// solution: real-time loops that cannot take the latency of an allocation or the device-wide
// synchronisation that freeing memory implies, and host frameworks that own every byte of device
// memory through their own pool and forbid a library from allocating behind their back.
// shweno_step1d_noalloc serves them: the caller passes its input and output state, and the step's
// scratch (the per-face fluxes and interface states, plus the small control block of the step
// kernels) lives in one file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.  The call waits for its own work before it returns.
//
// Set-up: the device address of that array is looked up with cudaGetSymbolAddress the first
// time the entry point runs on a device (with that device current) and cached per device for
// the rest of the process; that first call should come before any stream capture.  The cached
// address belongs to the device's primary context: a process that destroys that context
// (cudaDeviceReset) must not call this entry point again.  Every call shares the one array per
// device, so calls whose work overlaps on the GPU (different streams, or different host threads)
// race on it; callers must order them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/shweno.h"
#include "shweno_kernels.h"

namespace {

using shweno::Ctl;
using shweno::Params;

constexpr size_t kCtlDoubles = 32;  // 256 bytes reserved for the control block
static_assert(sizeof(Ctl) <= kCtlDoubles * sizeof(double), "control block does not fit");
constexpr size_t kFaceDoubles = 2 * 3 * ((size_t)SHWENO_NOALLOC_MAX_NX + 1);  // F-hat and W(t+dt)

static __device__ __align__(256) double g_noalloc_scratch[kCtlDoubles + kFaceDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

__global__ void noalloc_begin_kernel(Ctl* c, double t, double dt) {
  c->t = t;
  c->dt = dt;
  c->t_final = INFINITY;
  c->cfl = 0.0;
  c->dt_fixed = dt;
  c->nsteps = 0;  // input buffer = state_in, output buffer = state_out
  c->err_step = -1;
  c->rate_cur = 0ull;
  c->rate_next = 0ull;
  c->mode = 0;
  c->err = shweno::ERR_NONE;
  c->active = 1;
}

}  // namespace

extern "C" shweno_status shweno_step1d_noalloc(int32_t eq, int64_t nx, double x0, double x1,
                                               double gamma, const int32_t bc_kind[2],
                                               const double inflow[2][4], int32_t flag_mode,
                                               const double* state_in, double* state_out,
                                               double t, double dt, void* cuda_stream) {
  if (eq != SHWENO_BURGERS && eq != SHWENO_EULER) return SHWENO_E_INVALID;
  if (nx < 4 || nx > SHWENO_NOALLOC_MAX_NX) return SHWENO_E_INVALID;
  if (!(x1 > x0) || !(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t)) return SHWENO_E_INVALID;
  if (eq == SHWENO_EULER && !(gamma > 1.0)) return SHWENO_E_INVALID;
  if (!bc_kind || !state_in || !state_out || state_in == state_out) return SHWENO_E_INVALID;
  if (flag_mode != 0 && flag_mode != 1) return SHWENO_E_INVALID;
  for (int s = 0; s < 2; ++s)
    if (bc_kind[s] < SHWENO_BC_PERIODIC || bc_kind[s] > SHWENO_BC_INFLOW) return SHWENO_E_INVALID;
  if ((bc_kind[0] == SHWENO_BC_PERIODIC) != (bc_kind[1] == SHWENO_BC_PERIODIC)) return SHWENO_E_INVALID;
  // an INFLOW side needs the state it imposes
  if (!inflow && (bc_kind[0] == SHWENO_BC_INFLOW || bc_kind[1] == SHWENO_BC_INFLOW)) return SHWENO_E_INVALID;
  const int ncomp = eq == SHWENO_BURGERS ? 1 : 3;
  {  // the two states must not overlap
    const size_t bytes = 2 * (size_t)ncomp * nx * sizeof(double);
    const char* a = (const char*)state_in;
    const char* b = (const char*)state_out;
    if (a < b + bytes && b < a + bytes) return SHWENO_E_INVALID;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SHWENO_E_CUDA;
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SHWENO_E_CUDA;
      }
      g_scratch_ptr[dev] = (double*)p;
    }
    base = g_scratch_ptr[dev];
  }
  Ctl* ctl = (Ctl*)base;
  double* FH = base + kCtlDoubles;
  double* WE = FH + (size_t)ncomp * (nx + 1);

  Params P{};
  P.dim = 1;
  P.eq = eq;
  P.ncomp = ncomp;
  P.nx = (int32_t)nx;
  P.ny = 1;
  P.x0 = x0;
  P.y0 = 0.0;
  P.dx = (x1 - x0) / (double)nx;
  P.dy = 1.0;
  P.gamma = gamma;
  for (int s = 0; s < 2; ++s) {
    P.bc[s] = bc_kind[s];
    for (int q = 0; q < 4; ++q) P.inflow[s][q] = inflow ? inflow[s][q] : 0.0;
  }
  P.eps = 1e-6;
  P.gam[0] = 0.994;
  P.gam[1] = 0.003;
  P.gam[2] = 0.003;
  P.flag_mode = flag_mode;
  shweno::finalize_params(P);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  noalloc_begin_kernel<<<1, 1, 0, st>>>(ctl, t, dt);
  shweno::launch_step1d(P, ctl, state_in, state_in, state_out, state_out, nullptr, FH, WE, st, nullptr);
  if (cudaGetLastError() != cudaSuccess) return SHWENO_E_CUDA;
  Ctl h;
  if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SHWENO_E_CUDA;
  return h.err == shweno::ERR_NONE ? SHWENO_OK : SHWENO_E_NONPHYSICAL;
}
