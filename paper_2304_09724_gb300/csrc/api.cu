// C ABI of the ADER-SHWENO library: handles, state transfer, the device-resident time loop.
//
// Time stepping protocol.  A device control block (Ctl) holds the committed time, step count,
// the CFL rate of the committed state and a sticky error word.  One step is
//   begin_step (1 thread): dt from the fixed value or from cfl / rate, clipped to t_final;
//   the step kernels (read Ctl, never write it except the error word and the next rate);
//   end_step (1 thread): commit t += dt, nsteps += 1, rate_cur = rate_next, unless an error
//   was raised, in which case nothing is committed.
// The committed state always lives in buffer nsteps % 2, so a failed step leaves the previous
// state in place and no copy is needed.  All launches of a step have fixed arguments, so a run
// of several steps is captured once as a CUDA graph and replayed; the host only polls Ctl.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/shweno.h"
#include "shweno_kernels.h"

using shweno::Ctl;
using shweno::Params;

namespace {

shweno_alloc_fn g_alloc = nullptr;
shweno_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
std::string g_create_error;

void* dev_alloc(size_t bytes) {
  if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_alloc_ctx);
  else cudaFree(p);
}

__global__ void config_kernel(Ctl* c, int mode, double t_final, double cfl, double dt_fixed) {
  c->mode = mode;
  c->t_final = t_final;
  c->cfl = cfl;
  c->dt_fixed = dt_fixed;
  c->err = shweno::ERR_NONE;
  c->active = 0;
}
__global__ void reset_kernel(Ctl* c, double t) {
  c->t = t;
  c->dt = 0.0;
  c->nsteps = 0;
  c->err_step = -1;
  c->err = shweno::ERR_NONE;
  c->active = 0;
  c->rate_cur = 0ull;
  c->rate_next = 0ull;
  c->mode = 0;
}
__global__ void begin_step_kernel(Ctl* c) {
  if (c->err != shweno::ERR_NONE) { c->active = 0; return; }
  double dt;
  if (c->mode == 0) {
    dt = c->dt_fixed;
  } else {
    if (!(c->t < c->t_final)) { c->active = 0; return; }
    const double rate = __longlong_as_double((long long)c->rate_cur);
    dt = c->cfl / rate;
    if (!(dt <= c->t_final - c->t)) dt = c->t_final - c->t;
  }
  c->dt = dt;
  c->rate_next = 0ull;
  c->active = 1;
}
__global__ void end_step_kernel(Ctl* c) {
  if (!c->active) return;
  c->active = 0;
  if (c->err != shweno::ERR_NONE) { c->err_step = c->nsteps; return; }
  c->t = c->t + c->dt;
  c->nsteps += 1;
  c->rate_cur = c->rate_next;
}
__global__ void rate_kernel(Params P, Ctl* ctl, const double* s0, const double* s1) {
  __shared__ double red[32];
  const size_t cells = (size_t)P.nx * (P.dim == 2 ? P.ny : 1);
  const double* st = (ctl->nsteps & 1) ? s1 : s0;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (c < cells) {
    double W[4];
    for (int q = 0; q < P.ncomp; ++q) W[q] = st[q * cells + c];
    if (!shweno::cell_physical(P, W)) atomicCAS(&ctl->err, shweno::ERR_NONE, shweno::ERR_NONPHYSICAL);
    else r = shweno::cell_rate(P, W);
  }
  shweno::block_max_rate(r, &ctl->rate_cur, red);
}
__global__ void zero_rate_kernel(Ctl* c) { c->rate_cur = 0ull; }

}  // namespace

namespace shweno {
void launch_begin_step(Ctl* ctl, cudaStream_t st) { begin_step_kernel<<<1, 1, 0, st>>>(ctl); }
void launch_end_step(Ctl* ctl, cudaStream_t st) { end_step_kernel<<<1, 1, 0, st>>>(ctl); }
void launch_rate(const Params& P, Ctl* ctl, const double* s0, const double* s1, cudaStream_t st) {
  const size_t cells = (size_t)P.nx * (P.dim == 2 ? P.ny : 1);
  zero_rate_kernel<<<1, 1, 0, st>>>(ctl);
  rate_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(P, ctl, s0, s1);
}
}  // namespace shweno

struct shweno_handle {
  Params P{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t cells = 0, nfields = 0, state_doubles = 0;
  double* buf[2] = {nullptr, nullptr};
  double* scratch = nullptr;
  shweno::Scratch2D S{};
  double* FH = nullptr;
  double* WE = nullptr;
  uint8_t* flags = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;  // pinned, two slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // profiling: events around every kernel of every timed step
  bool timing = false;
  // learned flag
  bool learned = false;
  float* net = nullptr;
  uint8_t* raw_flags = nullptr;
  float logit_thr = 0.f;
  std::vector<cudaEvent_t> tev;
  size_t tev_used = 0;
  int64_t timed_steps = 0;
  std::string err;
};

namespace {

shweno_status fail(shweno_handle* h, shweno_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}
shweno_status cuda_fail(shweno_handle* h, cudaError_t e, const char* where) {
  return fail(h, SHWENO_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(h, call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);          \
  } while (0)

int kernel_count(const shweno_handle* h) {
  return h->P.dim == 1 ? shweno::kKernels1D : shweno::kKernels2D + (h->learned ? 1 : 0);
}

// Enqueues one step; with timing on, records events around each step kernel.
cudaError_t enqueue_step(shweno_handle* h) {
  cudaEvent_t* ev = nullptr;
  if (h->timing) {
    const size_t need = h->tev_used + kernel_count(h) + 1;
    while (h->tev.size() < need) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      h->tev.push_back(e);
    }
    ev = &h->tev[h->tev_used];
    h->tev_used = need;
    ++h->timed_steps;
  }
  shweno::launch_begin_step(h->ctl, h->stream);
  if (h->P.dim == 1) {
    shweno::launch_step1d(h->P, h->ctl, h->buf[0], h->buf[1], h->buf[0], h->buf[1], h->flags,
                          h->FH, h->WE, h->stream, ev);
  } else {
    if (h->learned) {
      if (ev) cudaEventRecord(ev[0], h->stream);
      shweno::launch_infer2d(h->P, h->ctl, h->buf[0], h->buf[1], h->net, h->logit_thr, h->raw_flags,
                             h->flags, h->stream);
      if (ev) ++ev;
    }
    shweno::launch_step2d(h->P, h->ctl, h->buf[0], h->buf[1], h->buf[0], h->buf[1], h->flags,
                          h->S, h->stream, ev);
  }
  shweno::launch_end_step(h->ctl, h->stream);
  return cudaGetLastError();
}

shweno_status read_ctl(shweno_handle* h, Ctl* out) {
  CK(h, cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  *out = h->ctl_host[0];
  return SHWENO_OK;
}

shweno_status build_graph(shweno_handle* h, int steps) {
  if (h->graph && h->graph_steps == steps) return SHWENO_OK;
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  cudaGraph_t g = nullptr;
  CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const bool timing = h->timing;
  h->timing = false;
  for (int s = 0; s < steps; ++s) enqueue_step(h);
  h->timing = timing;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  h->graph_steps = steps;
  return SHWENO_OK;
}

bool valid_bc(int k, int dim, int side) {
  if (k < 0 || k > 5) return false;
  if (k == SHWENO_BC_DMR_BOTTOM) return dim == 2 && side == 2;
  if (k == SHWENO_BC_DMR_TOP) return dim == 2 && side == 3;
  return true;
}

}  // namespace

namespace shweno {
bool handle_view(shweno_handle* h, HandleView* v) {
  if (!h || !v) return false;
  v->P = h->P;
  v->ctl = h->ctl;
  v->buf[0] = h->buf[0];
  v->buf[1] = h->buf[1];
  v->flags = h->flags;
  v->S = h->S;
  v->net = h->net;
  v->raw = h->raw_flags;
  v->flags_out = h->flags;
  v->logit_thr = h->logit_thr;
  v->learned = h->learned ? 1 : 0;
  v->stream = h->stream;
  return true;
}
}  // namespace shweno

extern "C" {

shweno_status shweno_set_allocator(shweno_alloc_fn alloc, shweno_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(nullptr, SHWENO_E_INVALID, "allocator and release must both be set or both NULL");
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return SHWENO_OK;
}

const char* shweno_last_error(const shweno_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

shweno_status shweno_create(const shweno_grid* grid, double gamma, const shweno_bc* bc,
                            const shweno_opts* opts, void* cuda_stream, shweno_handle** out) {
  if (!grid || !bc || !out) return fail(nullptr, SHWENO_E_INVALID, "null argument");
  *out = nullptr;
  const int dim = grid->dim;
  if (dim != 1 && dim != 2) return fail(nullptr, SHWENO_E_INVALID, "dim must be 1 or 2");
  if (grid->eq != SHWENO_BURGERS && grid->eq != SHWENO_EULER)
    return fail(nullptr, SHWENO_E_INVALID, "unknown equation");
  if (grid->nx < 4 || (dim == 2 && grid->ny < 4) || grid->nx > (1 << 26) || (dim == 2 && grid->ny > (1 << 26)))
    return fail(nullptr, SHWENO_E_INVALID, "nx, ny must be in [4, 2^26]");
  if (dim == 2 && (size_t)grid->nx * (size_t)grid->ny > ((size_t)1 << 31))
    return fail(nullptr, SHWENO_E_INVALID, "2D meshes are limited to 2^31 cells");
  if (!(grid->x1 > grid->x0) || (dim == 2 && !(grid->y1 > grid->y0)))
    return fail(nullptr, SHWENO_E_INVALID, "empty domain");
  if (grid->eq == SHWENO_EULER && !(gamma > 1.0)) return fail(nullptr, SHWENO_E_INVALID, "gamma must be > 1");
  for (int s = 0; s < (dim == 2 ? 4 : 2); ++s) {
    if (!valid_bc(bc->kind[s], dim, s)) return fail(nullptr, SHWENO_E_INVALID, "invalid boundary condition");
    if (grid->eq == SHWENO_BURGERS && (bc->kind[s] == SHWENO_BC_DMR_BOTTOM || bc->kind[s] == SHWENO_BC_DMR_TOP))
      return fail(nullptr, SHWENO_E_INVALID, "the double Mach reflection boundaries carry Euler states");
  }
  for (int a = 0; a < dim; ++a)
    if ((bc->kind[2 * a] == SHWENO_BC_PERIODIC) != (bc->kind[2 * a + 1] == SHWENO_BC_PERIODIC))
      return fail(nullptr, SHWENO_E_INVALID, "periodic boundaries must be paired");
  shweno_opts o{0, 1e-6, {0.994, 0.003, 0.003}, 0, 0};
  if (opts) o = *opts;
  if (o.flag_mode < 0 || o.flag_mode > 2 || o.charwise < 0 || o.charwise > 1 || o.quintic < 0 ||
      o.quintic > 1 || !(o.eps > 0.0) ||
      !(o.gam[0] > 0 && o.gam[1] > 0 && o.gam[2] > 0) ||
      std::fabs(o.gam[0] + o.gam[1] + o.gam[2] - 1.0) > 1e-12)
    return fail(nullptr, SHWENO_E_INVALID, "invalid options");

  shweno_handle* h = new (std::nothrow) shweno_handle();
  if (!h) return fail(nullptr, SHWENO_E_NOMEM, "host allocation failed");
  Params& P = h->P;
  P.dim = dim;
  P.eq = grid->eq;
  P.ncomp = grid->eq == SHWENO_BURGERS ? 1 : (dim == 1 ? 3 : 4);
  P.nx = (int32_t)grid->nx;
  P.ny = dim == 2 ? (int32_t)grid->ny : 1;
  P.x0 = grid->x0;
  P.y0 = dim == 2 ? grid->y0 : 0.0;
  P.dx = (grid->x1 - grid->x0) / grid->nx;
  P.dy = dim == 2 ? (grid->y1 - grid->y0) / grid->ny : 1.0;
  P.gamma = gamma;
  for (int s = 0; s < 4; ++s) {
    P.bc[s] = (s < 2 || dim == 2) ? bc->kind[s] : 0;
    for (int q = 0; q < 4; ++q) P.inflow[s][q] = bc->inflow[s][q];
  }
  P.eps = o.eps;
  for (int k = 0; k < 3; ++k) P.gam[k] = o.gam[k];
  P.flag_mode = o.flag_mode;
  P.charwise = grid->eq == SHWENO_EULER ? o.charwise : 0;
  P.quintic = o.quintic;
  shweno::finalize_params(P);

  h->cells = (size_t)P.nx * P.ny;
  h->nfields = dim == 2 ? 4 : 2;
  h->state_doubles = h->nfields * P.ncomp * h->cells;
  auto bail = [&](shweno_status s, const std::string& m) {
    g_create_error = m;
    shweno_destroy(h);
    return s;
  };
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreate(&h->stream) != cudaSuccess) return bail(SHWENO_E_CUDA, "cudaStreamCreate failed");
    h->own_stream = true;
  }
  for (int b = 0; b < 2; ++b) {
    h->buf[b] = (double*)dev_alloc(h->state_doubles * sizeof(double));
    if (!h->buf[b]) return bail(SHWENO_E_NOMEM, "device allocation of the state failed");
  }
  const size_t scr = dim == 2 ? shweno::scratch2d_doubles(P) : 2 * (size_t)P.ncomp * (P.nx + 1);
  h->scratch = (double*)dev_alloc(scr * sizeof(double));
  if (!h->scratch) return bail(SHWENO_E_NOMEM, "device allocation of the step scratch failed");
  if (dim == 2) {
    h->S = shweno::carve_scratch2d(P, h->scratch);
    const cudaError_t ea = shweno::init_kernels2d();
    if (ea != cudaSuccess) {
      cudaGetLastError();
      return bail(SHWENO_E_CUDA, std::string("setting the face kernels' shared memory limit failed: ") +
                                     cudaGetErrorString(ea));
    }
  }
  else { h->FH = h->scratch; h->WE = h->scratch + (size_t)P.ncomp * (P.nx + 1); }
  h->ctl = (Ctl*)dev_alloc(sizeof(Ctl));
  if (!h->ctl) return bail(SHWENO_E_NOMEM, "device allocation of the control block failed");
  if (cudaMallocHost(&h->ctl_host, 2 * sizeof(Ctl)) != cudaSuccess) return bail(SHWENO_E_CUDA, "cudaMallocHost failed");
  for (int k = 0; k < 2; ++k)
    if (cudaEventCreateWithFlags(&h->ev[k], cudaEventDisableTiming) != cudaSuccess)
      return bail(SHWENO_E_CUDA, "cudaEventCreate failed");
  if (cudaMemsetAsync(h->buf[0], 0, h->state_doubles * sizeof(double), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->buf[1], 0, h->state_doubles * sizeof(double), h->stream) != cudaSuccess)
    return bail(SHWENO_E_CUDA, "cudaMemsetAsync failed");
  reset_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 0.0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bail(SHWENO_E_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  *out = h;
  return SHWENO_OK;
}

shweno_status shweno_destroy(shweno_handle* h) {
  if (!h) return SHWENO_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (int b = 0; b < 2; ++b) dev_free(h->buf[b]);
  dev_free(h->scratch);
  dev_free(h->flags);
  dev_free(h->raw_flags);
  dev_free(h->net);
  dev_free(h->ctl);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k)
    if (h->ev[k]) cudaEventDestroy(h->ev[k]);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return SHWENO_OK;
}

shweno_status shweno_set_state(shweno_handle* h, const double* W, const double* V, const double* Y,
                               const double* Z, double t, int on_device) {
  if (!h) return SHWENO_E_INVALID;
  if (!W || !V || (h->P.dim == 2 && (!Y || !Z))) return fail(h, SHWENO_E_INVALID, "null state array");
  if (!std::isfinite(t)) return fail(h, SHWENO_E_INVALID, "time must be finite");
  const size_t n = (size_t)h->P.ncomp * h->cells;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const double* src[4] = {W, V, Y, Z};
  for (size_t f = 0; f < h->nfields; ++f)
    CK(h, cudaMemcpyAsync(h->buf[0] + f * n, src[f], n * sizeof(double), k, h->stream));
  reset_kernel<<<1, 1, 0, h->stream>>>(h->ctl, t);
  CK(h, cudaGetLastError());
  return SHWENO_OK;
}

shweno_status shweno_get_state(shweno_handle* h, double* W, double* V, double* Y, double* Z,
                               int on_device) {
  if (!h) return SHWENO_E_INVALID;
  if (!W || !V || (h->P.dim == 2 && (!Y || !Z))) return fail(h, SHWENO_E_INVALID, "null state array");
  Ctl c;
  shweno_status s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  const double* b = h->buf[c.nsteps & 1];
  const size_t n = (size_t)h->P.ncomp * h->cells;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* dst[4] = {W, V, Y, Z};
  for (size_t f = 0; f < h->nfields; ++f)
    CK(h, cudaMemcpyAsync(dst[f], b + f * n, n * sizeof(double), k, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return SHWENO_OK;
}

shweno_status shweno_get_time(shweno_handle* h, double* t_out, int64_t* nsteps_out) {
  if (!h) return SHWENO_E_INVALID;
  Ctl c;
  shweno_status s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  if (t_out) *t_out = c.t;
  if (nsteps_out) *nsteps_out = c.nsteps;
  return SHWENO_OK;
}

shweno_status shweno_set_flags(shweno_handle* h, const uint8_t* flags, int on_device) {
  if (!h || !flags) return fail(h, SHWENO_E_INVALID, "null argument");
  if (!h->flags) {
    h->flags = (uint8_t*)dev_alloc(h->cells);
    if (!h->flags) return fail(h, SHWENO_E_NOMEM, "device allocation of the flags failed");
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; h->graph_steps = 0; }
  }
  CK(h, cudaMemcpyAsync(h->flags, flags, h->cells, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream));
  return SHWENO_OK;
}

shweno_status shweno_step(shweno_handle* h, double dt) {
  if (!h) return SHWENO_E_INVALID;
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, SHWENO_E_INVALID, "dt must be positive and finite");
  if (h->P.flag_mode == shweno::FLAG_PER_CELL && !h->flags)
    return fail(h, SHWENO_E_STATE, "flag_mode 2 needs flags (shweno_set_flags)");
  config_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 0, 0.0, 0.0, dt);
  CK(h, enqueue_step(h));
  Ctl c;
  shweno_status s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  if (c.err == shweno::ERR_NONPHYSICAL)
    return fail(h, SHWENO_E_NONPHYSICAL, "the step produced a non-physical state; it was not committed");
  return SHWENO_OK;
}

shweno_status shweno_cfl_dt(shweno_handle* h, double cfl, double* dt_out, double* rate_out) {
  if (!h || !(cfl > 0.0)) return fail(h, SHWENO_E_INVALID, "cfl must be positive");
  config_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 0, 0.0, cfl, 0.0);
  shweno::launch_rate(h->P, h->ctl, h->buf[0], h->buf[1], h->stream);
  CK(h, cudaGetLastError());
  Ctl c;
  shweno_status s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  if (c.err != shweno::ERR_NONE) return fail(h, SHWENO_E_NONPHYSICAL, "the state is not physical");
  double rate;
  std::memcpy(&rate, &c.rate_cur, sizeof(double));
  if (rate_out) *rate_out = rate;
  if (dt_out) *dt_out = cfl / rate;
  return SHWENO_OK;
}

shweno_status shweno_run(shweno_handle* h, double t_final, double cfl, double* t_out,
                         int64_t* nsteps_out) {
  if (!h) return SHWENO_E_INVALID;
  if (!(cfl > 0.0) || !std::isfinite(t_final)) return fail(h, SHWENO_E_INVALID, "invalid t_final or cfl");
  if (h->P.flag_mode == shweno::FLAG_PER_CELL && !h->flags)
    return fail(h, SHWENO_E_STATE, "flag_mode 2 needs flags (shweno_set_flags)");
  config_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 1, t_final, cfl, 0.0);
  shweno::launch_rate(h->P, h->ctl, h->buf[0], h->buf[1], h->stream);
  CK(h, cudaGetLastError());
  Ctl c;
  shweno_status s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  if (c.err != shweno::ERR_NONE) return fail(h, SHWENO_E_NONPHYSICAL, "the initial state is not physical");
  const int64_t n0 = c.nsteps;
  if (!(c.t < t_final)) {
    if (t_out) *t_out = c.t;
    if (nsteps_out) *nsteps_out = 0;
    return SHWENO_OK;
  }
  // steps per graph launch: enough to amortise launches, few enough to stop soon after t_final
  const double work = (double)h->cells * (h->P.dim == 2 ? 64.0 : 1.0);
  const int chunk = work > 4e6 ? 2 : (work > 2.5e5 ? 8 : 32);
  s = build_graph(h, chunk);
  if (s != SHWENO_OK) return s;
  if (h->timing) {  // profiling: one step at a time with events, checked every chunk
    for (;;) {
      for (int k = 0; k < chunk; ++k) CK(h, enqueue_step(h));
      s = read_ctl(h, &c);
      if (s != SHWENO_OK) return s;
      if (c.err != shweno::ERR_NONE || !(c.t < t_final)) break;
    }
    if (t_out) *t_out = c.t;
    if (nsteps_out) *nsteps_out = c.nsteps - n0;
    if (c.err == shweno::ERR_NONPHYSICAL)
      return fail(h, SHWENO_E_NONPHYSICAL, "a step produced a non-physical state; stopped at the last good one");
    return SHWENO_OK;
  }
  // two graph launches in flight; the control block of the older one is checked
  int slot = 0;
  bool pending[2] = {false, false};
  for (;;) {
    CK(h, cudaGraphLaunch(h->graph, h->stream));
    CK(h, cudaMemcpyAsync(&h->ctl_host[slot], h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaEventRecord(h->ev[slot], h->stream));
    pending[slot] = true;
    slot ^= 1;
    if (pending[slot]) {
      CK(h, cudaEventSynchronize(h->ev[slot]));
      pending[slot] = false;
      c = h->ctl_host[slot];
      if (c.err != shweno::ERR_NONE || !(c.t < t_final)) break;
    }
  }
  CK(h, cudaStreamSynchronize(h->stream));
  s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  if (t_out) *t_out = c.t;
  if (nsteps_out) *nsteps_out = c.nsteps - n0;
  if (c.err == shweno::ERR_NONPHYSICAL)
    return fail(h, SHWENO_E_NONPHYSICAL, "a step produced a non-physical state; stopped at the last good one");
  return SHWENO_OK;
}

shweno_status shweno_advance(shweno_handle* h, int64_t nsteps, double cfl) {
  if (!h) return SHWENO_E_INVALID;
  if (nsteps < 0 || !(cfl > 0.0)) return fail(h, SHWENO_E_INVALID, "invalid nsteps or cfl");
  if (h->P.flag_mode == shweno::FLAG_PER_CELL && !h->flags)
    return fail(h, SHWENO_E_STATE, "flag_mode 2 needs flags (shweno_set_flags)");
  config_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 1, INFINITY, cfl, 0.0);
  shweno::launch_rate(h->P, h->ctl, h->buf[0], h->buf[1], h->stream);
  CK(h, cudaGetLastError());
  if (h->timing) {
    for (int64_t k = 0; k < nsteps; ++k) CK(h, enqueue_step(h));
    return SHWENO_OK;
  }
  const int G = 4;
  int64_t k = 0;
  if (nsteps >= G) {  // fewer steps go out as plain launches: no graph to capture for them
    shweno_status s = build_graph(h, G);
    if (s != SHWENO_OK) return s;
    for (; k + G <= nsteps; k += G) CK(h, cudaGraphLaunch(h->graph, h->stream));
  }
  for (; k < nsteps; ++k) CK(h, enqueue_step(h));
  return SHWENO_OK;
}

shweno_status shweno_sync(shweno_handle* h) {
  if (!h) return SHWENO_E_INVALID;
  Ctl c;
  shweno_status s = read_ctl(h, &c);
  if (s != SHWENO_OK) return s;
  if (c.err == shweno::ERR_NONPHYSICAL)
    return fail(h, SHWENO_E_NONPHYSICAL, "a step produced a non-physical state; stopped at the last good one");
  return SHWENO_OK;
}

shweno_status shweno_set_timing(shweno_handle* h, int enable) {
  if (!h) return SHWENO_E_INVALID;
  h->timing = enable != 0;
  return SHWENO_OK;
}

shweno_status shweno_get_timing(shweno_handle* h, double* ms, int max_kernels, int* nkernels,
                                int64_t* nsteps) {
  if (!h) return SHWENO_E_INVALID;
  CK(h, cudaStreamSynchronize(h->stream));
  const int nk = kernel_count(h);
  if (nkernels) *nkernels = nk;
  if (nsteps) *nsteps = h->timed_steps;
  for (int k = 0; k < max_kernels && ms; ++k) ms[k] = 0.0;
  for (size_t base = 0; base + nk + 1 <= h->tev_used; base += nk + 1)
    for (int k = 0; k < nk; ++k) {
      float t = 0.f;
      CK(h, cudaEventElapsedTime(&t, h->tev[base + k], h->tev[base + k + 1]));
      if (k < max_kernels && ms) ms[k] += t;
    }
  h->tev_used = 0;
  h->timed_steps = 0;
  return SHWENO_OK;
}

const char* shweno_kernel_name(const shweno_handle* h, int k) {
  static const char* n1[] = {"face1d", "update1d"};
  static const char* n2[] = {"coef2d", "xface2d", "yface2d", "update2d"};
  if (!h || k < 0 || k >= kernel_count(h)) return "";
  if (h->P.dim == 1) return n1[k];
  if (h->learned) return k == 0 ? "flags2d" : n2[k - 1];
  return n2[k];
}

shweno_status shweno_flag_features(shweno_handle* h, float* out) {
  if (!h || !out) return fail(h, SHWENO_E_INVALID, "null argument");
  if (h->P.dim != 2 || h->P.eq != SHWENO_EULER) return fail(h, SHWENO_E_STATE, "features need a 2D Euler handle");
  shweno::launch_features2d(h->P, h->ctl, h->buf[0], h->buf[1], out, h->stream);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->stream));
  return SHWENO_OK;
}

shweno_status shweno_weight_deviation(shweno_handle* h, double* out) {
  if (!h || !out) return fail(h, SHWENO_E_INVALID, "null argument");
  if (h->P.dim != 2 || h->P.eq != SHWENO_EULER) return fail(h, SHWENO_E_STATE, "needs a 2D Euler handle");
  shweno::launch_wdev2d(h->P, h->ctl, h->buf[0], h->buf[1], out, h->stream);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->stream));
  return SHWENO_OK;
}

shweno_status shweno_face_deviation(shweno_handle* h, double floor_rel, double* out) {
  if (!h || !out) return fail(h, SHWENO_E_INVALID, "null argument");
  if (!(floor_rel >= 1e-9) || !std::isfinite(floor_rel)) return fail(h, SHWENO_E_INVALID, "floor_rel must be >= 1e-9");
  if (h->P.dim != 2 || h->P.eq != SHWENO_EULER) return fail(h, SHWENO_E_STATE, "needs a 2D Euler handle");
  shweno::launch_fdev2d(h->P, h->ctl, h->buf[0], h->buf[1], floor_rel, out, h->stream);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->stream));
  return SHWENO_OK;
}

shweno_status shweno_mlp_forward(const float* params, const float* x, int64_t n, float* prob,
                                 void* cuda_stream) {
  if (!params || (n > 0 && (!x || !prob)) || n < 0) return SHWENO_E_INVALID;
  shweno::mlp_forward(params, x, n, prob, (cudaStream_t)cuda_stream);
  return cudaGetLastError() == cudaSuccess ? SHWENO_OK : SHWENO_E_CUDA;
}

shweno_status shweno_mlp_grad(const float* params, const float* x, const float* y, int64_t n,
                              float pos_weight, float* grad, float* loss, void* cuda_stream) {
  if (!params || !grad || !loss || n <= 0 || !x || !y) return SHWENO_E_INVALID;
  return shweno::mlp_grad(params, x, y, n, pos_weight, grad, loss, (cudaStream_t)cuda_stream) == cudaSuccess
             ? SHWENO_OK : SHWENO_E_CUDA;
}

shweno_status shweno_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t step,
                              float lr, float beta1, float beta2, float eps, void* cuda_stream) {
  if (!params || !grad || !m || !v || step < 1) return SHWENO_E_INVALID;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
  shweno::mlp_adam(params, grad, m, v, lr, beta1, beta2, eps, bc1, bc2, (cudaStream_t)cuda_stream);
  return cudaGetLastError() == cudaSuccess ? SHWENO_OK : SHWENO_E_CUDA;
}

shweno_status shweno_set_flag_net(shweno_handle* h, const float* params, double threshold,
                                  int on_device) {
  if (!h || !params) return fail(h, SHWENO_E_INVALID, "null argument");
  if (!(threshold > 0.0 && threshold < 1.0)) return fail(h, SHWENO_E_INVALID, "threshold must be in (0, 1)");
  if (h->P.dim != 2 || h->P.eq != SHWENO_EULER || h->P.flag_mode != shweno::FLAG_PER_CELL)
    return fail(h, SHWENO_E_STATE, "the learned flag needs a 2D Euler handle created with flag_mode 2");
  if (!h->net) {
    h->net = (float*)dev_alloc(SHWENO_FLAG_PARAMS * sizeof(float));
    h->raw_flags = (uint8_t*)dev_alloc(h->cells);
    if (!h->flags) h->flags = (uint8_t*)dev_alloc(h->cells);
    if (!h->net || !h->raw_flags || !h->flags) return fail(h, SHWENO_E_NOMEM, "device allocation of the flag network failed");
  }
  CK(h, cudaMemcpyAsync(h->net, params, SHWENO_FLAG_PARAMS * sizeof(float),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  h->logit_thr = (float)std::log(threshold / (1.0 - threshold));
  h->learned = true;
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; h->graph_steps = 0; }
  return SHWENO_OK;
}

shweno_status shweno_get_flags(shweno_handle* h, uint8_t* out, int on_device) {
  if (!h || !out) return fail(h, SHWENO_E_INVALID, "null argument");
  if (!h->flags) return fail(h, SHWENO_E_STATE, "no flags yet");
  CK(h, cudaMemcpyAsync(out, h->flags, h->cells, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return SHWENO_OK;
}

}  // extern "C"
