// One ADER-SHWENO time step in one space dimension (Section 2; Section 4 Steps 1-5).
//   face1d:   one thread per interface x_{f-1/2}: SHWENO reconstruction of both neighbours
//             (Section 2.4 reading), leading term (exact Burgers / HLLC, Eq. 2.5), linearised
//             derivative Riemann problems (Eq. 2.8), Cauchy-Kovalevskaya (Eq. 2.6), Lobatto
//             time quadrature of the flux (Eq. 2.9, Remark 2) and the state at t_{n+1}
//             (Eq. 2.12, Remark 1).  Writes F-hat and W(t_{n+1}) per face.  Instantiated for
//             reading R1 (quartic p1) and the R1' option (quintic p1).
//   update1d: one thread per cell: Eq. (2.2) for the averages, Eq. (2.11) for the derivative
//             averages; fused max characteristic rate of the new state (next CFL step) and the
//             physical-state check.
#include <cuda_runtime.h>

#include "shweno_kernels.h"
#include "step1d_items.cuh"

namespace shweno {

template <int NC, bool Q>
__global__ void __launch_bounds__(128) face1d_kernel(Params P, const Ctl* __restrict__ ctl,
                                                     const double* s0, const double* s1,
                                                     const uint8_t* __restrict__ flag,
                                                     double* __restrict__ FH,
                                                     double* __restrict__ WE) {
  if (!ctl->active) return;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;  // face between cells f-1 and f
  if (f > P.nx) return;
  const StepView sv = step_view(ctl);
  double Fh[NC], We[NC];
  face1d_point<NC, Q>(P, sv.odd ? s1 : s0, flag, f, sv.t, sv.dt, Fh, We);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    FH[(size_t)q * (P.nx + 1) + f] = Fh[q];
    WE[(size_t)q * (P.nx + 1) + f] = We[q];
  }
}

__global__ void __launch_bounds__(256) update1d_kernel(Params P, Ctl* __restrict__ ctl,
                                                       const double* s0, const double* s1,
                                                       double* o0, double* o1,
                                                       const double* __restrict__ FH,
                                                       const double* __restrict__ WE) {
  __shared__ double red[32];
  if (!ctl->active) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool odd = ctl->nsteps & 1;
  const double* st = odd ? s1 : s0;
  double* out = odd ? o0 : o1;
  const double dt = ctl->dt;
  const int nc = P.ncomp, N = P.nx;
  double rate = 0.0;
  if (j < N) {
    double Wn[4];
    for (int q = 0; q < nc; ++q) {
      const size_t fo = (size_t)q * (N + 1) + j;
      Wn[q] = st[(size_t)q * N + j] - dt / P.dx * (FH[fo + 1] - FH[fo]);
      out[(size_t)q * N + j] = Wn[q];
      out[(size_t)(nc + q) * N + j] = (WE[fo + 1] - WE[fo]) * P.idx;  // 1 / dx from the host
    }
    if (!cell_physical(P, Wn)) atomicCAS(&ctl->err, ERR_NONE, ERR_NONPHYSICAL);
    else rate = cell_rate(P, Wn);
  }
  block_max_rate(rate, &ctl->rate_next, red);
}

void launch_step1d(const Params& P, Ctl* ctl, const double* s0, const double* s1, double* o0,
                   double* o1, const uint8_t* flag, double* FH, double* WE, cudaStream_t st,
                   cudaEvent_t* ev) {
  const int nf = P.nx + 1;
  const int b = 128;
  if (ev) cudaEventRecord(ev[0], st);
  const dim3 g((nf + b - 1) / b);
  if (P.ncomp == 1) {
    if (P.quintic) face1d_kernel<1, true><<<g, b, 0, st>>>(P, ctl, s0, s1, flag, FH, WE);
    else face1d_kernel<1, false><<<g, b, 0, st>>>(P, ctl, s0, s1, flag, FH, WE);
  } else {
    if (P.quintic) face1d_kernel<3, true><<<g, b, 0, st>>>(P, ctl, s0, s1, flag, FH, WE);
    else face1d_kernel<3, false><<<g, b, 0, st>>>(P, ctl, s0, s1, flag, FH, WE);
  }
  if (ev) cudaEventRecord(ev[1], st);
  update1d_kernel<<<(P.nx + 255) / 256, 256, 0, st>>>(P, ctl, s0, s1, o0, o1, FH, WE);
  if (ev) cudaEventRecord(ev[2], st);
}

}  // namespace shweno
