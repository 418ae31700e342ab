// One ADER-SHWENO time step in one space dimension (Section 2; Section 4 Steps 1-5).
//   face1d:   one thread per interface x_{f-1/2}: SHWENO reconstruction of both neighbours
//             (Section 2.4 reading), leading term (exact Burgers / HLLC, Eq. 2.5), linearised
//             derivative Riemann problems (Eq. 2.8), Cauchy-Kovalevskaya (Eq. 2.6), Lobatto
//             time quadrature of the flux (Eq. 2.9, Remark 2) and the state at t_{n+1}
//             (Eq. 2.12, Remark 1).  Writes F-hat and W(t_{n+1}) per face.
//   update1d: one thread per cell: Eq. (2.2) for the averages, Eq. (2.11) for the derivative
//             averages; fused max characteristic rate of the new state (next CFL step) and the
//             physical-state check.
#include <cuda_runtime.h>

#include "ck_generated.cuh"
#include "shweno_device.cuh"
#include "shweno_kernels.h"

namespace shweno {

// Normalised Taylor coefficients e[m] of the polynomial sum C[k] xi^k about xi0, m <= mmax
// (repeated synthetic division).
__device__ __forceinline__ void taylor_shift(double e[5], double xi0, int mmax) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i > mmax) break;
#pragma unroll
    for (int k = 3; k >= 0; --k)
      if (k >= i) e[k] += xi0 * e[k + 1];
  }
}

template <int NC>
__global__ void __launch_bounds__(128) face1d_kernel(Params P, const Ctl* __restrict__ ctl,
                                                     const double* s0, const double* s1,
                                                     const uint8_t* __restrict__ flag,
                                                     double* __restrict__ FH,
                                                     double* __restrict__ WE) {
  if (!ctl->active) return;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;  // face between cells f-1 and f
  if (f > P.nx) return;
  const double* st = (ctl->nsteps & 1) ? s1 : s0;
  const double dt = ctl->dt, t = ctl->t, g = P.gamma;

  double a[NC][25], dR[NC][25];
  double WL0[NC], WR0[NC];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int cell = f - 1 + side;
    const int nonlinear = cell_flag(P, flag, cell, 0);
    const double xi0 = side == 0 ? 0.5 : -0.5;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double Wm = fetch(P, st, 0, q, cell - 1, 0, t);
      const double W0 = fetch(P, st, 0, q, cell, 0, t);
      const double Wp = fetch(P, st, 0, q, cell + 1, 0, t);
      const double vm = P.dx * fetch(P, st, 1, q, cell - 1, 0, t);
      const double vp = P.dx * fetch(P, st, 1, q, cell + 1, 0, t);
      double c[5], e[5];
      p1_coeffs(Wm, W0, Wp, vm, vp, c);
      const Mix mx = shweno_mix(P, Wm, W0, Wp, c, nonlinear);
      mix_coeffs(mx, Wm, W0, Wp, c, e);
      taylor_shift(e, xi0, 4);
#pragma unroll
      for (int m = 0; m < 5; ++m) (side == 0 ? a : dR)[q][m * 5] = e[m];
      (side == 0 ? WL0 : WR0)[q] = e[0];
    }
  }
  // leading term and the linearised problems for the derivatives
  double Ws[NC];
  if constexpr (NC == 1) Ws[0] = burgers_godunov(WL0[0], WR0[0]);
  else hllc_state<NC>(WL0, WR0, g, 0, Ws);
  Upwinder<NC> U;
  U.setup(Ws, g, 0, NC == 1 ? fmax(fabs(WL0[0]), fabs(WR0[0])) : 0.0);
#pragma unroll
  for (int m = 1; m < 5; ++m) {
    double dl[NC], dr[NC], o[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { dl[q] = a[q][m * 5]; dr[q] = dR[q][m * 5]; }
    U.apply(dl, dr, o);
#pragma unroll
    for (int q = 0; q < NC; ++q) a[q][m * 5] = o[q];
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) a[q][0] = Ws[q];
  double cx[5][4], cy[5][4];
  const double ih = 1.0 / P.dx;
#pragma unroll
  for (int m = 0; m < 5; ++m)
#pragma unroll
    for (int k = 0; k < 4; ++k) { cx[m][k] = (m + 1) * ih / (k + 1); cy[m][k] = 0.0; }
  double tc[NC][5];
  if constexpr (NC == 1) ck_burgers1d(a, tc, cx, cy, g - 1.0);
  else ck_euler1d(a, tc, cx, cy, g - 1.0);
#pragma unroll
  for (int q = 0; q < NC; ++q) tc[q][0] = Ws[q];
  // Lobatto rule in time (nodes 0, l1, l2, 1; weights 1/12, 5/12, 5/12, 1/12)
  using namespace shweno_tables;
  const double taus[4] = {0.0, LOB_L1 * dt, LOB_L2 * dt, dt};
  const double wts[4] = {LOB_W0, LOB_W1, LOB_W1, LOB_W0};
  double Fh[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) Fh[q] = 0.0;
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    double W[NC], F[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double tau = taus[al];
      W[q] = (((tc[q][4] * tau + tc[q][3]) * tau + tc[q][2]) * tau + tc[q][1]) * tau + tc[q][0];
    }
    phys_flux<NC>(W, g, 0, F);
#pragma unroll
    for (int q = 0; q < NC; ++q) Fh[q] += wts[al] * F[q];
    if (al == 3) {
#pragma unroll
      for (int q = 0; q < NC; ++q) WE[(size_t)q * (P.nx + 1) + f] = W[q];
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) FH[(size_t)q * (P.nx + 1) + f] = Fh[q];
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
      out[(size_t)(nc + q) * N + j] = (WE[fo + 1] - WE[fo]) / P.dx;
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
  if (P.ncomp == 1)
    face1d_kernel<1><<<(nf + b - 1) / b, b, 0, st>>>(P, ctl, s0, s1, flag, FH, WE);
  else
    face1d_kernel<3><<<(nf + b - 1) / b, b, 0, st>>>(P, ctl, s0, s1, flag, FH, WE);
  if (ev) cudaEventRecord(ev[1], st);
  update1d_kernel<<<(P.nx + 255) / 256, 256, 0, st>>>(P, ctl, s0, s1, o0, o1, FH, WE);
  if (ev) cudaEventRecord(ev[2], st);
}

}  // namespace shweno
