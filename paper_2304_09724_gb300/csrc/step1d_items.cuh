// Per-item device functions of the 1D step, shared by the one-mesh kernels (step1d.cu) and the
// batched persistent kernel (batch.cu).
#pragma once
#include "ck_generated.cuh"
#include "shweno_device.cuh"

namespace shweno {

// One interface x_{f-1/2} (between cells f-1 and f) of state st: SHWENO reconstruction of both
// neighbours, leading term, linearised derivative problems, CK, Lobatto flux; returns the
// time-averaged flux Fh and the state We at t + dt.  Q: reading R1' (quintic p1).
template <int NC, bool Q = false>
__device__ __forceinline__ void face1d_point(const Params& P, const double* st,
                                             const uint8_t* __restrict__ flag, int f, double t,
                                             double dt, double Fh[NC], double We[NC]) {
  const double g = P.gamma;
  double a[NC][25], dR[NC][25];
  double WL0[NC], WR0[NC];
  bool done = false;
  if constexpr (NC > 1) if (P.charwise) {
    // characteristic fields of F'(W_ref), W_ref = mean of the two cells next to the face
    double Wref[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) Wref[q] = 0.5 * (fetch(P, st, 0, q, f - 1, 0, t) + fetch(P, st, 0, q, f, 0, t));
    CharBasis<NC> B;
    B.setup(Wref, g, 0);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int cell = f - 1 + side;
      const int nonlinear = cell_flag(P, flag, cell, 0);
      const double xi0 = side == 0 ? 0.5 : -0.5;
      constexpr int ND = Q ? 6 : 5;
      double d[ND][NC], x[ND][NC];  // W-, W0, W+, h V-, h V+ (, h V0): physical, then fields
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        d[0][q] = fetch(P, st, 0, q, cell - 1, 0, t);
        d[1][q] = fetch(P, st, 0, q, cell, 0, t);
        d[2][q] = fetch(P, st, 0, q, cell + 1, 0, t);
        d[3][q] = P.dx * fetch(P, st, 1, q, cell - 1, 0, t);
        d[4][q] = P.dx * fetch(P, st, 1, q, cell + 1, 0, t);
        if constexpr (Q) d[5][q] = P.dx * fetch(P, st, 1, q, cell, 0, t);
      }
#pragma unroll
      for (int r = 0; r < ND; ++r) B.to_fields(d[r], x[r]);
      double e[NC][6];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        double c[6];
        p1_coeffs_t<Q>(x[0][k], x[1][k], x[2][k], x[3][k], Q ? x[ND - 1][k] : 0.0, x[4][k], c);
        const Mix mx = shweno_mix_t<Q>(P, x[0][k], x[1][k], x[2][k], c, nonlinear);
        mix_coeffs_t<Q>(mx, x[0][k], x[1][k], x[2][k], c, e[k]);
        taylor_shift_d<Q ? 5 : 4>(e[k], xi0);
      }
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        double xm[NC], ym[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) xm[k] = e[k][m];
        B.to_physical(xm, ym);
#pragma unroll
        for (int q = 0; q < NC; ++q) (side == 0 ? a : dR)[q][m * 5] = ym[q];
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) (side == 0 ? WL0 : WR0)[q] = (side == 0 ? a : dR)[q][0];
    }
    done = true;
  }
  if (!done) {
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
        const double v0 = Q ? P.dx * fetch(P, st, 1, q, cell, 0, t) : 0.0;
        double c[6], e[6];
        p1_coeffs_t<Q>(Wm, W0, Wp, vm, v0, vp, c);
        const Mix mx = shweno_mix_t<Q>(P, Wm, W0, Wp, c, nonlinear);
        mix_coeffs_t<Q>(mx, Wm, W0, Wp, c, e);
        taylor_shift_d<Q ? 5 : 4>(e, xi0);
#pragma unroll
        for (int m = 0; m < 5; ++m) (side == 0 ? a : dR)[q][m * 5] = e[m];
        (side == 0 ? WL0 : WR0)[q] = e[0];
      }
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
      for (int q = 0; q < NC; ++q) We[q] = W[q];
    }
  }
}

}  // namespace shweno
