// Per-item device functions of the 2D step, shared by the one-mesh kernels (step2d.cu) and the
// batched persistent kernel (batch.cu).  See step2d.cu for the structure of the step.
#pragma once
#include "ck_generated.cuh"
#include "shweno_device.cuh"

namespace shweno {

constexpr int SEG = 128;          // threads of a face CTA
constexpr int NFACE = SEG - 1;    // faces of a face CTA: its threads own the SEG cells next to them
constexpr int SPAN = NFACE + 3;   // first-pass evaluations a CTA needs
constexpr int TX = 32;            // first-pass tile width

// ------------------------------------------------------------------ second pass, cell by cell
// Second pass across the face.  ev[set*NC+q][k][col] holds the first-pass Taylor coefficients
// (order k along the face) of a row of stencil columns; column c holds the cell whose stencil is
// columns c-1..c+1.  Each cell's weights come from its order-0 data and serve every order
// (remark ending Section 2.1.2) and both of the cell's ends, so one thread per cell forms its
// weights once and then, order by order, the Taylor coefficients across the face at both ends
// (EndTable); one thread per face then reads the left cell's right end and the right cell's left
// end.  The two ends of a cell share their arithmetic: with s = W- + W+, a = W+ - W-,
// dv = v+ - v-, sv = v- + v+, p1's coefficient p at xi = +-1/2 is U_p + V_p and (-1)^p (U_p - V_p)
// (U_p from the even monomials, V_p from the odd ones; end_u / end_v of recon_tables.cuh).
struct EndTable {
  // left ends (xi = -1/2) of the cells, two buffers (orders of even / odd K) so that one barrier
  // per order suffices: [buffer][comp][p][slot], the cell in column c at slot c - 1
  double L[2][4][5][SEG];
};
// Flags of the cells next to the faces, for the characteristic-wise path (whose weights belong to
// each face point): lin[c] = 1 when the cell in column c uses the linear weights.
struct FlagTable {
  int lin[SPAN];
};

constexpr size_t kEvBytes = sizeof(double) * 8 * 5 * SPAN;
constexpr size_t kFaceSmem = kEvBytes + (sizeof(EndTable) > sizeof(FlagTable) ? sizeof(EndTable) : sizeof(FlagTable));

// Weights of one cell's reconstruction across the face: p = A p1 + B p2 + C p3 per component.
template <int NC>
struct CellMix {
  double A[NC], B[NC], C[NC];
  bool lin;  // linear weights: p = p1 (A = 1, B = C = 0)
};

template <int NC, bool Q>
__device__ __forceinline__ void cell_mix(const Params& P, const double (*ev)[5][SPAN], int c, bool lin,
                                         CellMix<NC>& m) {
  m.lin = lin;
  if (lin) {  // one branch for the whole cell: a warp of linear cells skips the weights
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      m.A[q] = 1.0;
      m.B[q] = m.C[q] = 0.0;
    }
    return;
  }
  if constexpr (NC == 4 && !Q) {
    // the four components' weights normalised in pairs: 1/S0 = S1 / (S0 S1), 1/S1 = S0 / (S0 S1)
    // (two divisions instead of four; the sums are products of smoothness indicators, far from
    // the range where their product could overflow)
    RawWeights rw[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double Wm = ev[q][0][c - 1], W0 = ev[q][0][c], Wp = ev[q][0][c + 1];
      double cf[6];
      p1_coeffs_t<Q>(Wm, W0, Wp, ev[NC + q][0][c - 1], ev[NC + q][0][c], ev[NC + q][0][c + 1], cf);
      rw[q] = shweno_raw_weights(P, Wm, W0, Wp, cf);
    }
#pragma unroll
    for (int h = 0; h < NC; h += 2) {
      const double r = 1.0 / (rw[h].sum * rw[h + 1].sum);
      const Mix m0 = mix_from_raw(P, rw[h], r * rw[h + 1].sum), m1 = mix_from_raw(P, rw[h + 1], r * rw[h].sum);
      m.A[h] = m0.A; m.B[h] = m0.B; m.C[h] = m0.C;
      m.A[h + 1] = m1.A; m.B[h + 1] = m1.B; m.C[h + 1] = m1.C;
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double Wm = ev[q][0][c - 1], W0 = ev[q][0][c], Wp = ev[q][0][c + 1];
      double cf[6];
      p1_coeffs_t<Q>(Wm, W0, Wp, ev[NC + q][0][c - 1], ev[NC + q][0][c], ev[NC + q][0][c + 1], cf);
      const Mix mm = shweno_mix_t<Q>(P, Wm, W0, Wp, cf, 1);
      m.A[q] = mm.A;
      m.B[q] = mm.B;
      m.C[q] = mm.C;
    }
  }
}

// Taylor coefficients p = 0..4-K across the face of tangential order K at both ends of the cell in
// column c, into slot c - 1 of the EndTable.  The small stencils p2 = W0 + (W0 - W-) xi and
// p3 = W0 + (W+ - W0) xi add h +- g/2 to the value and g to the slope at the ends, with
// h = (B + C) W0 and g = B (W0 - W-) + C (W+ - W0).  LIN: a cell with the linear weights (p = p1,
// A = 1, B = C = 0; the general form gives the same values bit for bit with more operations).
template <int NC, bool LIN, bool Q, int K>
__device__ __forceinline__ void cell_ends_t(const double (*ev)[5][SPAN], int c, const CellMix<NC>& m,
                                            EndTable& et, double eRo[NC][5]) {
  using namespace shweno_tables;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const double Wm = ev[q][K][c - 1], W0 = ev[q][K][c], Wp = ev[q][K][c + 1];
    const double vm = ev[NC + q][K][c - 1], vp = ev[NC + q][K][c + 1];
    const double v0 = Q ? ev[NC + q][K][c] : 0.0;
    const double s = Wm + Wp, a = Wp - Wm, dv = vp - vm, sv = vm + vp;
    const double A = m.A[q];
    double g = 0.0, hR = 0.0, hL = 0.0;
    if (!LIN) {
      g = m.B[q] * (W0 - Wm) + m.C[q] * (Wp - W0);
      const double h = (m.B[q] + m.C[q]) * W0;
      hR = fma(0.5, g, h);
      hL = fma(-0.5, g, h);
    }
#pragma unroll
    for (int p = 0; p + K <= 4; ++p) {
      const double U = end_u(p, W0, s, dv);
      double eR, eL;
      if (!Q && p == 4) {  // V_4 = 0 for the quartic: both ends are U_4
        eR = eL = LIN ? U : A * U;
      } else {
        const double V = Q ? qend_v(p, a, sv, v0) : end_v(p, a, sv);
        if (LIN) {
          eR = U + V;
          eL = (p & 1) ? V - U : U - V;
        } else if (p == 0) {
          eR = fma(A, V, fma(A, U, hR));
          eL = fma(-A, V, fma(A, U, hL));
        } else if (p == 1) {
          eR = fma(A, V, fma(A, U, g));
          eL = fma(A, V, fma(-A, U, g));
        } else {
          const double AU = A * U;
          eR = fma(A, V, AU);
          eL = (p & 1) ? fma(A, V, -AU) : fma(-A, V, AU);
        }
      }
      eRo[q][p] = eR;
      et.L[K & 1][q][p][c - 1] = eL;
    }
  }
}
// FLAGS = false: every cell is nonlinear (no branch on the flag); otherwise one branch per cell.
template <int NC, bool FLAGS, bool Q, int K>
__device__ __forceinline__ void cell_ends(const double (*ev)[5][SPAN], int c, const CellMix<NC>& m,
                                          EndTable& et, double eR[NC][5]) {
  if (FLAGS && m.lin) cell_ends_t<NC, true, Q, K>(ev, c, m, et, eR);
  else cell_ends_t<NC, false, Q, K>(ev, c, m, et, eR);
}

// Order K of the face point between cell columns f + 1 and f + 2: the two sides from the
// EndTable; at K = 0 the leading term (Burgers: exact Godunov state; Euler: HLLC) and the
// eigen-decomposition of the upwinding; every derivative vector upwinded into a[q][m*5+n]
// (m along x, n along y; dir = 0: x-face, p across = m; dir = 1: y-face, p across = n).
template <int NC, int K>
__device__ __forceinline__ void face_order(const Params& P, const EndTable& et, const double eR[NC][5], int f,
                                           int dir, double Ws[NC], Upwinder<NC>& U, double a[NC][25]) {
  double dr[NC][5];
#pragma unroll
  for (int q = 0; q < NC; ++q)
#pragma unroll
    for (int p = 0; p + K <= 4; ++p) dr[q][p] = et.L[K & 1][q][p][f + 1];
  if constexpr (K == 0) {
    double WL[NC], WR[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { WL[q] = eR[q][0]; WR[q] = dr[q][0]; }
    if constexpr (NC == 1) Ws[0] = burgers_godunov(WL[0], WR[0]);  // the same flux u^2/2 along x and y
    else hllc_state<NC>(WL, WR, P.gamma, dir, Ws);
    U.setup(Ws, P.gamma, dir, NC == 1 ? fmax(fabs(WL[0]), fabs(WR[0])) : 0.0);
  }
#pragma unroll
  for (int p = 0; p + K <= 4; ++p) {
    if (p == 0 && K == 0) continue;
    double x[NC], y[NC], o[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { x[q] = eR[q][p]; y[q] = dr[q][p]; }
    U.apply(x, y, o);
    const int idx = dir == 0 ? p * 5 + K : K * 5 + p;
#pragma unroll
    for (int q = 0; q < NC; ++q) a[q][idx] = o[q];
  }
}

// One order of the two-phase second pass: every cell thread keeps its right ends and publishes its
// left ends (buffer K & 1), one barrier, then every face thread upwinds its own cell's right end
// against the next cell's left end.  The next order writes the other buffer, so a thread still
// reading this one cannot be overtaken.  Called by all threads of the CTA (it holds the barrier).
template <int NC, bool FLAGS, bool Q, int K>
__device__ __forceinline__ void pass_order(const Params& P, const double (*ev)[5][SPAN], EndTable& et,
                                           bool has_cell, const CellMix<NC>& m, bool has_face,
                                           int dir, double Ws[NC], Upwinder<NC>& U, double a[NC][25]) {
  double eR[NC][5];
  if (has_cell) cell_ends<NC, FLAGS, Q, K>(ev, threadIdx.x + 1, m, et, eR);
  __syncthreads();
  if (has_face) face_order<NC, K>(P, et, eR, threadIdx.x, dir, Ws, U, a);
}

// Second pass, leading term, upwinding and CK of the nf faces of a CTA (nf <= NFACE): thread t
// owns the cell in column t + 1 (t <= nf) and the face between columns t + 1 and t + 2 (t < nf).
// Returns true for a face thread, whose tc[q][0..4] are then the time-Taylor coefficients of its
// face point.  nl(c): whether the cell in column c uses the nonlinear weights.
template <int NC, bool FLAGS, bool Q, typename FlagOf>
__device__ __forceinline__ bool second_pass_cells(const Params& P, const double (*ev)[5][SPAN],
                                                  unsigned char* tbl, int nf, int dir, FlagOf nl,
                                                  double tc[NC][5]) {
  EndTable& et = *reinterpret_cast<EndTable*>(tbl);
  const bool has_cell = (int)threadIdx.x <= nf, has_face = (int)threadIdx.x < nf;
  CellMix<NC> m;
  if (has_cell) cell_mix<NC, Q>(P, ev, threadIdx.x + 1, FLAGS && !nl(threadIdx.x + 1), m);
  double a[NC][25], Ws[NC];
  Upwinder<NC> U;
  pass_order<NC, FLAGS, Q, 0>(P, ev, et, has_cell, m, has_face, dir, Ws, U, a);
  pass_order<NC, FLAGS, Q, 1>(P, ev, et, has_cell, m, has_face, dir, Ws, U, a);
  pass_order<NC, FLAGS, Q, 2>(P, ev, et, has_cell, m, has_face, dir, Ws, U, a);
  pass_order<NC, FLAGS, Q, 3>(P, ev, et, has_cell, m, has_face, dir, Ws, U, a);
  pass_order<NC, FLAGS, Q, 4>(P, ev, et, has_cell, m, has_face, dir, Ws, U, a);
  if (!has_face) return false;
#pragma unroll
  for (int q = 0; q < NC; ++q) a[q][0] = Ws[q];
  double t4[NC][5];
  if constexpr (NC == 1) ck_burgers2d(a, t4, P.ckx, P.cky, P.gamma - 1.0);
  else ck_euler2d(a, t4, P.ckx, P.cky, P.gamma - 1.0);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    tc[q][0] = Ws[q];
#pragma unroll
    for (int k = 1; k < 5; ++k) tc[q][k] = t4[q][k];
  }
  return true;
}

// ------------------------------------------------------------------ characteristic-wise face point
// Cross-face Taylor coefficients e[p] (p <= 4 - k) of tangential order k at the right end
// (PLUS, xi = +1/2) or left end of a cell, from its field data d = (W-, W0, W+, v-, v+) of that
// order ((W-, W0, W+, v-, v0, v+) for reading R1', Q): e[p] = A * END[p] . d + (small-stencil
// terms for p <= 1).
template <bool PLUS, bool Q = false>
__device__ __forceinline__ void side_out_d(const double* d, int k, double A, double B, double C,
                                           bool lin, double e[5]) {
  using namespace shweno_tables;
  if (lin) {  // linear weights: p = p1
#pragma unroll
    for (int p = 0; p + k <= 4; ++p) e[p] = Q ? qend_dot<PLUS>(p, d) : end_dot<PLUS>(p, d);
    return;
  }
#pragma unroll
  for (int p = 0; p + k <= 4; ++p) e[p] = A * (Q ? qend_dot<PLUS>(p, d) : end_dot<PLUS>(p, d));
  // p2 = W0 + (W0 - W-) xi and p3 = W0 + (W+ - W0) xi: value and slope at the end
  if (PLUS) e[0] += (1.5 * B + 0.5 * C) * d[1] - 0.5 * B * d[0] + 0.5 * C * d[2];
  else e[0] += (0.5 * B + 1.5 * C) * d[1] + 0.5 * B * d[0] - 0.5 * C * d[2];
  if (k <= 3) e[1] += (B - C) * d[1] - B * d[0] + C * d[2];
}

// Characteristic-wise counterpart for one face point (Euler, NC = 4): the first-pass data of
// tangential order k of the four stencil columns c0..c0+3, projected onto the fields of basis
// Bs; xw[c][f] from {W, Y} (x-face) or {W, V} (y-face), xv[c][f] from the derivative set.
template <int NC>
__device__ __forceinline__ void fields_at(const double (*ev)[5][SPAN], const CharBasis<NC>& Bs, int c0,
                                          int k, double xw[4][NC], double xv[4][NC]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double w[NC], v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { w[q] = ev[q][k][c0 + c]; v[q] = ev[NC + q][k][c0 + c]; }
    Bs.to_fields(w, xw[c]);
    Bs.to_fields(v, xv[c]);
  }
}
// Cross-face Taylor coefficients of both sides in physical variables, tangential order k, from
// the field data: left cell = column 1 (stencil 0..2), right cell = column 2 (stencil 1..3).
template <int NC, bool Q>
__device__ __forceinline__ void char_sides(const CharBasis<NC>& Bs, const double xw[4][NC],
                                           const double xv[4][NC], int k, const double* AL,
                                           const double* BL, const double* CL, bool linL,
                                           const double* AR, const double* BR, const double* CR,
                                           bool linR, double dl[NC][5], double dr[NC][5]) {
  double el[NC][5], er[NC][5];
#pragma unroll
  for (int f = 0; f < NC; ++f) {
    if constexpr (Q) {
      const double dL[6] = {xw[0][f], xw[1][f], xw[2][f], xv[0][f], xv[1][f], xv[2][f]};
      const double dR[6] = {xw[1][f], xw[2][f], xw[3][f], xv[1][f], xv[2][f], xv[3][f]};
      side_out_d<true, true>(dL, k, AL[f], BL[f], CL[f], linL, el[f]);
      side_out_d<false, true>(dR, k, AR[f], BR[f], CR[f], linR, er[f]);
    } else {
      const double dL5[5] = {xw[0][f], xw[1][f], xw[2][f], xv[0][f], xv[2][f]};
      const double dR5[5] = {xw[1][f], xw[2][f], xw[3][f], xv[1][f], xv[3][f]};
      side_out_d<true>(dL5, k, AL[f], BL[f], CL[f], linL, el[f]);
      side_out_d<false>(dR5, k, AR[f], BR[f], CR[f], linR, er[f]);
    }
  }
#pragma unroll
  for (int p = 0; p + k <= 4; ++p) {
    double x[NC], y[NC];
#pragma unroll
    for (int f = 0; f < NC; ++f) x[f] = el[f][p];
    Bs.to_physical(x, y);
#pragma unroll
    for (int q = 0; q < NC; ++q) dl[q][p] = y[q];
#pragma unroll
    for (int f = 0; f < NC; ++f) x[f] = er[f][p];
    Bs.to_physical(x, y);
#pragma unroll
    for (int q = 0; q < NC; ++q) dr[q][p] = y[q];
  }
}

// Face point of the characteristic-wise option (Euler): the second pass across the face runs in
// the characteristic fields of the Jacobian along the face normal at Wref (the mean of the cell
// averages next to the point), with its own weights per field and side; then the leading term
// (HLLC), the upwinding and CK.  Left cell in column c0 + 1, right cell in c0 + 2; dir = 0:
// x-face (first pass along y), 1: y-face.  Returns the time-Taylor coefficients tc[q][0..4].
template <int NC, bool FLAGS, bool Q>
__device__ __forceinline__ void char_face_point(const Params& P, const double (*ev)[5][SPAN],
                                                const FlagTable& ft, int c0, int dir, double tc[NC][5],
                                                const double* Wref) {
  static_assert(NC == 4, "characteristic fields are for the Euler system");
  const double g = P.gamma;
  double a[NC][25];
  double dl[NC][5], dr[NC][5];
  double AL[NC], BL[NC], CL[NC], AR[NC], BR[NC], CR[NC];
  // FLAGS = false: every cell uses the nonlinear weights (compile-time, no branch)
  const bool linL = FLAGS && ft.lin[c0 + 1], linR = FLAGS && ft.lin[c0 + 2];
  CharBasis<NC> Bs;
  Bs.setup(Wref, g, dir);
  {
    double xw[4][NC], xv[4][NC];
    fields_at<NC>(ev, Bs, c0, 0, xw, xv);
#pragma unroll
    for (int f = 0; f < NC; ++f) {
      AL[f] = AR[f] = 1.0;
      BL[f] = CL[f] = BR[f] = CR[f] = 0.0;
      if (!linL) {
        double cf[6];
        p1_coeffs_t<Q>(xw[0][f], xw[1][f], xw[2][f], xv[0][f], xv[1][f], xv[2][f], cf);
        const Mix m = shweno_mix_t<Q>(P, xw[0][f], xw[1][f], xw[2][f], cf, 1);
        AL[f] = m.A; BL[f] = m.B; CL[f] = m.C;
      }
      if (!linR) {
        double cf[6];
        p1_coeffs_t<Q>(xw[1][f], xw[2][f], xw[3][f], xv[1][f], xv[2][f], xv[3][f], cf);
        const Mix m = shweno_mix_t<Q>(P, xw[1][f], xw[2][f], xw[3][f], cf, 1);
        AR[f] = m.A; BR[f] = m.B; CR[f] = m.C;
      }
    }
    char_sides<NC, Q>(Bs, xw, xv, 0, AL, BL, CL, linL, AR, BR, CR, linR, dl, dr);
  }
  double WL[NC], WR[NC], Ws[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) { WL[q] = dl[q][0]; WR[q] = dr[q][0]; }
  hllc_state<NC>(WL, WR, g, dir, Ws);
  Upwinder<NC> U;
  U.setup(Ws, g, dir);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (k > 0) {
      double xw[4][NC], xv[4][NC];
      fields_at<NC>(ev, Bs, c0, k, xw, xv);
      char_sides<NC, Q>(Bs, xw, xv, k, AL, BL, CL, linL, AR, BR, CR, linR, dl, dr);
    }
#pragma unroll
    for (int p = 0; p + k <= 4; ++p) {
      if (p == 0 && k == 0) continue;
      double x[NC], y[NC], o[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) { x[q] = dl[q][p]; y[q] = dr[q][p]; }
      U.apply(x, y, o);
      // p is the order across the face, k the order along it
      const int idx = dir == 0 ? p * 5 + k : k * 5 + p;
#pragma unroll
      for (int q = 0; q < NC; ++q) a[q][idx] = o[q];
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) a[q][0] = Ws[q];
  double t4[NC][5];
  ck_euler2d(a, t4, P.ckx, P.cky, g - 1.0);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    tc[q][0] = Ws[q];
#pragma unroll
    for (int k = 1; k < 5; ++k) tc[q][k] = t4[q][k];
  }
}

// Lobatto time average of the flux along dir and the state at tau = dt.  Euler: the nodes tau > 0
// share one division (1/rho1 = rho2 rho3 / (rho1 rho2 rho3) and so on).
template <int NC>
__device__ __forceinline__ void lobatto(const double tc[NC][5], double dt, double g, int dir,
                                        double Fh[NC], double We[NC]) {
  using namespace shweno_tables;
  const double taus[4] = {0.0, LOB_L1 * dt, LOB_L2 * dt, dt};
  const double wts[4] = {LOB_W0, LOB_W1, LOB_W1, LOB_W0};
  double W[4][NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) W[0][q] = tc[q][0];  // tau = 0: the leading term itself
#pragma unroll
  for (int al = 1; al < 4; ++al)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double tau = taus[al];
      W[al][q] = (((tc[q][4] * tau + tc[q][3]) * tau + tc[q][2]) * tau + tc[q][1]) * tau + tc[q][0];
    }
  double ir[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (NC > 1) {
    ir[0] = 1.0 / W[0][0];
    const double r23 = W[2][0] * W[3][0];
    const double inv = 1.0 / (W[1][0] * r23);
    ir[1] = inv * r23;
    const double i23 = inv * W[1][0];  // 1 / (rho2 rho3)
    ir[2] = i23 * W[3][0];
    ir[3] = i23 * W[2][0];
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) Fh[q] = 0.0;
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    double F[NC];
    phys_flux_ir<NC>(W[al], ir[al], g, dir, F);
#pragma unroll
    for (int q = 0; q < NC; ++q) Fh[q] += wts[al] * F[q];
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) We[q] = W[3][q];
}

__device__ __forceinline__ double state_at(const double tc[5], double tau) {
  return (((tc[4] * tau + tc[3]) * tau + tc[2]) * tau + tc[1]) * tau + tc[0];
}

// Combined coefficients C[u] of NU = 1 or 2 components of one cell from their stencil averages
// w[u] = (W-, W0, W+) and p1 coefficients c[u] (C = c for a cell with the linear weights).  PAIR
// (Euler, reading R1): the two components' weights share one division, 1/S0 = S1 / (S0 S1) and
// 1/S1 = S0 / (S0 S1), as in the second pass.
template <bool Q, bool PAIR>
__device__ __forceinline__ void first_pass_mix(const Params& P, int nl, const double (*w)[3], const double (*c)[6],
                                               double (*C)[6]) {
  constexpr int NU = PAIR ? 2 : 1;
  if (!nl) {
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int k = 0; k < 6; ++k) C[u][k] = c[u][k];
    return;
  }
  if constexpr (PAIR) {
    const RawWeights r0 = shweno_raw_weights(P, w[0][0], w[0][1], w[0][2], c[0]);
    const RawWeights r1 = shweno_raw_weights(P, w[1][0], w[1][1], w[1][2], c[1]);
    const double inv = 1.0 / (r0.sum * r1.sum);
    mix_coeffs_t<Q>(mix_from_raw(P, r0, inv * r1.sum), w[0][0], w[0][1], w[0][2], c[0], C[0]);
    mix_coeffs_t<Q>(mix_from_raw(P, r1, inv * r0.sum), w[1][0], w[1][1], w[1][2], c[1], C[1]);
  } else {
    mix_coeffs_t<Q>(shweno_mix_t<Q>(P, w[0][0], w[0][1], w[0][2], c[0], 1), w[0][0], w[0][1], w[0][2], c[0], C[0]);
  }
}

// First-pass polynomials of the cells of one tile: thread (tx, ty) of a TX x TYB block owns the
// extended cell (bx + tx, by + ty); the 4 * NC fields of the tile plus a one-cell halo are staged
// in shared memory `tile` (room for 16) by all nthreads threads first.  Q: reading R1', whose
// quintic p1 also uses the cell's own derivative average; it stores six coefficients per
// polynomial instead of five (the scratch layout's KC).
template <int NC, int TYB, bool Q = false>
__device__ __forceinline__ void coef2d_item(const Params& P, const StepView& sv, const double* s0,
                                            const double* s1, const uint8_t* __restrict__ flag,
                                            double* __restrict__ ycoef, double* __restrict__ xcoef,
                                            int bx, int by, double (*tile)[TYB + 2][TX + 2], int tx,
                                            int ty) {
  const double* st = sv.odd ? s1 : s0;
  const double t = sv.t;
  const int tid = ty * TX + tx;
  for (int idx = tid; idx < 4 * NC * (TYB + 2) * (TX + 2); idx += TX * TYB) {
    const int xx = idx % (TX + 2), rest = idx / (TX + 2);
    const int yy = rest % (TYB + 2), fq = rest / (TYB + 2);
    const int i = bx - 1 + xx, j = by - 1 + yy;
    double v = 0.0;
    if (i >= -3 && i <= P.nx + 2 && j >= -3 && j <= P.ny + 2) v = fetch(P, st, fq / NC, fq % NC, i, j, t);
    tile[fq][yy][xx] = v;
  }
  __syncthreads();
  const int ic = bx + tx, jr = by + ty;
  const int lx = tx + 1, ly = ty + 1;
  const int NX4 = P.nx + 4, NY2 = P.ny + 2, NY4 = P.ny + 4;
  constexpr int KC = Q ? 6 : 5;
  constexpr bool PAIR = NC == 4 && !Q;
  constexpr int NU = PAIR ? 2 : 1;
  if (ic <= P.nx + 1 && jr >= -1 && jr <= P.ny) {  // y-pass: {W,Y} and {V,Z} along a column
    const int nl = cell_flag(P, flag, ic, jr);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int q0 = 0; q0 < NC; q0 += NU) {
        double w[NU][3], c[NU][6], C[NU][6];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int fa = (s == 0 ? 0 : 1) * NC + q0 + u, fd = (s == 0 ? 2 : 3) * NC + q0 + u;
          w[u][0] = tile[fa][ly - 1][lx]; w[u][1] = tile[fa][ly][lx]; w[u][2] = tile[fa][ly + 1][lx];
          const double vm = P.dy * tile[fd][ly - 1][lx], vp = P.dy * tile[fd][ly + 1][lx];
          const double v0 = Q ? P.dy * tile[fd][ly][lx] : 0.0;
          p1_coeffs_t<Q>(w[u][0], w[u][1], w[u][2], vm, v0, vp, c[u]);
        }
        first_pass_mix<Q, PAIR>(P, nl, w, c, C);
        const double sc = s == 0 ? 1.0 : P.dx;  // x-pass derivative data: dx * avg(W_x)
#pragma unroll
        for (int u = 0; u < NU; ++u)
#pragma unroll
          for (int k = 0; k < KC; ++k)
            ycoef[((size_t)((s * NC + q0 + u) * KC + k) * NY2 + (jr + 1)) * NX4 + (ic + 2)] = sc * C[u][k];
      }
  }
  if (ic >= 0 && ic < P.nx && jr <= P.ny + 1) {  // x-pass: {W,V} and {Y,Z} along a row
    const int nl = cell_flag(P, flag, ic, jr);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int q0 = 0; q0 < NC; q0 += NU) {
        double w[NU][3], c[NU][6], C[NU][6];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int fa = (s == 0 ? 0 : 2) * NC + q0 + u, fd = (s == 0 ? 1 : 3) * NC + q0 + u;
          w[u][0] = tile[fa][ly][lx - 1]; w[u][1] = tile[fa][ly][lx]; w[u][2] = tile[fa][ly][lx + 1];
          const double vm = P.dx * tile[fd][ly][lx - 1], vp = P.dx * tile[fd][ly][lx + 1];
          const double v0 = Q ? P.dx * tile[fd][ly][lx] : 0.0;
          p1_coeffs_t<Q>(w[u][0], w[u][1], w[u][2], vm, v0, vp, c[u]);
        }
        first_pass_mix<Q, PAIR>(P, nl, w, c, C);
        const double sc = s == 0 ? 1.0 : P.dy;  // y-pass derivative data: dy * avg(W_y)
#pragma unroll
        for (int u = 0; u < NU; ++u)
#pragma unroll
          for (int k = 0; k < KC; ++k)
            xcoef[((size_t)((s * NC + q0 + u) * KC + k) * P.nx + ic) * NY4 + (jr + 2)] = sc * C[u][k];
      }
  }
}

// x-face Gauss points (slice 0..2, cell row `row`) or corner points (slice 3, corner row `row`
// at y_{row-1/2}) of faces x_{f0-1/2} .. x_{f0+NFACE-3/2}; SEG threads, smem_raw of kFaceSmem
// bytes.
template <int NC, bool FLAGS, bool CHAR = false, bool Q = false>
__device__ __forceinline__ void xface_item(const Params& P, const StepView& sv, const double* st,
                                           const double* __restrict__ ycoef,
                                           const uint8_t* __restrict__ flag, double* __restrict__ FX,
                                           double* __restrict__ WX, double* __restrict__ WC, int f0,
                                           int row, int slice, unsigned char* smem_raw) {
  double(*ev)[5][SPAN] = reinterpret_cast<double(*)[5][SPAN]>(smem_raw);
  const int NX4 = P.nx + 4, NY2 = P.ny + 2;
  using namespace shweno_tables;
  // faces x_{f0-1/2} .. x_{f0+nf-3/2} exist; their stencils span columns 0 .. nf + 2
  const int nf = min(NFACE, P.nx + 1 - f0), ncol = nf + 3;
  for (int it = threadIdx.x; it < 2 * NC * ncol; it += SEG) {
    const int col = it % ncol, rq = it / ncol;
    const int tcol = f0 + col;
    double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (tcol >= NX4) {
    } else if constexpr (Q) {  // six coefficients per polynomial (reading R1')
      if (slice < 3) {
        const double* src = ycoef + ((size_t)(rq * 6) * NY2 + (row + 1)) * NX4 + tcol;
#pragma unroll
        for (int k = 0; k < 6; ++k) e[k] = __ldcg(src + (size_t)k * NY2 * NX4);
        if (slice != 1) taylor_shift_d<5>(e, slice == 0 ? -GAUSS_G : GAUSS_G);
      } else {
        double lo[6], hi[6];
        const double* slo = ycoef + ((size_t)(rq * 6) * NY2 + row) * NX4 + tcol;
        const double* shi = slo + NX4;
#pragma unroll
        for (int k = 0; k < 6; ++k) { lo[k] = __ldcg(slo + (size_t)k * NY2 * NX4); hi[k] = __ldcg(shi + (size_t)k * NY2 * NX4); }
        taylor_shift_d<5>(lo, 0.5);
        taylor_shift_d<5>(hi, -0.5);
#pragma unroll
        for (int k = 0; k < 5; ++k) e[k] = 0.5 * (lo[k] + hi[k]);
      }
    } else if (slice < 3) {
      const double* src = ycoef + ((size_t)(rq * 5) * NY2 + (row + 1)) * NX4 + tcol;
#pragma unroll
      for (int k = 0; k < 5; ++k) e[k] = __ldcg(src + (size_t)k * NY2 * NX4);
      if (slice != 1) taylor_shift(e, slice == 0 ? -GAUSS_G : GAUSS_G, 4);
    } else {
      double lo[5], hi[5];
      const double* slo = ycoef + ((size_t)(rq * 5) * NY2 + row) * NX4 + tcol;
      const double* shi = slo + NX4;
#pragma unroll
      for (int k = 0; k < 5; ++k) { lo[k] = __ldcg(slo + (size_t)k * NY2 * NX4); hi[k] = __ldcg(shi + (size_t)k * NY2 * NX4); }
      taylor_shift(lo, 0.5, 4);
      taylor_shift(hi, -0.5, 4);
#pragma unroll
      for (int k = 0; k < 5; ++k) e[k] = 0.5 * (lo[k] + hi[k]);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) ev[rq][k][col] = e[k];
  }
  __syncthreads();
  // cell column c holds cell i = f0 + c - 2; a corner row uses the rows below and above
  auto nl = [&](int c) {
    const int i = f0 + c - 2;
    return slice < 3 ? cell_flag(P, flag, i, row)
                     : (cell_flag(P, flag, i, row - 1) | cell_flag(P, flag, i, row));
  };
  const int fi = f0 + threadIdx.x;  // face x_{fi-1/2}
  double tc[NC][5];
  if constexpr (CHAR) {
    FlagTable& ft = *reinterpret_cast<FlagTable*>(smem_raw + kEvBytes);
    for (int c = 1 + threadIdx.x; c <= nf + 1; c += SEG) ft.lin[c] = !nl(c);
    __syncthreads();
    if ((int)threadIdx.x >= nf) return;  // no barrier follows
    double Wref[NC];  // cells next to the face point (the four around a corner)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      if (slice < 3)
        Wref[q] = 0.5 * (fetch(P, st, 0, q, fi - 1, row, sv.t) + fetch(P, st, 0, q, fi, row, sv.t));
      else
        Wref[q] = 0.25 * (fetch(P, st, 0, q, fi - 1, row - 1, sv.t) + fetch(P, st, 0, q, fi, row - 1, sv.t) +
                          fetch(P, st, 0, q, fi - 1, row, sv.t) + fetch(P, st, 0, q, fi, row, sv.t));
    }
    char_face_point<NC, FLAGS, Q>(P, ev, ft, threadIdx.x, 0, tc, Wref);
  } else {
    if (!second_pass_cells<NC, FLAGS, Q>(P, ev, smem_raw + kEvBytes, nf, 0, nl, tc)) return;
  }
  const double dt = sv.dt;
  if (slice < 3) {
    double Fh[NC], We[NC];
    lobatto<NC>(tc, dt, P.gamma, 0, Fh, We);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const size_t o = ((size_t)(slice * NC + q) * P.ny + row) * (P.nx + 1) + fi;
      FX[o] = Fh[q];
      WX[o] = We[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < NC; ++q) WC[((size_t)q * (P.ny + 1) + row) * (P.nx + 1) + fi] = state_at(tc[q], dt);
  }
}

// y-face Gauss points (slice 0..2) of column `col`, faces y_{f0-1/2} .. y_{f0+NFACE-3/2}.
template <int NC, bool FLAGS, bool CHAR = false, bool Q = false>
__device__ __forceinline__ void yface_item(const Params& P, const StepView& sv, const double* st,
                                           const double* __restrict__ xcoef,
                                           const uint8_t* __restrict__ flag, double* __restrict__ FY,
                                           double* __restrict__ WY, int f0, int col, int slice,
                                           unsigned char* smem_raw) {
  double(*ev)[5][SPAN] = reinterpret_cast<double(*)[5][SPAN]>(smem_raw);
  const int NY4 = P.ny + 4;
  using namespace shweno_tables;
  // faces y_{f0-1/2} .. y_{f0+nf-3/2} exist; their stencils span rows 0 .. nf + 2
  const int nf = min(NFACE, P.ny + 1 - f0), nrow = nf + 3;
  for (int it = threadIdx.x; it < 2 * NC * nrow; it += SEG) {
    const int r = it % nrow, rq = it / nrow;
    const int trow = f0 + r;
    double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (trow < NY4) {
      constexpr int KC = Q ? 6 : 5;
      const double* src = xcoef + ((size_t)(rq * KC) * P.nx + col) * NY4 + trow;
#pragma unroll
      for (int k = 0; k < KC; ++k) e[k] = __ldcg(src + (size_t)k * P.nx * NY4);
      if constexpr (Q) {
        if (slice != 1) taylor_shift_d<5>(e, slice == 0 ? -GAUSS_G : GAUSS_G);
      } else {
        if (slice != 1) taylor_shift(e, slice == 0 ? -GAUSS_G : GAUSS_G, 4);
      }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) ev[rq][k][r] = e[k];
  }
  __syncthreads();
  auto nl = [&](int c) { return cell_flag(P, flag, col, f0 + c - 2); };
  const int fj = f0 + threadIdx.x;  // face y_{fj-1/2}
  double tc[NC][5];
  if constexpr (CHAR) {
    FlagTable& ft = *reinterpret_cast<FlagTable*>(smem_raw + kEvBytes);
    for (int c = 1 + threadIdx.x; c <= nf + 1; c += SEG) ft.lin[c] = !nl(c);
    __syncthreads();
    if ((int)threadIdx.x >= nf) return;
    double Wref[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q)
      Wref[q] = 0.5 * (fetch(P, st, 0, q, col, fj - 1, sv.t) + fetch(P, st, 0, q, col, fj, sv.t));
    char_face_point<NC, FLAGS, Q>(P, ev, ft, threadIdx.x, 1, tc, Wref);
  } else {
    if (!second_pass_cells<NC, FLAGS, Q>(P, ev, smem_raw + kEvBytes, nf, 1, nl, tc)) return;
  }
  double Gh[NC], We[NC];
  lobatto<NC>(tc, sv.dt, P.gamma, 1, Gh, We);
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const size_t o = ((size_t)(slice * NC + q) * (P.ny + 1) + fj) * P.nx + col;
    FY[o] = Gh[q];
    WY[o] = We[q];
  }
}

// Update of cell (i, j) (Eq. 3.2, 3.10) into `out`; returns the cell's CFL rate (0 when the new
// state is non-physical, which raises the control block's error word).
template <int NC>
__device__ __forceinline__ double update2d_cell(const Params& P, Ctl* __restrict__ ctl, const StepView& sv,
                                                const double* st,
                                                double* out, const double* __restrict__ FX,
                                                const double* __restrict__ WX,
                                                const double* __restrict__ FY,
                                                const double* __restrict__ WY,
                                                const double* __restrict__ WC, int i, int j) {
  const double dt = sv.dt;
  const int nx = P.nx, ny = P.ny;
  using namespace shweno_tables;
  const double gw[3] = {GAUSS_W0, GAUSS_W1, GAUSS_W0};
  double Wn[NC];
  const size_t cells = (size_t)nx * ny, c = (size_t)j * nx + i;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double fl = 0.0, fr = 0.0, gb = 0.0, gt = 0.0, wl = 0.0, wr = 0.0, wb = 0.0, wt = 0.0;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      const size_t ox = ((size_t)(g * NC + q) * ny + j) * (nx + 1) + i;
      const size_t oy = ((size_t)(g * NC + q) * (ny + 1) + j) * nx + i;
      fl += gw[g] * __ldcg(FX + ox);
      fr += gw[g] * __ldcg(FX + ox + 1);
      wl += gw[g] * __ldcg(WX + ox);
      wr += gw[g] * __ldcg(WX + ox + 1);
      gb += gw[g] * __ldcg(FY + oy);
      gt += gw[g] * __ldcg(FY + oy + nx);
      wb += gw[g] * __ldcg(WY + oy);
      wt += gw[g] * __ldcg(WY + oy + nx);
    }
    const size_t oc = ((size_t)q * (ny + 1) + j) * (nx + 1) + i;
    // the derivative averages scale by reciprocals of the mesh widths (set by the host), which
    // spares the FP64 pipe twelve divisions per cell
    const double z = (__ldcg(WC + oc + (nx + 1) + 1) - __ldcg(WC + oc + (nx + 1)) - __ldcg(WC + oc + 1) + __ldcg(WC + oc)) * P.idxy;
    Wn[q] = __ldcg(st + q * cells + c) - dt / P.dx * (fr - fl) - dt / P.dy * (gt - gb);
    out[q * cells + c] = Wn[q];
    out[(NC + q) * cells + c] = (wr - wl) * P.idx;
    out[(2 * NC + q) * cells + c] = (wt - wb) * P.idy;
    out[(3 * NC + q) * cells + c] = z;
  }
  if (!cell_physical(P, Wn)) {
    atomicCAS(&ctl->err, ERR_NONE, ERR_NONPHYSICAL);
    return 0.0;
  }
  return cell_rate(P, Wn);
}

}  // namespace shweno
