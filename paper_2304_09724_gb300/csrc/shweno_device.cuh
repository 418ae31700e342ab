// Device building blocks of the ADER-SHWENO step (arXiv 2304.09724), shared by the 1D and 2D
// kernels: boundary-condition lookup, the SHWENO reconstruction pieces, the leading-term
// Riemann solvers, the eigen-upwinded linearised Riemann problem and the physical fluxes.
// Everything is FP64; the FP64 pipe (2 DFMA/clk/SM on sm_103) bounds the step, so each
// routine is arranged to spend as few FP64 instructions as the mathematics allows.
#pragma once
#include <cstdint>

#include "recon_tables.cuh"

namespace shweno {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3, BC_DMR_BOTTOM = 4,
       BC_DMR_TOP = 5 };
enum { EQ_BURGERS = 0, EQ_EULER = 1 };
enum { FLAG_ALL_NONLINEAR = 0, FLAG_ALL_LINEAR = 1, FLAG_PER_CELL = 2 };
enum { ERR_NONE = 0, ERR_NONPHYSICAL = 4, ERR_TIMEOUT = 5 };

// Problem description as the kernels see it (plain values, passed by value to every launch).
struct Params {
  int32_t dim, eq, ncomp;
  int32_t nx, ny;
  double x0, y0, dx, dy;
  double gamma;
  int32_t bc[4];          // x-low, x-high, y-low, y-high
  double inflow[4][4];    // imposed conserved state of BC_INFLOW sides
  double eps;             // epsilon of the nonlinear weights
  double gam[3];          // linear weights
  int32_t flag_mode;      // FLAG_*
  int32_t charwise;       // 1: Euler reconstructions across a face in characteristic fields
  int32_t quintic;        // 1: reading R1' (quintic p1 that also matches the cell's own V)
  // Cauchy-Kovalevskaya scale factors (m+1)/((k+1) dx) and (n+1)/((k+1) dy), set by the host
  double ckx[5][4], cky[5][4];
  double igam[3];  // 1 / gam, set by the host
  double idx, idy, idxy;  // 1 / dx, 1 / dy, 1 / (dx dy), set by the host
};

// Fills the derived members of Params (ckx, cky, igam, idx, idy, idxy) from dx, dy and gam.
inline void finalize_params(Params& P) {
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < 4; ++k) {
      P.ckx[m][k] = (m + 1) / ((k + 1) * P.dx);
      P.cky[m][k] = (m + 1) / ((k + 1) * P.dy);
    }
  for (int l = 0; l < 3; ++l) P.igam[l] = 1.0 / P.gam[l];
  P.idx = 1.0 / P.dx;
  P.idy = 1.0 / P.dy;
  P.idxy = 1.0 / (P.dx * P.dy);
}

// Device-resident time-stepping control block.  One step = begin_step, the step kernels,
// end_step; only begin_step/end_step (one thread each) write it, the step kernels only read.
struct Ctl {
  double t;                    // time of the committed state
  double dt;                   // step being taken (valid while active)
  double t_final, cfl, dt_fixed;
  int64_t nsteps;              // committed steps; the committed state is buffer nsteps % 2
  int64_t err_step;            // step index that failed (state of that index is kept)
  unsigned long long rate_cur; // max characteristic rate of the committed state (double bits)
  unsigned long long rate_next;
  int32_t mode;                // 0: fixed dt, 1: CFL with t_final
  int32_t active;              // 1 while a step is in flight
  int32_t err;                 // first error code seen (ERR_*), sticky
  int32_t pad;
};

// Snapshot of the step in flight, read with volatile loads: inside the batched persistent
// kernel the control block is rewritten by other CTAs between steps, so an L1-cached copy
// could be stale.
struct StepView {
  int odd;    // committed state is buffer 1 (else 0)
  double t;   // time of the committed state
  double dt;  // step being taken
};
__device__ __forceinline__ StepView step_view(const Ctl* c) {
  const volatile Ctl* v = c;
  StepView s;
  s.odd = (int)(v->nsteps & 1);
  s.t = v->t;
  s.dt = v->dt;
  return s;
}

// ------------------------------------------------------------------ boundary conditions
// Ghost cells are never stored: every load maps its (i, j) onto the interior, or onto an imposed
// state.  Fields: 0 = W (averages), 1 = V (x-derivative averages), 2 = Y (y-derivative averages),
// 3 = Z (xy-derivative averages).  Mirror images flip the normal momentum and every derivative
// normal to the wall.  Double Mach reflection (Example 5.10): bottom is the exact post-shock state
// for x < 1/6 and a wall beyond; the top carries the exact Mach 10 shock sampled at the ghost-cell
// centre.
__device__ __constant__ const double kDmrPost[4] = {8.0, 57.1597, -33.0012, 563.544};
__device__ __constant__ const double kDmrPre[4] = {1.4, 0.0, 0.0, 2.5};

struct Mapped {
  int i, j;       // interior cell to read (when fixed == 0)
  double sign;    // parity factor
  int fixed;      // 1: value is `value`
  double value;
};

__device__ __forceinline__ double mirror_parity(const Params& P, int f, int q, int axis) {
  double s = 1.0;
  if (P.eq == EQ_EULER && q == 1 + axis) s = -s;
  const bool has_dx = (f == 1 || f == 3), has_dy = (f == 2 || f == 3);
  if ((axis == 0 && has_dx) || (axis == 1 && has_dy)) s = -s;
  return s;
}

__device__ __forceinline__ Mapped map_cell(const Params& P, int f, int q, int i, int j, double t) {
  Mapped r{i, j, 1.0, 0, 0.0};
  if (i < 0 || i >= P.nx) {
    const int side = i < 0 ? 0 : 1;
    switch (P.bc[side]) {
      case BC_PERIODIC: r.i = ((i % P.nx) + P.nx) % P.nx; break;
      case BC_OUTFLOW: r.i = i < 0 ? 0 : P.nx - 1; break;
      case BC_REFLECTIVE:
        r.i = i < 0 ? -1 - i : 2 * P.nx - 1 - i;
        r.sign *= mirror_parity(P, f, q, 0);
        break;
      default: r.fixed = 1; r.value = f == 0 ? P.inflow[side][q] : 0.0; return r;
    }
  }
  if (P.dim == 2 && (j < 0 || j >= P.ny)) {
    const int side = j < 0 ? 2 : 3;
    int kind = P.bc[side];
    const double xc = P.x0 + (i + 0.5) * P.dx, yc = P.y0 + (j + 0.5) * P.dy;
    if (kind == BC_DMR_BOTTOM) {
      if (xc < 1.0 / 6.0) { r.fixed = 1; r.value = f == 0 ? kDmrPost[q] : 0.0; return r; }
      kind = BC_REFLECTIVE;
    }
    if (kind == BC_DMR_TOP) {
      const bool post = yc >= 1.7320508075688772 * (xc - 1.0 / 6.0) - 20.0 * t;
      r.fixed = 1;
      r.value = f == 0 ? (post ? kDmrPost[q] : kDmrPre[q]) : 0.0;
      return r;
    }
    switch (kind) {
      case BC_PERIODIC: r.j = ((j % P.ny) + P.ny) % P.ny; break;
      case BC_OUTFLOW: r.j = j < 0 ? 0 : P.ny - 1; break;
      case BC_REFLECTIVE:
        r.j = j < 0 ? -1 - j : 2 * P.ny - 1 - j;
        r.sign *= mirror_parity(P, f, q, 1);
        break;
      default: r.fixed = 1; r.value = f == 0 ? P.inflow[side][q] : 0.0; return r;
    }
  }
  return r;
}

// Loads field f, component q of cell (i, j) (any i, j) from a state laid out [f][q][ny][nx].
// Loads go through L2 only (ld.global.cg): the batched persistent kernel reads states that other
// SMs wrote earlier in the same launch.
__device__ __forceinline__ double fetch(const Params& P, const double* __restrict__ state, int f,
                                        int q, int i, int j, double t) {
  if (i >= 0 && i < P.nx && (P.dim == 1 || (j >= 0 && j < P.ny)))
    return __ldcg(state + (((size_t)f * P.ncomp + q) * P.ny + j) * P.nx + i);
  const Mapped m = map_cell(P, f, q, i, j, t);
  if (m.fixed) return m.value;
  return m.sign * __ldcg(state + (((size_t)f * P.ncomp + q) * P.ny + m.j) * P.nx + m.i);
}

// Flag of the cell a reconstruction is anchored on (1 = nonlinear weights).  Ghost cells take
// the flag of the cell they copy; imposed-state ghosts count as troubled.
__device__ __forceinline__ int cell_flag(const Params& P, const uint8_t* __restrict__ flag, int i,
                                         int j) {
  if (P.flag_mode == FLAG_ALL_NONLINEAR) return 1;
  if (P.flag_mode == FLAG_ALL_LINEAR) return 0;
  if (i < 0 || i >= P.nx) {
    const int k = P.bc[i < 0 ? 0 : 1];
    if (k == BC_PERIODIC) i = ((i % P.nx) + P.nx) % P.nx;
    else if (k == BC_OUTFLOW) i = i < 0 ? 0 : P.nx - 1;
    else if (k == BC_REFLECTIVE) i = i < 0 ? -1 - i : 2 * P.nx - 1 - i;
    else return 1;
  }
  if (P.dim == 2 && (j < 0 || j >= P.ny)) {
    const int k = P.bc[j < 0 ? 2 : 3];
    if (k == BC_PERIODIC) j = ((j % P.ny) + P.ny) % P.ny;
    else if (k == BC_OUTFLOW) j = j < 0 ? 0 : P.ny - 1;
    else if (k == BC_REFLECTIVE) j = j < 0 ? -1 - j : 2 * P.ny - 1 - j;
    else return 1;
  }
  return __ldcg(flag + (size_t)j * P.nx + i) ? 1 : 0;
}

// ------------------------------------------------------------------ SHWENO reconstruction
// Reading of Section 2.4 (procedure omitted by the paper): quartic p1 on {j-1, j, j+1} matching
// the three averages and the two outer derivative averages; linear p2 on {j-1, j}, p3 on
// {j, j+1}; beta = Jiang-Shu indicators; simple-WENO weights
//   tau = ((|b1-b2| + |b1-b3|)/2)^2,  w_l ~ gamma_l (1 + tau/(b_l + eps));
// combined polynomial p = (w1/g1) p1 + (w2 - w1 g2/g1) p2 + (w3 - w1 g3/g1) p3.
// The result is carried as (A, B, C): p = A p1 + B p2 + C p3.  Linear weights give (1, 0, 0).
struct Mix { double A, B, C; };

// Monomial coefficients of p1 in xi from (W-, W0, W+, v-, v+), v = h * derivative average.
__device__ __forceinline__ void p1_coeffs(double Wm, double W0, double Wp, double vm, double vp,
                                          double c[5]) {
  using namespace shweno_tables;
  const double s = Wm + Wp, dv = vp - vm, a = Wp - Wm, sv = vm + vp;
  c[0] = P1_C0_W0 * W0 + P1_C0_s * s + P1_C0_dv * dv;
  c[1] = P1_C1_a * a + P1_C1_sv * sv;
  c[2] = P1_C2_W0 * W0 + P1_C2_s * s + P1_C2_dv * dv;
  c[3] = P1_C3_a * a + P1_C3_sv * sv;
  c[4] = P1_C4_W0 * W0 + P1_C4_s * s + P1_C4_dv * dv;
}

// The three unnormalised weights of the cell (see shweno_mix) and their sum.
struct RawWeights { double w1, w2, w3, sum; };
__device__ __forceinline__ RawWeights shweno_raw_weights(const Params& P, double Wm, double W0, double Wp,
                                                         const double c[5]) {
  using namespace shweno_tables;
  const double b1 = c[1] * (BETA_11 * c[1] + BETA_13 * c[3]) + BETA_33 * c[3] * c[3] +
                    c[2] * (BETA_22 * c[2] + BETA_24 * c[4]) + BETA_44 * c[4] * c[4];
  const double d2 = W0 - Wm, d3 = Wp - W0;
  const double b2 = d2 * d2, b3 = d3 * d3;
  double tau = 0.5 * (fabs(b1 - b2) + fabs(b1 - b3));
  tau = tau * tau;
  const double e1 = b1 + P.eps, e2 = b2 + P.eps, e3 = b3 + P.eps;
  RawWeights r;
  r.w1 = P.gam[0] * (e1 + tau) * (e2 * e3);
  r.w2 = P.gam[1] * (e2 + tau) * (e1 * e3);
  r.w3 = P.gam[2] * (e3 + tau) * (e1 * e2);
  r.sum = r.w1 + r.w2 + r.w3;
  return r;
}
// (A, B, C) from the unnormalised weights and inv = 1 / their sum.
__device__ __forceinline__ Mix mix_from_raw(const Params& P, const RawWeights& r, double inv) {
  const double A = r.w1 * inv * P.igam[0];
  return Mix{A, r.w2 * inv - A * P.gam[1], r.w3 * inv - A * P.gam[2]};
}

__device__ __forceinline__ Mix shweno_mix(const Params& P, double Wm, double W0, double Wp,
                                          const double c[5], int nonlinear) {
  using namespace shweno_tables;
  if (!nonlinear) return Mix{1.0, 0.0, 0.0};
  const double b1 = c[1] * (BETA_11 * c[1] + BETA_13 * c[3]) + BETA_33 * c[3] * c[3] +
                    c[2] * (BETA_22 * c[2] + BETA_24 * c[4]) + BETA_44 * c[4] * c[4];
  const double d2 = W0 - Wm, d3 = Wp - W0;
  const double b2 = d2 * d2, b3 = d3 * d3;
  double tau = 0.5 * (fabs(b1 - b2) + fabs(b1 - b3));
  tau = tau * tau;
  // w_l is proportional to gam_l (1 + tau/e_l) = gam_l (e_l + tau) / e_l; scaling all three by
  // e1 e2 e3 leaves the normalised weights unchanged and leaves one division (the normalisation)
  const double e1 = b1 + P.eps, e2 = b2 + P.eps, e3 = b3 + P.eps;
  const double w1 = P.gam[0] * (e1 + tau) * (e2 * e3);
  const double w2 = P.gam[1] * (e2 + tau) * (e1 * e3);
  const double w3 = P.gam[2] * (e3 + tau) * (e1 * e2);
  const double inv = 1.0 / (w1 + w2 + w3);
  const double A = w1 * inv * P.igam[0];
  return Mix{A, w2 * inv - A * P.gam[1], w3 * inv - A * P.gam[2]};
}

// Combined-polynomial coefficients C[0..4] = A c + B p2 + C p3 (p2, p3 are linear).
__device__ __forceinline__ void mix_coeffs(const Mix& m, double Wm, double W0, double Wp,
                                           const double c[5], double C[5]) {
  C[0] = m.A * c[0] + (m.B + m.C) * W0;
  C[1] = m.A * c[1] + m.B * (W0 - Wm) + m.C * (Wp - W0);
  C[2] = m.A * c[2];
  C[3] = m.A * c[3];
  C[4] = m.A * c[4];
}

// ---- reading R1' (option): quintic p1 that also matches v0 = h * the cell's own derivative
// average.  Its even coefficients are R1's; the odd ones c1, c3, c5 come from (a, sv, v0).
// The templates below take Q = false for R1 (c[5] = 0 and v0 unused) and Q = true for R1'.
template <bool Q>
__device__ __forceinline__ void p1_coeffs_t(double Wm, double W0, double Wp, double vm, double v0,
                                            double vp, double c[6]) {
  using namespace shweno_tables;
  if constexpr (!Q) {
    p1_coeffs(Wm, W0, Wp, vm, vp, c);
    c[5] = 0.0;
  } else {
    const double s = Wm + Wp, dv = vp - vm, a = Wp - Wm, sv = vm + vp;
    c[0] = P1_C0_W0 * W0 + P1_C0_s * s + P1_C0_dv * dv;
    c[1] = QP1_C1_a * a + QP1_C1_sv * sv + QP1_C1_v0 * v0;
    c[2] = P1_C2_W0 * W0 + P1_C2_s * s + P1_C2_dv * dv;
    c[3] = QP1_C3_a * a + QP1_C3_sv * sv + QP1_C3_v0 * v0;
    c[4] = P1_C4_W0 * W0 + P1_C4_s * s + P1_C4_dv * dv;
    c[5] = QP1_C5_a * a + QP1_C5_sv * sv + QP1_C5_v0 * v0;
  }
}

template <bool Q>
__device__ __forceinline__ Mix shweno_mix_t(const Params& P, double Wm, double W0, double Wp,
                                            const double c[6], int nonlinear) {
  using namespace shweno_tables;
  if constexpr (!Q) {
    return shweno_mix(P, Wm, W0, Wp, c, nonlinear);
  } else {
    if (!nonlinear) return Mix{1.0, 0.0, 0.0};
    const double b1 = c[1] * (QBETA_11 * c[1] + QBETA_13 * c[3] + QBETA_15 * c[5]) +
                      c[3] * (QBETA_33 * c[3] + QBETA_35 * c[5]) + QBETA_55 * c[5] * c[5] +
                      c[2] * (QBETA_22 * c[2] + QBETA_24 * c[4]) + QBETA_44 * c[4] * c[4];
    const double d2 = W0 - Wm, d3 = Wp - W0;
    const double b2 = d2 * d2, b3 = d3 * d3;
    double tau = 0.5 * (fabs(b1 - b2) + fabs(b1 - b3));
    tau = tau * tau;
    const double e1 = b1 + P.eps, e2 = b2 + P.eps, e3 = b3 + P.eps;
    const double w1 = P.gam[0] * (e1 + tau) * (e2 * e3);
    const double w2 = P.gam[1] * (e2 + tau) * (e1 * e3);
    const double w3 = P.gam[2] * (e3 + tau) * (e1 * e2);
    const double inv = 1.0 / (w1 + w2 + w3);
    const double A = w1 * inv * P.igam[0];
    return Mix{A, w2 * inv - A * P.gam[1], w3 * inv - A * P.gam[2]};
  }
}

// Combined-polynomial coefficients C[0..K-1], K = 5 (R1) or 6 (R1').
template <bool Q>
__device__ __forceinline__ void mix_coeffs_t(const Mix& m, double Wm, double W0, double Wp,
                                             const double c[6], double C[6]) {
  mix_coeffs(m, Wm, W0, Wp, c, C);
  if constexpr (Q) C[5] = m.A * c[5];
}

// ------------------------------------------------------------------ physics
struct Prim {
  double rho, u, v, p, c, H;
  double ir;  // 1 / rho
};

__device__ __forceinline__ Prim euler_prim(const double* W, int ncomp, double g) {
  Prim s;
  s.rho = W[0];
  const double ir = 1.0 / s.rho;
  s.ir = ir;
  s.u = W[1] * ir;
  if (ncomp == 4) {
    s.v = W[2] * ir;
    s.p = (g - 1.0) * (W[3] - 0.5 * (W[1] * s.u + W[2] * s.v));
    s.H = (W[3] + s.p) * ir;
  } else {
    s.v = 0.0;
    s.p = (g - 1.0) * (W[2] - 0.5 * W[1] * s.u);
    s.H = (W[2] + s.p) * ir;
  }
  s.c = sqrt(g * s.p * ir);
  return s;
}

// Exact Burgers Riemann solution at x/t = 0 (shock of speed (uL+uR)/2, speed 0 keeps uL;
// rarefaction fan with the sonic value 0).
__device__ __forceinline__ double burgers_godunov(double uL, double uR) {
  if (uL > uR) return 0.5 * (uL + uR) >= 0.0 ? uL : uR;
  if (uL >= 0.0) return uL;
  if (uR <= 0.0) return uR;
  return 0.0;
}

// HLLC state at x/t = 0 (Toro Ch. 10) with Davis speeds; dir = 0 normal along x, 1 along y.
// A wave of speed exactly 0 hands over its left-hand state.
template <int NC>
__device__ __forceinline__ void hllc_state(const double* WL, const double* WR, double g, int dir,
                                           double* out) {
  const Prim L = euler_prim(WL, NC, g), R = euler_prim(WR, NC, g);
  const double uL = dir == 0 ? L.u : L.v, uR = dir == 0 ? R.u : R.v;
  const double SL = fmin(uL - L.c, uR - R.c);
  const double SR = fmax(uL + L.c, uR + R.c);
  const double mL = L.rho * (SL - uL), mR = R.rho * (SR - uR);
  const double Ss = (R.p - L.p + uL * mL - uR * mR) / (mL - mR);
  if (0.0 <= SL) {
    for (int q = 0; q < NC; ++q) out[q] = WL[q];
    return;
  }
  if (0.0 > SR) {
    for (int q = 0; q < NC; ++q) out[q] = WR[q];
    return;
  }
  // a contact within rounding of standing (|S*| <= 1e-12 c) hands over the left star state
  const bool left = -1e-12 * fmax(L.c, R.c) <= Ss;
  const double* W = left ? WL : WR;
  const Prim& K = left ? L : R;
  const double S = left ? SL : SR, un = left ? uL : uR, mK = left ? mL : mR;
  const double f = mK / (S - Ss);
  const double e = W[NC - 1] * K.ir + (Ss - un) * (Ss + K.p / mK);
  out[0] = f;
  if (NC == 3) {
    out[1] = f * Ss;
    out[2] = f * e;
  } else {
    out[1 + dir] = f * Ss;
    out[2 - dir] = f * (dir == 0 ? K.v : K.u);
    out[3] = f * e;
  }
}

// Physical flux along dir of a conserved state whose 1/rho is ir (Euler; unused for Burgers).
template <int NC>
__device__ __forceinline__ void phys_flux_ir(const double* W, double ir, double g, int dir, double* F) {
  if (NC == 1) {
    F[0] = 0.5 * W[0] * W[0];
    return;
  }
  if (NC == 3) {
    const double u = W[1] * ir;
    const double p = (g - 1.0) * (W[2] - 0.5 * W[1] * u);
    F[0] = W[1];
    F[1] = W[1] * u + p;
    F[2] = u * (W[2] + p);
    return;
  }
  const double u = W[1] * ir, v = W[2] * ir;
  const double p = (g - 1.0) * (W[3] - 0.5 * (W[1] * u + W[2] * v));
  const double un = dir == 0 ? u : v;
  F[0] = W[1 + dir];
  F[1] = W[1] * un + (dir == 0 ? p : 0.0);
  F[2] = W[2] * un + (dir == 1 ? p : 0.0);
  F[3] = un * (W[3] + p);
}

// Physical flux along dir of a conserved state.
template <int NC>
__device__ __forceinline__ void phys_flux(const double* W, double g, int dir, double* F) {
  if (NC == 1) {
    F[0] = 0.5 * W[0] * W[0];
    return;
  }
  const double ir = 1.0 / W[0];
  if (NC == 3) {
    const double u = W[1] * ir;
    const double p = (g - 1.0) * (W[2] - 0.5 * W[1] * u);
    F[0] = W[1];
    F[1] = W[1] * u + p;
    F[2] = u * (W[2] + p);
    return;
  }
  const double u = W[1] * ir, v = W[2] * ir;
  const double p = (g - 1.0) * (W[3] - 0.5 * (W[1] * u + W[2] * v));
  const double un = dir == 0 ? u : v;
  F[0] = W[1 + dir];
  F[1] = W[1] * un + (dir == 0 ? p : 0.0);
  F[2] = W[2] * un + (dir == 1 ? p : 0.0);
  F[3] = un * (W[3] + p);
}

// ------------------------------------------------------------------ linearised Riemann problem
// Eq. (2.8) / (3.7): with A = F'(W*) = R diag(lambda) L, the derivative state is
//   d* = R (H o L dL + (1-H) o L dR),  H = 1 / 0 / 1/2 for a right-moving / left-moving /
// standing wave; a wave is standing when |lambda| <= 1e-12 * scale (scale = sound speed of W*;
// Burgers: the larger face speed), so a speed that is exactly zero (normal velocity at a wall)
// is not decided by rounding;
// evaluated as d* = base + sum_k s_k (l_k . (dL - dR)) r_k over the few waves that carry a
// nonzero s_k: base = dR with s = H, or base = dL with s = H - 1, whichever needs fewer waves
// (subsonic flow needs one acoustic wave).
// Eigen-decomposition of the Euler flux Jacobian along dir (0: x, 1: y) at the primitive state
// P (NC = 3: 1D, 4: 2D): r[k] = k-th right eigenvector, l[k] = k-th left eigenvector (rows of
// R^{-1}), lam[k] = its speed; waves ordered u-c, entropy, (shear), u+c.
template <int NC>
__device__ __forceinline__ void euler_eigvecs(const Prim& P, double g, int dir, double r[NC][NC],
                                              double l[NC][NC], double lam[NC]) {
  const double un = dir == 0 ? P.u : P.v;
  const double ut = dir == 0 ? P.v : P.u;
  const double ic = 1.0 / P.c;
  const double b1 = (g - 1.0) * ic * ic;
  const double q2 = P.u * P.u + P.v * P.v;
  const double b2 = 0.5 * b1 * q2;
  lam[0] = un - P.c;
  lam[NC - 1] = un + P.c;
  const int in = 1 + dir;        // normal momentum slot
  const int it = NC == 4 ? 2 - dir : -1;  // tangential momentum slot
  // acoustic waves
  for (int side = 0; side < 2; ++side) {
    const int k = side == 0 ? 0 : NC - 1;
    const double sg = side == 0 ? -1.0 : 1.0;
    r[k][0] = 1.0;
    r[k][in] = un + sg * P.c;
    if (NC == 4) r[k][it] = ut;
    r[k][NC - 1] = P.H + sg * un * P.c;
    l[k][0] = 0.5 * (b2 - sg * un * ic);
    l[k][in] = 0.5 * (-b1 * (dir == 0 ? P.u : P.v) + sg * ic);
    if (NC == 4) l[k][it] = -0.5 * b1 * ut;
    l[k][NC - 1] = 0.5 * b1;
  }
  // entropy wave
  r[1][0] = 1.0;
  r[1][in] = un;
  if (NC == 4) r[1][it] = ut;
  r[1][NC - 1] = 0.5 * q2;
  l[1][0] = 1.0 - b2;
  l[1][in] = b1 * un;
  if (NC == 4) l[1][it] = b1 * ut;
  l[1][NC - 1] = -b1;
  lam[1] = un;
  if (NC == 4) {  // shear wave
    r[2][0] = 0.0; r[2][in] = 0.0; r[2][it] = 1.0; r[2][3] = ut;
    l[2][0] = -ut; l[2][in] = 0.0; l[2][it] = 1.0; l[2][3] = 0.0;
    lam[2] = un;
  }
}

template <int NC>
struct Upwinder {
  double r[NC][NC];  // r[k] = k-th right eigenvector
  double l[NC][NC];  // l[k] = k-th left eigenvector
  double s[NC];      // wave coefficients (0 for a wave that does not contribute)
  int base_left;

  __device__ __forceinline__ void setup(const double* Ws, double g, int dir, double burgers_scale = 0.0) {
    double lam[NC];
    double tol;
    if (NC == 1) {
      r[0][0] = 1.0; l[0][0] = 1.0; lam[0] = Ws[0];
      tol = 1e-12 * burgers_scale;
    } else {
      const Prim P = euler_prim(Ws, NC, g);
      tol = 1e-12 * P.c;
      euler_eigvecs<NC>(P, g, dir, r, l, lam);
    }
    int npos = 0, nneg = 0;
    for (int k = 0; k < NC; ++k) {
      if (lam[k] > tol) ++npos;
      else if (lam[k] < -tol) ++nneg;
    }
    // waves with H != 0 measured from dR, or with H != 1 measured from dL
    base_left = (NC - nneg) > (NC - npos) ? 1 : 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const double H = lam[k] > tol ? 1.0 : (lam[k] < -tol ? 0.0 : 0.5);
      s[k] = base_left ? H - 1.0 : H;
#pragma unroll
      for (int q = 0; q < NC; ++q) l[k][q] *= s[k];  // apply() then needs no extra product
    }
  }

  __device__ __forceinline__ void apply(const double* dL, const double* dR, double* out) const {
    double d[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      d[q] = dL[q] - dR[q];
      out[q] = base_left ? dL[q] : dR[q];
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if (s[k] != 0.0) {
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < NC; ++q) a += l[k][q] * d[q];
#pragma unroll
        for (int q = 0; q < NC; ++q) out[q] += a * r[k][q];
      }
    }
  }
};

// Basis of the characteristic-wise reconstruction across a face with normal dir: the
// eigenvectors of the Euler flux Jacobian at Wref (conserved), the mean of the two states
// next to the face.  Stencil data are projected with L (v -> L v), reconstructed field by
// field, and mapped back with R (x -> R x).
template <int NC>
struct CharBasis {
  double r[NC][NC];  // r[k] = k-th right eigenvector: physical = sum_k x_k r[k]
  double l[NC][NC];  // l[k] = k-th left eigenvector: field k = l[k] . physical
  __device__ __forceinline__ void setup(const double* Wref, double g, int dir) {
    double lam[NC];
    euler_eigvecs<NC>(euler_prim(Wref, NC, g), g, dir, r, l, lam);
  }
  __device__ __forceinline__ void to_fields(const double* v, double* out) const {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      double a = 0.0;
#pragma unroll
      for (int q = 0; q < NC; ++q) a = fma(l[k][q], v[q], a);
      out[k] = a;
    }
  }
  __device__ __forceinline__ void to_physical(const double* x, double* out) const {
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      double a = 0.0;
#pragma unroll
      for (int k = 0; k < NC; ++k) a = fma(r[k][q], x[k], a);
      out[q] = a;
    }
  }
};

// Normalised Taylor coefficients about xi0 of a polynomial of degree D given by its monomial
// coefficients e[0..D] (in place; repeated synthetic division).
template <int D>
__device__ __forceinline__ void taylor_shift_d(double* e, double xi0) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = D - 1; k >= i; --k) e[k] += xi0 * e[k + 1];
}

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

// Max characteristic rate of one cell for the CFL step size: (|u|+c)/dx (+ (|v|+c)/dy).
__device__ __forceinline__ double cell_rate(const Params& P, const double* W) {
  if (P.eq == EQ_BURGERS) {
    const double a = fabs(W[0]);
    return P.dim == 1 ? a / P.dx : a / P.dx + a / P.dy;
  }
  const Prim s = euler_prim(W, P.ncomp, P.gamma);
  if (P.dim == 1) return (fabs(s.u) + s.c) / P.dx;
  return (fabs(s.u) + s.c) / P.dx + (fabs(s.v) + s.c) / P.dy;
}

__device__ __forceinline__ bool cell_physical(const Params& P, const double* W) {
  if (P.eq == EQ_BURGERS) return isfinite(W[0]);
  const double rho = W[0];
  const double ke = P.ncomp == 4 ? 0.5 * (W[1] * W[1] + W[2] * W[2]) / rho : 0.5 * W[1] * W[1] / rho;
  const double p = (P.gamma - 1.0) * (W[P.ncomp - 1] - ke);
  return rho > 0.0 && p > 0.0 && isfinite(rho) && isfinite(p);
}

// Block-wide max of a non-negative double, then one atomicMax on its bit pattern (the order of
// non-negative IEEE doubles equals the order of their bit patterns as unsigned integers).
__device__ __forceinline__ void block_max_rate(double r, unsigned long long* dst, double* red) {
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) red[warp] = r;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    r = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0 && r > 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(r));
  }
}

}  // namespace shweno
