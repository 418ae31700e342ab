/*
 * ADER-SHWENO oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the one-stage ADER scheme with the
 * simple HWENO (SHWENO) reconstruction of Luo, Li, Qiu, Zhu and Chen, "A compact simple HWENO
 * scheme with ADER time discretization for hyperbolic conservation laws I: structured meshes"
 * (arXiv 2304.09724).  It exists so that the tests, the smoke check and the CPU-baseline leg of
 * the benchmark have something independent to compare the CUDA library against.  The library
 * never links, loads or calls it, and it shares no code, header, table or generator with the
 * library.
 *
 * Every step follows the paper's order (Section 4, Steps 1-5) and is written for a reader to
 * check against the paper by eye, with no fusion, blocking or reordering:
 *   Step 1  SHWENO reconstruction (Section 2.4 and Section 3.2).  The paper omits the 1D
 *           procedure and defers to the simple HWENO of its reference [li2021]; this file takes
 *           the following reading of it: one quartic on {I_{j-1}, I_j, I_{j+1}} that
 *           matches the three cell averages and the two outer derivative averages, two linear
 *           polynomials on {I_{j-1}, I_j} and {I_j, I_{j+1}}, linear weights (0.994, 0.003,
 *           0.003), Jiang-Shu smoothness indicators and simple-WENO nonlinear weights.
 *   Step 2  Lax-Wendroff / Cauchy-Kovalevskaya procedure (Eq. 2.6 and the 2D expressions of
 *           Section 3.1), computed as the exact Taylor coefficients of a truncated power
 *           series in (x, y, t) that satisfies W_t = -F(W)_x - G(W)_y term by term.
 *   Step 3  Leading term from the exact (Burgers) or HLLC (Euler) Riemann solver, Eq. (2.5)
 *           and (3.6); derivative terms from the linearised Riemann problems Eq. (2.8) and
 *           (3.7) with the Jacobian at the leading term.
 *   Step 4  State-expansion flux, Eq. (2.4), (2.9), (3.3)-(3.5), (3.8), with the 4-node
 *           Gauss-Lobatto rule in time (Remark 2) and the 3-node Gauss rule along faces.
 *   Step 5  Update of the cell averages, Eq. (2.2) and (3.2), and of the derivative averages
 *           from the interface values at t_{n+1}, Eq. (2.11), (2.12), (3.10), (3.11).
 * Pins for each function live in tests/test_oracle_*.py.
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ----------------------------------------------------------------------------------------
// Problem description (the oracle's own; deliberately not the library's struct).
// ----------------------------------------------------------------------------------------
enum { EQ_BURGERS = 0, EQ_EULER = 1 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3, BC_DMR_BOTTOM = 4,
       BC_DMR_TOP = 5 };

struct Problem {
  int32_t dim, eq, nx, ny;
  double x0, y0, dx, dy, gamma;
  int32_t bc[4];         // x-low, x-high, y-low, y-high
  double inflow[4][4];   // conserved state imposed by a BC_INFLOW side
  int32_t linear;        // 1: every reconstruction uses the linear weights
  double eps;            // epsilon in the nonlinear weights
  double gam[3];         // linear weights gamma_1..3 (Section 2.4)
  int32_t charwise;      // 1: Euler reconstructions across a face in characteristic fields
  int32_t quintic;       // 1: reading R1' (quintic p1 that also matches the cell's own V)
};

int ncomp(const Problem& P) {
  if (P.eq == EQ_BURGERS) return 1;
  return P.dim == 1 ? 3 : 4;
}

// ----------------------------------------------------------------------------------------
// Quadrature rules.
// ----------------------------------------------------------------------------------------
// Gauss-Lobatto with 4 nodes on [0,1] for the time integral of the flux, Eq. (2.9) and
// Remark 2 (the rule contains both t_n and t_{n+1}); exact for polynomials of degree 5.
void lobatto4(double lam[4], double w[4]) {
  lam[0] = 0.0;
  lam[1] = 0.5 - std::sqrt(5.0) / 10.0;
  lam[2] = 0.5 + std::sqrt(5.0) / 10.0;
  lam[3] = 1.0;
  w[0] = 1.0 / 12.0; w[1] = 5.0 / 12.0; w[2] = 5.0 / 12.0; w[3] = 1.0 / 12.0;
}
// Gauss-Legendre with 3 nodes on [-1/2, 1/2] for the face integrals, Eq. (3.3), (3.4), (3.10).
void gauss3(double s[3], double w[3]) {
  s[0] = -std::sqrt(15.0) / 10.0; s[1] = 0.0; s[2] = std::sqrt(15.0) / 10.0;
  w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
}

// ----------------------------------------------------------------------------------------
// Small dense linear algebra (Gaussian elimination with partial pivoting).
// ----------------------------------------------------------------------------------------
// Solves A x = b for an n x n row-major A (n <= 8).  A and b are copied.
void solve(int n, const double* A_in, const double* b_in, double* x) {
  double A[8][9];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) A[i][j] = A_in[i * n + j];
    A[i][n] = b_in[i];
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (piv != col)
      for (int j = 0; j <= n; ++j) std::swap(A[piv][j], A[col][j]);
    for (int r = col + 1; r < n; ++r) {
      double f = A[r][col] / A[col][col];
      for (int j = col; j <= n; ++j) A[r][j] -= f * A[col][j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = A[i][n];
    for (int j = i + 1; j < n; ++j) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
}
// Inverse of an n x n matrix by solving for the columns of the identity.
void invert(int n, const double* A, double* Ainv) {
  for (int c = 0; c < n; ++c) {
    double e[8] = {0}, col[8];
    e[c] = 1.0;
    solve(n, A, e, col);
    for (int r = 0; r < n; ++r) Ainv[r * n + c] = col[r];
  }
}

// ----------------------------------------------------------------------------------------
// Step 1: the SHWENO reconstruction in one dimension (Section 2.4), on the local coordinate
// xi = (x - x_j)/h in [-1/2, 1/2].  Input for cell j: the cell averages Wb = (W_{j-1}, W_j,
// W_{j+1}) and the derivative averages scaled by h, v = (h V_{j-1}, h V_j, h V_{j+1}) (the
// middle one is used by reading R1' only).  Polynomials are held as monomial coefficients
// c[0..5] in xi (c[5] = 0 for the quartic of reading R1).
// ----------------------------------------------------------------------------------------
double mono_avg(int k, double a, double b) {  // (1/(b-a)) * integral_a^b xi^k d xi, b - a = 1
  return (std::pow(b, k + 1) - std::pow(a, k + 1)) / (k + 1);
}

// p1 on the big stencil: its averages over cells -1, 0, +1 equal Wb, and the averages of its
// xi-derivative over cells -1 and +1 equal v- and v+ (reading R1 of the omitted procedure: a
// quartic, five conditions); reading R1' adds the derivative average over cell 0 (v0) and
// raises the degree to five.  The conditions are written out as rows of a matrix; its inverse
// is formed once by Gaussian elimination and applied to the data.
const double* big_poly_inverse(int quintic) {
  static double Minv[2][36];
  static bool ready[2] = {false, false};
  const int n = quintic ? 6 : 5;
  if (!ready[quintic]) {
    double A[36];
    for (int l = -1; l <= 1; ++l)
      for (int k = 0; k < n; ++k) A[(l + 1) * n + k] = mono_avg(k, l - 0.5, l + 0.5);
    const int quint_cells[3] = {-1, 1, 0}, quart_cells[2] = {-1, 1};
    const int* dcell = quintic ? quint_cells : quart_cells;
    for (int r = 0; r < n - 3; ++r) {
      int l = dcell[r];
      // average of p' over cell l = p(l + 1/2) - p(l - 1/2)
      for (int k = 0; k < n; ++k) A[(3 + r) * n + k] = std::pow(l + 0.5, k) - std::pow(l - 0.5, k);
    }
    invert(n, A, Minv[quintic]);
    ready[quintic] = true;
  }
  return Minv[quintic];
}
void big_poly(const double Wb[3], const double v[3], int quintic, double c[6]) {
  const double* Minv = big_poly_inverse(quintic);
  const int n = quintic ? 6 : 5;
  const double rhs[6] = {Wb[0], Wb[1], Wb[2], v[0], v[2], v[1]};
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += Minv[k * n + r] * rhs[r];
    c[k] = s;
  }
  if (!quintic) c[5] = 0.0;
}
// Linear polynomials on the two small stencils, matching two cell averages each.
void small_polys(const double Wb[3], double c2[6], double c3[6]) {
  for (int k = 0; k < 6; ++k) c2[k] = c3[k] = 0.0;
  c2[0] = Wb[1]; c2[1] = Wb[1] - Wb[0];   // {I_{j-1}, I_j}
  c3[0] = Wb[1]; c3[1] = Wb[2] - Wb[1];   // {I_j, I_{j+1}}
}
// Jiang-Shu smoothness indicator beta = sum_{a>=1} integral_{-1/2}^{1/2} (d^a p / d xi^a)^2,
// computed exactly by squaring the derivative polynomial and integrating its monomials.
double smoothness(const double c[6]) {
  double beta = 0.0;
  double d[6];
  for (int k = 0; k < 6; ++k) d[k] = c[k];
  for (int a = 1; a <= 5; ++a) {
    double nd[6] = {0};
    for (int k = 1; k < 6; ++k) nd[k - 1] = k * d[k];
    for (int k = 0; k < 6; ++k) d[k] = nd[k];
    double sq[11] = {0};
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) sq[i + j] += d[i] * d[j];
    for (int k = 0; k < 11; k += 2) beta += sq[k] * 2.0 * std::ldexp(1.0, -(k + 1)) / (k + 1);
  }
  return beta;
}
// Nonlinear weights of the simple-WENO form: tau = ((|b1-b2| + |b1-b3|)/2)^2 and
// w_l proportional to gamma_l (1 + tau/(beta_l + eps)).  linear=1 returns gamma itself.
void shweno_weights(const double Wb[3], const double v[3], int quintic, int linear, double eps,
                    const double gam[3], double w[3]) {
  if (linear) { for (int l = 0; l < 3; ++l) w[l] = gam[l]; return; }
  double c1[6], c2[6], c3[6];
  big_poly(Wb, v, quintic, c1);
  small_polys(Wb, c2, c3);
  double b[3] = {smoothness(c1), smoothness(c2), smoothness(c3)};
  double tau = 0.5 * (std::fabs(b[0] - b[1]) + std::fabs(b[0] - b[2]));
  tau = tau * tau;
  double s = 0.0;
  for (int l = 0; l < 3; ++l) { w[l] = gam[l] * (1.0 + tau / (b[l] + eps)); s += w[l]; }
  for (int l = 0; l < 3; ++l) w[l] /= s;
}
// Combined SHWENO polynomial p = w1 (p1/g1 - g2/g1 p2 - g3/g1 p3) + w2 p2 + w3 p3 for given
// weights.  With w = gamma it is p1.  The same weights serve the value and every derivative
// (end of Section 2.1.2).
void shweno_poly(const double Wb[3], const double v[3], int quintic, const double w[3],
                 const double gam[3], double c[6]) {
  double c1[6], c2[6], c3[6];
  big_poly(Wb, v, quintic, c1);
  small_polys(Wb, c2, c3);
  for (int k = 0; k < 6; ++k)
    c[k] = w[0] * (c1[k] / gam[0] - gam[1] / gam[0] * c2[k] - gam[2] / gam[0] * c3[k]) +
           w[1] * c2[k] + w[2] * c3[k];
}
// d^k p / d xi^k at xi, k = 0..4.
void poly_derivs(const double c[6], double xi, double d[5]) {
  for (int k = 0; k < 5; ++k) {
    double s = 0.0, xp = 1.0;
    for (int i = k; i < 6; ++i) {
      double f = 1.0;
      for (int q = 0; q < k; ++q) f *= (i - q);
      s += c[i] * f * xp;
      xp *= xi;
    }
    d[k] = s;
  }
}

// ----------------------------------------------------------------------------------------
// Physics (Eq. 2.1, 3.1, 5.1, 5.2): Burgers F = G = W^2/2; Euler with E = p/(g-1) + rho|u|^2/2.
// ----------------------------------------------------------------------------------------
void physical_flux(const Problem& P, int dir, const double* W, double* F) {
  if (P.eq == EQ_BURGERS) { F[0] = 0.5 * W[0] * W[0]; return; }
  const double g = P.gamma;
  if (P.dim == 1) {
    double rho = W[0], u = W[1] / rho, E = W[2];
    double p = (g - 1.0) * (E - 0.5 * rho * u * u);
    F[0] = rho * u; F[1] = rho * u * u + p; F[2] = u * (E + p);
    return;
  }
  double rho = W[0], u = W[1] / rho, v = W[2] / rho, E = W[3];
  double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  double un = dir == 0 ? u : v;
  F[0] = rho * un;
  F[1] = W[1] * un + (dir == 0 ? p : 0.0);
  F[2] = W[2] * un + (dir == 1 ? p : 0.0);
  F[3] = un * (E + p);
}

// ----------------------------------------------------------------------------------------
// Step 3a: leading term, the Godunov state at x/t = 0 of the conventional Riemann problem
// Eq. (2.5) / (3.6).
// ----------------------------------------------------------------------------------------
// Exact solution of the Burgers Riemann problem sampled at x/t = 0.  A shock of speed
// (uL+uR)/2 when uL > uR (speed 0 takes uL), otherwise a rarefaction fan (sonic point -> 0).
double burgers_godunov(double uL, double uR) {
  if (uL > uR) {
    double s = 0.5 * (uL + uR);
    return s >= 0.0 ? uL : uR;
  }
  if (uL >= 0.0) return uL;
  if (uR <= 0.0) return uR;
  return 0.0;
}
// HLLC state at x/t = 0 (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
// Section 10.4): Davis wave-speed estimates S_L = min(uL-cL, uR-cR), S_R = max(uL+cL, uR+cR),
// contact speed S*, star states U*_K = rho_K (S_K-u_K)/(S_K-S*) (1, S*, v_K,
// E_K/rho_K + (S*-u_K)(S* + p_K/(rho_K (S_K-u_K)))) with the normal and tangential velocity
// placed by the face direction.  A wave of speed exactly 0 hands over its left-hand state; a
// contact whose speed is within STANDING_WAVE_TOL x (larger sound speed) of zero counts as
// standing (the normal velocity of a gas at rest is zero in exact arithmetic, and rounding must
// not pick the star state).
const double STANDING_WAVE_TOL = 1e-12;

void hllc_state(const Problem& P, int dir, const double* WL, const double* WR, double* out) {
  const double g = P.gamma;
  const int nc = ncomp(P);
  auto prim = [&](const double* W, double& rho, double& un, double& ut, double& p, double& c) {
    rho = W[0];
    if (nc == 3) { un = W[1] / rho; ut = 0.0; p = (g - 1.0) * (W[2] - 0.5 * rho * un * un); }
    else {
      double u = W[1] / rho, v = W[2] / rho;
      un = dir == 0 ? u : v; ut = dir == 0 ? v : u;
      p = (g - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v));
    }
    c = std::sqrt(g * p / rho);
  };
  double rL, uL, tL, pL, cL, rR, uR, tR, pR, cR;
  prim(WL, rL, uL, tL, pL, cL);
  prim(WR, rR, uR, tR, pR, cR);
  double SL = std::fmin(uL - cL, uR - cR);
  double SR = std::fmax(uL + cL, uR + cR);
  double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
              (rL * (SL - uL) - rR * (SR - uR));
  auto star = [&](const double* W, double r, double u, double t, double p, double S, double* U) {
    double f = r * (S - u) / (S - Ss);
    double Ek = W[nc - 1];
    double e = Ek / r + (Ss - u) * (Ss + p / (r * (S - u)));
    U[0] = f;
    if (nc == 3) { U[1] = f * Ss; U[2] = f * e; }
    else {
      U[1 + dir] = f * Ss;
      U[2 - dir] = f * t;
      U[3] = f * e;
    }
  };
  if (0.0 <= SL) { for (int q = 0; q < nc; ++q) out[q] = WL[q]; }
  else if (-STANDING_WAVE_TOL * std::fmax(cL, cR) <= Ss) star(WL, rL, uL, tL, pL, SL, out);
  else if (0.0 <= SR) star(WR, rR, uR, tR, pR, SR, out);
  else { for (int q = 0; q < nc; ++q) out[q] = WR[q]; }
}

// ----------------------------------------------------------------------------------------
// Step 3b: linearised Riemann problems for the derivatives, Eq. (2.8) / (3.7).  With
// A = F'(W*) = R diag(lambda) L the solution at x/t = 0 is R (H o L d_L + (1-H) o L d_R) where
// H = 1 for lambda > 0, 0 for lambda < 0 and 1/2 for a standing wave (the average of both
// sides).  A wave counts as standing when |lambda| <= 1e-12 * scale (scale: the sound speed of
// W*, or for Burgers the larger face speed), so that a speed that is zero in exact arithmetic
// (the normal velocity at a reflective wall) is not decided by rounding.
// Right eigenvectors of the Euler Jacobian (Toro, Section 3.2), L = R^{-1} by elimination.
// ----------------------------------------------------------------------------------------
void eigensystem(const Problem& P, int dir, const double* W, double* lam, double* R) {
  const int nc = ncomp(P);
  if (P.eq == EQ_BURGERS) { lam[0] = W[0]; R[0] = 1.0; return; }
  const double g = P.gamma;
  if (nc == 3) {
    double rho = W[0], u = W[1] / rho, E = W[2];
    double p = (g - 1.0) * (E - 0.5 * rho * u * u);
    double c = std::sqrt(g * p / rho), H = (E + p) / rho;
    double r[3][3] = {{1.0, u - c, H - u * c}, {1.0, u, 0.5 * u * u}, {1.0, u + c, H + u * c}};
    lam[0] = u - c; lam[1] = u; lam[2] = u + c;
    for (int k = 0; k < 3; ++k)
      for (int q = 0; q < 3; ++q) R[q * 3 + k] = r[k][q];
    return;
  }
  double rho = W[0], u = W[1] / rho, v = W[2] / rho, E = W[3];
  double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  double c = std::sqrt(g * p / rho), H = (E + p) / rho;
  double un = dir == 0 ? u : v;
  double r[4][4];
  if (dir == 0) {
    double rr[4][4] = {{1.0, u - c, v, H - u * c}, {1.0, u, v, 0.5 * (u * u + v * v)},
                       {0.0, 0.0, 1.0, v}, {1.0, u + c, v, H + u * c}};
    std::memcpy(r, rr, sizeof(r));
  } else {
    double rr[4][4] = {{1.0, u, v - c, H - v * c}, {1.0, u, v, 0.5 * (u * u + v * v)},
                       {0.0, 1.0, 0.0, u}, {1.0, u, v + c, H + v * c}};
    std::memcpy(r, rr, sizeof(r));
  }
  lam[0] = un - c; lam[1] = un; lam[2] = un; lam[3] = un + c;
  for (int k = 0; k < 4; ++k)
    for (int q = 0; q < 4; ++q) R[q * 4 + k] = r[k][q];
}

void upwind(int nc, const double* lam, double scale, const double* R, const double* L,
            const double* dL, const double* dR, double* out) {
  double a[4];
  const double tol = STANDING_WAVE_TOL * scale;
  for (int k = 0; k < nc; ++k) {
    double aL = 0.0, aR = 0.0;
    for (int q = 0; q < nc; ++q) { aL += L[k * nc + q] * dL[q]; aR += L[k * nc + q] * dR[q]; }
    double H = lam[k] > tol ? 1.0 : (lam[k] < -tol ? 0.0 : 0.5);
    a[k] = H * aL + (1.0 - H) * aR;
  }
  for (int q = 0; q < nc; ++q) {
    double s = 0.0;
    for (int k = 0; k < nc; ++k) s += R[q * nc + k] * a[k];
    out[q] = s;
  }
}

// Speed scale of the standing-wave test: sound speed of W* (Euler), max |u| of the face states
// (Burgers).
double wave_scale(const Problem& P, const double* Ws, double uL, double uR) {
  if (P.eq == EQ_BURGERS) return std::fmax(std::fabs(uL), std::fabs(uR));
  const int nc = ncomp(P);
  double rho = Ws[0], ke = 0.0;
  for (int q = 1; q < nc - 1; ++q) ke += 0.5 * Ws[q] * Ws[q] / rho;
  double p = (P.gamma - 1.0) * (Ws[nc - 1] - ke);
  return std::sqrt(P.gamma * p / rho);
}

// ----------------------------------------------------------------------------------------
// Step 2: the Cauchy-Kovalevskaya procedure by truncated power series.
// A series s holds the normalised Taylor coefficients s[m][n][k] = d^{m+n+k} f / (dx^m dy^n
// dt^k) / (m! n! k!) at the interface point, for m + n + k <= 4.  Products and quotients of
// series are the Cauchy products of the coefficient arrays.  The PDE W_t = -F_x - G_y says
// (k+1) a[m][n][k+1] = -(m+1) f[m+1][n][k] - (n+1) g[m][n+1][k]; the time slices are filled one
// after another, each from fluxes evaluated on the slices already known.  This gives the full
// nonlinear expressions of Eq. (2.6) and of Section 3.1 (written out there only for the first
// derivatives) to fourth order.
// ----------------------------------------------------------------------------------------
const int ORD = 4;
struct Ser { double c[5][5][5]; };

void ser_zero(Ser& s) { std::memset(s.c, 0, sizeof(s.c)); }
bool in_range(int m, int n, int k) { return m + n + k <= ORD; }

Ser ser_mul(const Ser& a, const Ser& b) {
  Ser r; ser_zero(r);
  for (int m = 0; m <= ORD; ++m)
    for (int n = 0; m + n <= ORD; ++n)
      for (int k = 0; m + n + k <= ORD; ++k) {
        double s = 0.0;
        for (int p = 0; p <= m; ++p)
          for (int q = 0; q <= n; ++q)
            for (int t = 0; t <= k; ++t) s += a.c[p][q][t] * b.c[m - p][n - q][k - t];
        r.c[m][n][k] = s;
      }
  return r;
}
// q = a / b, from b * q = a solved index by index in lexicographic order (every index below a
// given one in the product order comes first).
Ser ser_div(const Ser& a, const Ser& b) {
  Ser q; ser_zero(q);
  for (int m = 0; m <= ORD; ++m)
    for (int n = 0; m + n <= ORD; ++n)
      for (int k = 0; m + n + k <= ORD; ++k) {
        double s = a.c[m][n][k];
        for (int p = 0; p <= m; ++p)
          for (int r = 0; r <= n; ++r)
            for (int t = 0; t <= k; ++t) {
              if (p == m && r == n && t == k) continue;
              s -= b.c[m - p][n - r][k - t] * q.c[p][r][t];
            }
        q.c[m][n][k] = s / b.c[0][0][0];
      }
  return q;
}
Ser ser_lin(double a, const Ser& x, double b, const Ser& y) {
  Ser r; ser_zero(r);
  for (int m = 0; m <= ORD; ++m)
    for (int n = 0; n <= ORD; ++n)
      for (int k = 0; k <= ORD; ++k) r.c[m][n][k] = a * x.c[m][n][k] + b * y.c[m][n][k];
  return r;
}

// Flux series F (x-direction) and G (y-direction) of the state series W.
void flux_series(const Problem& P, const Ser* W, Ser* F, Ser* G) {
  const int nc = ncomp(P);
  const double g = P.gamma;
  if (P.eq == EQ_BURGERS) {
    Ser h = ser_mul(W[0], W[0]);
    F[0] = ser_lin(0.5, h, 0.0, h);
    if (P.dim == 2) G[0] = F[0]; else ser_zero(G[0]);
    return;
  }
  if (nc == 3) {
    Ser u = ser_div(W[1], W[0]);
    Ser mu = ser_mul(W[1], u);
    Ser p = ser_lin(g - 1.0, W[2], -0.5 * (g - 1.0), mu);
    Ser H = ser_lin(1.0, W[2], 1.0, p);
    F[0] = W[1];
    F[1] = ser_lin(1.0, mu, 1.0, p);
    F[2] = ser_mul(u, H);
    for (int q = 0; q < 3; ++q) ser_zero(G[q]);
    return;
  }
  Ser u = ser_div(W[1], W[0]);
  Ser v = ser_div(W[2], W[0]);
  Ser mu = ser_mul(W[1], u);
  Ser mv = ser_mul(W[1], v);
  Ser nv = ser_mul(W[2], v);
  Ser ke = ser_lin(0.5, mu, 0.5, nv);
  Ser p = ser_lin(g - 1.0, W[3], -(g - 1.0), ke);
  Ser H = ser_lin(1.0, W[3], 1.0, p);
  F[0] = W[1];
  F[1] = ser_lin(1.0, mu, 1.0, p);
  F[2] = mv;
  F[3] = ser_mul(u, H);
  G[0] = W[2];
  G[1] = mv;
  G[2] = ser_lin(1.0, nv, 1.0, p);
  G[3] = ser_mul(v, H);
}

// Fills the time slices k = 1..4 of W from its spatial slice k = 0.
void cauchy_kovalevskaya(const Problem& P, Ser* W) {
  const int nc = ncomp(P);
  for (int k = 0; k < ORD; ++k) {
    Ser F[4], G[4];
    flux_series(P, W, F, G);
    for (int q = 0; q < nc; ++q)
      for (int m = 0; m <= ORD; ++m)
        for (int n = 0; m + n + k + 1 <= ORD; ++n)
          W[q].c[m][n][k + 1] =
              -((m + 1) * F[q].c[m + 1][n][k] + (n + 1) * G[q].c[m][n + 1][k]) / (k + 1);
  }
}

// ----------------------------------------------------------------------------------------
// Steps 3-4 at one interface quadrature point: given the one-sided spatial derivatives
// dL[q][m][n], dR[q][m][n] = d^{m+n} W_q / dx^m dy^n (m+n <= 4; in 1D n = 0), direction dir of
// the face normal, returns the time-Taylor coefficients tc[q][k] = d^k W*/dt^k / k!.
// ----------------------------------------------------------------------------------------
typedef double Deriv[5][5];  // [m][n]

double factorial(int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; }

void grp_point(const Problem& P, int dir, const Deriv* dL, const Deriv* dR, double tc[4][5]) {
  const int nc = ncomp(P);
  double WL[4], WR[4], Ws[4];
  for (int q = 0; q < nc; ++q) { WL[q] = dL[q][0][0]; WR[q] = dR[q][0][0]; }
  if (P.eq == EQ_BURGERS) Ws[0] = burgers_godunov(WL[0], WR[0]);
  else hllc_state(P, dir, WL, WR, Ws);
  double lam[4], R[16], L[16];
  eigensystem(P, dir, Ws, lam, R);
  invert(nc, R, L);
  const double scale = wave_scale(P, Ws, WL[0], WR[0]);
  Ser S[4];
  for (int q = 0; q < nc; ++q) { ser_zero(S[q]); S[q].c[0][0][0] = Ws[q]; }
  const int nmax = P.dim == 2 ? ORD : 0;
  for (int m = 0; m <= ORD; ++m)
    for (int n = 0; n <= nmax && m + n <= ORD; ++n) {
      if (m == 0 && n == 0) continue;
      double a[4], b[4], o[4];
      for (int q = 0; q < nc; ++q) { a[q] = dL[q][m][n]; b[q] = dR[q][m][n]; }
      upwind(nc, lam, scale, R, L, a, b, o);
      for (int q = 0; q < nc; ++q) S[q].c[m][n][0] = o[q] / (factorial(m) * factorial(n));
    }
  cauchy_kovalevskaya(P, S);
  for (int q = 0; q < nc; ++q)
    for (int k = 0; k <= ORD; ++k) tc[q][k] = S[q].c[0][0][k];
}

// State of the Taylor expansion Eq. (2.4) at tau.
void taylor_state(int nc, const double tc[4][5], double tau, double* W) {
  for (int q = 0; q < nc; ++q) {
    double s = 0.0, tp = 1.0;
    for (int k = 0; k <= ORD; ++k) { s += tc[q][k] * tp; tp *= tau; }
    W[q] = s;
  }
}
// Time-averaged flux of Eq. (2.9) with the Lobatto rule, and the state at tau = dt used by
// Eq. (2.11) / (3.10) (Remark 1).
void ader_flux(const Problem& P, int dir, const double tc[4][5], double dt, double* Fhat,
               double* Wend) {
  const int nc = ncomp(P);
  double lam[4], w[4];
  lobatto4(lam, w);
  for (int q = 0; q < nc; ++q) Fhat[q] = 0.0;
  for (int a = 0; a < 4; ++a) {
    double W[4], F[4];
    taylor_state(nc, tc, lam[a] * dt, W);
    physical_flux(P, dir, W, F);
    for (int q = 0; q < nc; ++q) Fhat[q] += w[a] * F[q];
  }
  taylor_state(nc, tc, dt, Wend);
}

// ----------------------------------------------------------------------------------------
// Boundary conditions through ghost-cell lookup (Section 5 examples): periodic, outflow
// (zero-order extrapolation of every cell quantity), reflective walls (mirror images with the
// normal momentum and every derivative normal to the wall changing sign as the parity of the
// mirrored field requires), an imposed inflow state, and the two double-Mach-reflection sides
// of Example 5.10 (bottom: exact post-shock state for x < 1/6, reflective wall beyond; top:
// exact Mach 10 shock at x = 1/6 + (y + 20 t)/sqrt(3), sampled at the ghost-cell centre).
// Fields: 0 = W (averages), 1 = V (x-derivative averages), 2 = Y (y-derivative), 3 = Z (xy).
// ----------------------------------------------------------------------------------------
const double DMR_POST[4] = {8.0, 57.1597, -33.0012, 563.544};
const double DMR_PRE[4] = {1.4, 0.0, 0.0, 2.5};

struct State {
  const Problem* P;
  const double* f[4];  // W, V, Y, Z arrays [comp][ny][nx] (1D: ny = 1)
  const uint8_t* flag; // per-cell troubled flag, or null (all nonlinear)
  double t;
};

// Parity of field f, component q under the mirror normal to axis (0 = x, 1 = y).
double mirror_sign(const Problem& P, int f, int q, int axis) {
  double s = 1.0;
  int normal_momentum = (P.eq == EQ_EULER) ? 1 + axis : -1;
  if (q == normal_momentum) s = -s;
  bool has_dx = (f == 1 || f == 3), has_dy = (f == 2 || f == 3);
  if ((axis == 0 && has_dx) || (axis == 1 && has_dy)) s = -s;
  return s;
}

double fetch(const State& S, int f, int q, int i, int j) {
  const Problem& P = *S.P;
  const int i0 = i, j0 = j;
  double sign = 1.0;
  if (i < 0 || i >= P.nx) {
    int kind = i < 0 ? P.bc[0] : P.bc[1];
    int side = i < 0 ? 0 : 1;
    switch (kind) {
      case BC_PERIODIC: i = ((i % P.nx) + P.nx) % P.nx; break;
      case BC_OUTFLOW: i = i < 0 ? 0 : P.nx - 1; break;
      case BC_REFLECTIVE: i = i < 0 ? -1 - i : 2 * P.nx - 1 - i; sign *= mirror_sign(P, f, q, 0); break;
      default: return f == 0 ? P.inflow[side][q] : 0.0;  // imposed state, zero derivatives
    }
  }
  if (P.dim == 2 && (j < 0 || j >= P.ny)) {
    int kind = j < 0 ? P.bc[2] : P.bc[3];
    int side = j < 0 ? 2 : 3;
    double xc = P.x0 + (i0 + 0.5) * P.dx, yc = P.y0 + (j0 + 0.5) * P.dy;
    if (kind == BC_DMR_BOTTOM) {
      if (xc < 1.0 / 6.0) return f == 0 ? DMR_POST[q] : 0.0;
      kind = BC_REFLECTIVE;
    }
    if (kind == BC_DMR_TOP) {
      bool post = yc >= std::sqrt(3.0) * (xc - 1.0 / 6.0) - 20.0 * S.t;
      return f == 0 ? (post ? DMR_POST[q] : DMR_PRE[q]) : 0.0;
    }
    switch (kind) {
      case BC_PERIODIC: j = ((j % P.ny) + P.ny) % P.ny; break;
      case BC_OUTFLOW: j = j < 0 ? 0 : P.ny - 1; break;
      case BC_REFLECTIVE: j = j < 0 ? -1 - j : 2 * P.ny - 1 - j; sign *= mirror_sign(P, f, q, 1); break;
      default: return f == 0 ? P.inflow[side][q] : 0.0;
    }
  }
  return sign * S.f[f][((size_t)q * P.ny + j) * P.nx + i];
}
// Flag of the cell a reconstruction is anchored on; ghost cells take the flag of the interior
// cell they copy, imposed-state ghosts count as troubled.
int cell_flag(const State& S, int i, int j) {
  if (!S.flag) return 1;
  const Problem& P = *S.P;
  if (i < 0 || i >= P.nx) {
    int kind = i < 0 ? P.bc[0] : P.bc[1];
    if (kind == BC_PERIODIC) i = ((i % P.nx) + P.nx) % P.nx;
    else if (kind == BC_OUTFLOW) i = i < 0 ? 0 : P.nx - 1;
    else if (kind == BC_REFLECTIVE) i = i < 0 ? -1 - i : 2 * P.nx - 1 - i;
    else return 1;
  }
  if (P.dim == 2 && (j < 0 || j >= P.ny)) {
    int kind = j < 0 ? P.bc[2] : P.bc[3];
    if (kind == BC_PERIODIC) j = ((j % P.ny) + P.ny) % P.ny;
    else if (kind == BC_OUTFLOW) j = j < 0 ? 0 : P.ny - 1;
    else if (kind == BC_REFLECTIVE) j = j < 0 ? -1 - j : 2 * P.ny - 1 - j;
    else return 1;
  }
  return S.flag[(size_t)j * P.nx + i] ? 1 : 0;
}

// One 1D SHWENO reconstruction evaluated at xi: derivatives d^k/dxi^k, k = 0..4.
void recon_eval(const Problem& P, const double Wb[3], const double v[3], int nonlinear,
                double xi, double d[5]) {
  double w[3], c[6];
  shweno_weights(Wb, v, P.quintic, P.linear || !nonlinear, P.eps, P.gam, w);
  shweno_poly(Wb, v, P.quintic, w, P.gam, c);
  poly_derivs(c, xi, d);
}

// ----------------------------------------------------------------------------------------
// Fields of the reconstruction across a face (an option; the paper reconstructs the conserved
// variables).  Componentwise: R = L = identity.  Characteristic-wise (Euler, P.charwise = 1):
// the stencil data of both sides are projected with the left eigenvectors L = R^{-1} of the
// Jacobian along the face normal at W_ref, reconstructed field by field, and mapped back with R.
// ----------------------------------------------------------------------------------------
void basis_at(const Problem& P, int dir, const double* Wref, double* R, double* L) {
  const int nc = ncomp(P);
  if (!P.charwise || nc == 1) {
    for (int a = 0; a < nc * nc; ++a) R[a] = L[a] = (a % (nc + 1) == 0) ? 1.0 : 0.0;
    return;
  }
  double lam[4];
  eigensystem(P, dir, Wref, lam, R);
  invert(nc, R, L);
}
// W_ref = mean of the cell averages of cells (i0, j0) and (i1, j1) on the two sides.
void face_basis(const Problem& P, int dir, const State& S, int i0, int j0, int i1, int j1,
                double* R, double* L) {
  const int nc = ncomp(P);
  double Wref[4];
  for (int q = 0; q < nc; ++q) Wref[q] = 0.5 * (fetch(S, 0, q, i0, j0) + fetch(S, 0, q, i1, j1));
  basis_at(P, dir, Wref, R, L);
}
// out = M x for an nc x nc row-major matrix.
void project(int nc, const double* M, const double* x, double* out) {
  for (int a = 0; a < nc; ++a) {
    double s = 0.0;
    for (int b = 0; b < nc; ++b) s += M[a * nc + b] * x[b];
    out[a] = s;
  }
}

// ----------------------------------------------------------------------------------------
// One time step in 1D (Section 2; Section 4 Steps 1-5).
// ----------------------------------------------------------------------------------------
void step1d(const Problem& P, const State& S, double dt, double* Wn, double* Vn) {
  const int nc = ncomp(P), N = P.nx;
  const double h = P.dx;
  std::vector<double> Fh((size_t)(N + 1) * nc), We((size_t)(N + 1) * nc);
  for (int fc = 0; fc <= N; ++fc) {  // face between cells fc-1 and fc
    Deriv dL[4], dR[4];
    std::memset(dL, 0, sizeof(dL)); std::memset(dR, 0, sizeof(dR));
    // projection onto the fields in which each side is reconstructed: the identity
    // (componentwise), or the left eigenvectors of F'(W_ref) at the mean of the two cells
    double Rm[16], Lm[16];
    face_basis(P, 0, S, fc - 1, 0, fc, 0, Rm, Lm);
    for (int side = 0; side < 2; ++side) {
      const int cell = fc - 1 + side;
      double Wc[3][4], Vc[3][4];  // stencil data in the reconstruction fields
      for (int r = 0; r < 3; ++r) {
        double w[4];
        for (int q = 0; q < nc; ++q) w[q] = fetch(S, 0, q, cell - 1 + r, 0);
        project(nc, Lm, w, Wc[r]);
        for (int q = 0; q < nc; ++q) w[q] = h * fetch(S, 1, q, cell - 1 + r, 0);
        project(nc, Lm, w, Vc[r]);
      }
      double dk[4][5];
      for (int k = 0; k < nc; ++k) {
        double Wb[3] = {Wc[0][k], Wc[1][k], Wc[2][k]};
        double v[3] = {Vc[0][k], Vc[1][k], Vc[2][k]};
        recon_eval(P, Wb, v, cell_flag(S, cell, 0), side == 0 ? 0.5 : -0.5, dk[k]);
      }
      for (int m = 0; m <= ORD; ++m) {
        double a[4], b[4];
        for (int k = 0; k < nc; ++k) a[k] = dk[k][m];
        project(nc, Rm, a, b);
        for (int q = 0; q < nc; ++q) (side == 0 ? dL : dR)[q][m][0] = b[q] / std::pow(h, m);
      }
    }
    double tc[4][5], F[4], Wend[4];
    grp_point(P, 0, dL, dR, tc);
    ader_flux(P, 0, tc, dt, F, Wend);
    for (int q = 0; q < nc; ++q) { Fh[(size_t)fc * nc + q] = F[q]; We[(size_t)fc * nc + q] = Wend[q]; }
  }
  for (int j = 0; j < N; ++j)
    for (int q = 0; q < nc; ++q) {
      size_t o = (size_t)q * N + j;
      Wn[o] = S.f[0][o] - dt / h * (Fh[(size_t)(j + 1) * nc + q] - Fh[(size_t)j * nc + q]);
      Vn[o] = (We[(size_t)(j + 1) * nc + q] - We[(size_t)j * nc + q]) / h;
    }
}

// ----------------------------------------------------------------------------------------
// One time step in 2D (Section 3; Section 4 Steps 1-5), dimension by dimension (Section 3.2).
// ----------------------------------------------------------------------------------------
// y-direction reconstruction in column i, row j at eta: out[set][q][n] = d^n/dy^n of the line
// average in x of W (set 0, from {W, Y}) or of W_x (set 1, from {V, Z}) at y = y_j + eta dy.
void ypass(const State& S, int i, int j, double eta, double out[2][4][5]) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  for (int set = 0; set < 2; ++set)
    for (int q = 0; q < nc; ++q) {
      int fa = set == 0 ? 0 : 1, fd = set == 0 ? 2 : 3;
      double Wb[3] = {fetch(S, fa, q, i, j - 1), fetch(S, fa, q, i, j), fetch(S, fa, q, i, j + 1)};
      double v[3] = {P.dy * fetch(S, fd, q, i, j - 1), P.dy * fetch(S, fd, q, i, j),
                     P.dy * fetch(S, fd, q, i, j + 1)};
      double d[5];
      recon_eval(P, Wb, v, cell_flag(S, i, j), eta, d);
      for (int n = 0; n <= ORD; ++n) out[set][q][n] = d[n] / std::pow(P.dy, n);
    }
}
// x-direction counterpart: out[set][q][m] = d^m/dx^m of the line average in y of W (set 0,
// from {W, V}) or of W_y (set 1, from {Y, Z}) at x = x_i + xi dx.
void xpass(const State& S, int i, int j, double xi, double out[2][4][5]) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  for (int set = 0; set < 2; ++set)
    for (int q = 0; q < nc; ++q) {
      int fa = set == 0 ? 0 : 2, fd = set == 0 ? 1 : 3;
      double Wb[3] = {fetch(S, fa, q, i - 1, j), fetch(S, fa, q, i, j), fetch(S, fa, q, i + 1, j)};
      double v[3] = {P.dx * fetch(S, fd, q, i - 1, j), P.dx * fetch(S, fd, q, i, j),
                     P.dx * fetch(S, fd, q, i + 1, j)};
      double d[5];
      recon_eval(P, Wb, v, cell_flag(S, i, j), xi, d);
      for (int m = 0; m <= ORD; ++m) out[set][q][m] = d[m] / std::pow(P.dx, m);
    }
}
// Second pass across the face.  line[c][set][q][k] holds the first-pass output of the four
// cells c = 0..3 of the stencil (cells a-1, a, a+1, a+2 along the normal; face between a and
// a+1); k is the derivative order along the face.  The weights of each side come from the
// k = 0 data and serve every k (reading of Section 3.2 with the remark ending Section 2.1.2).
// Returns d[q][p][k]: p-th normal derivative of the k-th tangential derivative.
// Wref: state whose flux-Jacobian eigenvectors along dir span the reconstruction fields (used
// when P.charwise is set).
void second_pass(const Problem& P, int dir, double hn, const double line_in[4][2][4][5], int flagL,
                 int flagR, const double* Wref, Deriv* dL_out, Deriv* dR_out) {
  const int nc = ncomp(P);
  double Rm[16], Lm[16];
  basis_at(P, dir, Wref, Rm, Lm);
  double line[4][2][4][5];
  for (int c = 0; c < 4; ++c)
    for (int set = 0; set < 2; ++set)
      for (int k = 0; k <= ORD; ++k) {
        double x[4], y[4];
        for (int q = 0; q < nc; ++q) x[q] = line_in[c][set][q][k];
        project(nc, Lm, x, y);
        for (int q = 0; q < nc; ++q) line[c][set][q][k] = y[q];
      }
  Deriv dL[4], dR[4];
  std::memset(dL, 0, sizeof(dL)); std::memset(dR, 0, sizeof(dR));
  for (int side = 0; side < 2; ++side) {
    int base = side;  // stencil cells base..base+2; the reconstructed cell is base+1
    double xi = side == 0 ? 0.5 : -0.5;
    int fl = side == 0 ? flagL : flagR;
    for (int q = 0; q < nc; ++q) {
      double w[3];
      {
        double Wb[3] = {line[base][0][q][0], line[base + 1][0][q][0], line[base + 2][0][q][0]};
        double v[3] = {hn * line[base][1][q][0], hn * line[base + 1][1][q][0], hn * line[base + 2][1][q][0]};
        shweno_weights(Wb, v, P.quintic, P.linear || !fl, P.eps, P.gam, w);
      }
      for (int k = 0; k <= ORD; ++k) {
        double Wb[3] = {line[base][0][q][k], line[base + 1][0][q][k], line[base + 2][0][q][k]};
        double v[3] = {hn * line[base][1][q][k], hn * line[base + 1][1][q][k], hn * line[base + 2][1][q][k]};
        double c[6], d[5];
        shweno_poly(Wb, v, P.quintic, w, P.gam, c);
        poly_derivs(c, xi, d);
        for (int p = 0; p + k <= ORD; ++p) (side == 0 ? dL : dR)[q][p][k] = d[p] / std::pow(hn, p);
      }
    }
  }
  for (int side = 0; side < 2; ++side) {
    const Deriv* in = side == 0 ? dL : dR;
    Deriv* out = side == 0 ? dL_out : dR_out;
    for (int p = 0; p <= ORD; ++p)
      for (int k = 0; p + k <= ORD; ++k) {
        double x[4], y[4];
        for (int q = 0; q < nc; ++q) x[q] = in[q][p][k];
        project(nc, Rm, x, y);
        for (int q = 0; q < nc; ++q) out[q][p][k] = y[q];
      }
  }
}
// Swaps the roles of the indices of a derivative table so that [m][n] is always
// (x-order, y-order).
void to_xy(int nc, const Deriv* in, int normal_is_x, Deriv* out) {
  for (int q = 0; q < nc; ++q)
    for (int a = 0; a <= ORD; ++a)
      for (int b = 0; a + b <= ORD; ++b) {
        if (normal_is_x) out[q][a][b] = in[q][a][b];
        else out[q][b][a] = in[q][a][b];
      }
}

// Time-averaged flux F-hat (Eq. 3.3 with the Gauss sum of Eq. 3.8) and Gauss-weighted state
// at t_{n+1} (the sum in Eq. 3.10) of the x-face (i+1/2, j).
void xface(const State& S, int i, int j, double dt, double* Fs, double* Ws) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  double gs[3], gw[3];
  gauss3(gs, gw);
  for (int q = 0; q < nc; ++q) Fs[q] = Ws[q] = 0.0;
  for (int g = 0; g < 3; ++g) {
    double line[4][2][4][5];
    for (int c = 0; c < 4; ++c) ypass(S, i - 1 + c, j, gs[g], line[c]);
    Deriv a[4], b[4], dL[4], dR[4];
    double Wref[4];
    for (int q = 0; q < nc; ++q) Wref[q] = 0.5 * (fetch(S, 0, q, i, j) + fetch(S, 0, q, i + 1, j));
    second_pass(P, 0, P.dx, line, cell_flag(S, i, j), cell_flag(S, i + 1, j), Wref, a, b);
    to_xy(nc, a, 1, dL); to_xy(nc, b, 1, dR);
    double tc[4][5], F[4], We[4];
    grp_point(P, 0, dL, dR, tc);
    ader_flux(P, 0, tc, dt, F, We);
    for (int q = 0; q < nc; ++q) { Fs[q] += gw[g] * F[q]; Ws[q] += gw[g] * We[q]; }
  }
}
// Same for the y-face (i, j+1/2), Eq. (3.4).
void yface(const State& S, int i, int j, double dt, double* Gs, double* Ws) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  double gs[3], gw[3];
  gauss3(gs, gw);
  for (int q = 0; q < nc; ++q) Gs[q] = Ws[q] = 0.0;
  for (int g = 0; g < 3; ++g) {
    double line[4][2][4][5];
    for (int c = 0; c < 4; ++c) xpass(S, i, j - 1 + c, gs[g], line[c]);
    Deriv a[4], b[4], dB[4], dT[4];
    double Wref[4];
    for (int q = 0; q < nc; ++q) Wref[q] = 0.5 * (fetch(S, 0, q, i, j) + fetch(S, 0, q, i, j + 1));
    second_pass(P, 1, P.dy, line, cell_flag(S, i, j), cell_flag(S, i, j + 1), Wref, a, b);
    to_xy(nc, a, 0, dB); to_xy(nc, b, 0, dT);
    double tc[4][5], G[4], We[4];
    grp_point(P, 1, dB, dT, tc);
    ader_flux(P, 1, tc, dt, G, We);
    for (int q = 0; q < nc; ++q) { Gs[q] += gw[g] * G[q]; Ws[q] += gw[g] * We[q]; }
  }
}
// State at t_{n+1} at the corner (i+1/2, j+1/2): the y-direction traces of rows j (eta = +1/2)
// and j+1 (eta = -1/2) are averaged, then one x-direction generalised Riemann problem is solved
// and evaluated at tau = dt (the paper gives no detail for the corners, end of Section 3.3).
void corner(const State& S, int i, int j, double dt, double* We) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  double line[4][2][4][5];
  for (int c = 0; c < 4; ++c) {
    double lo[2][4][5], hi[2][4][5];
    ypass(S, i - 1 + c, j, 0.5, lo);
    ypass(S, i - 1 + c, j + 1, -0.5, hi);
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < nc; ++q)
        for (int n = 0; n <= ORD; ++n) line[c][s][q][n] = 0.5 * (lo[s][q][n] + hi[s][q][n]);
  }
  int fL = cell_flag(S, i, j) | cell_flag(S, i, j + 1);
  int fR = cell_flag(S, i + 1, j) | cell_flag(S, i + 1, j + 1);
  Deriv a[4], b[4], dL[4], dR[4];
  double Wref[4];
  for (int q = 0; q < nc; ++q)
    Wref[q] = 0.25 * (fetch(S, 0, q, i, j) + fetch(S, 0, q, i + 1, j) + fetch(S, 0, q, i, j + 1) +
                      fetch(S, 0, q, i + 1, j + 1));
  second_pass(P, 0, P.dx, line, fL, fR, Wref, a, b);
  to_xy(nc, a, 1, dL); to_xy(nc, b, 1, dR);
  double tc[4][5];
  grp_point(P, 0, dL, dR, tc);
  taylor_state(nc, tc, dt, We);
}

// Step 5 for one cell from its four faces and four corners: Eq. (3.2) and Eq. (3.10).
void update_cell(const State& S, int i, int j, double dt, const double Fx[2][4], const double Wx[2][4],
                 const double Gy[2][4], const double Wy[2][4], const double Wc[2][2][4],
                 double* Wn, double* Vn, double* Yn, double* Zn) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  for (int q = 0; q < nc; ++q) {
    size_t o = ((size_t)q * P.ny + j) * P.nx + i;
    Wn[q] = S.f[0][o] - dt / P.dx * (Fx[1][q] - Fx[0][q]) - dt / P.dy * (Gy[1][q] - Gy[0][q]);
    Vn[q] = (Wx[1][q] - Wx[0][q]) / P.dx;
    Yn[q] = (Wy[1][q] - Wy[0][q]) / P.dy;
    Zn[q] = (Wc[1][1][q] - Wc[1][0][q] - Wc[0][1][q] + Wc[0][0][q]) / (P.dx * P.dy);
  }
}

void step2d(const Problem& P, const State& S, double dt, double* Wn, double* Vn, double* Yn,
            double* Zn) {
  const int nc = ncomp(P), nx = P.nx, ny = P.ny;
  // every face and corner once, then the cell updates
  std::vector<double> FX((size_t)(nx + 1) * ny * nc), WX((size_t)(nx + 1) * ny * nc);
  std::vector<double> GY((size_t)nx * (ny + 1) * nc), WY((size_t)nx * (ny + 1) * nc);
  std::vector<double> WC((size_t)(nx + 1) * (ny + 1) * nc);
  for (int j = 0; j < ny; ++j)
    for (int i = -1; i < nx; ++i) {
      size_t o = ((size_t)j * (nx + 1) + (i + 1)) * nc;
      xface(S, i, j, dt, &FX[o], &WX[o]);
    }
  for (int j = -1; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t o = ((size_t)(j + 1) * nx + i) * nc;
      yface(S, i, j, dt, &GY[o], &WY[o]);
    }
  for (int j = -1; j < ny; ++j)
    for (int i = -1; i < nx; ++i) corner(S, i, j, dt, &WC[((size_t)(j + 1) * (nx + 1) + (i + 1)) * nc]);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double Fx[2][4], Wx[2][4], Gy[2][4], Wy[2][4], Wc[2][2][4], w[4], v[4], y[4], z[4];
      for (int q = 0; q < nc; ++q) {
        for (int s = 0; s < 2; ++s) {
          size_t ox = ((size_t)j * (nx + 1) + (i + s)) * nc + q;
          size_t oy = ((size_t)(j + s) * nx + i) * nc + q;
          Fx[s][q] = FX[ox]; Wx[s][q] = WX[ox]; Gy[s][q] = GY[oy]; Wy[s][q] = WY[oy];
          for (int r = 0; r < 2; ++r) Wc[r][s][q] = WC[((size_t)(j + r) * (nx + 1) + (i + s)) * nc + q];
        }
      }
      update_cell(S, i, j, dt, Fx, Wx, Gy, Wy, Wc, w, v, y, z);
      for (int q = 0; q < nc; ++q) {
        size_t o = ((size_t)q * ny + j) * nx + i;
        Wn[o] = w[q]; Vn[o] = v[q]; Yn[o] = y[q]; Zn[o] = z[q];
      }
    }
}

// The same step for the cells of a window [i0, i0+w) x [j0, j0+h) of the mesh (faces and
// corners inside the window computed once); outputs are [field][comp][h][w].
void step2d_window(const State& S, double dt, int i0, int j0, int w, int h, double* out) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  std::vector<double> FX((size_t)(w + 1) * h * nc), WX((size_t)(w + 1) * h * nc);
  std::vector<double> GY((size_t)w * (h + 1) * nc), WY((size_t)w * (h + 1) * nc);
  std::vector<double> WC((size_t)(w + 1) * (h + 1) * nc);
  for (int b = 0; b < h; ++b)
    for (int a = 0; a <= w; ++a) {
      size_t o = ((size_t)b * (w + 1) + a) * nc;
      xface(S, i0 + a - 1, j0 + b, dt, &FX[o], &WX[o]);
    }
  for (int b = 0; b <= h; ++b)
    for (int a = 0; a < w; ++a) {
      size_t o = ((size_t)b * w + a) * nc;
      yface(S, i0 + a, j0 + b - 1, dt, &GY[o], &WY[o]);
    }
  for (int b = 0; b <= h; ++b)
    for (int a = 0; a <= w; ++a) corner(S, i0 + a - 1, j0 + b - 1, dt, &WC[((size_t)b * (w + 1) + a) * nc]);
  const size_t plane = (size_t)nc * w * h;
  for (int b = 0; b < h; ++b)
    for (int a = 0; a < w; ++a) {
      double Fx[2][4], Wx[2][4], Gy[2][4], Wy[2][4], Wc[2][2][4], r[4][4];
      for (int q = 0; q < nc; ++q)
        for (int s2 = 0; s2 < 2; ++s2) {
          size_t ox = ((size_t)b * (w + 1) + (a + s2)) * nc + q;
          size_t oy = ((size_t)(b + s2) * w + a) * nc + q;
          Fx[s2][q] = FX[ox]; Wx[s2][q] = WX[ox]; Gy[s2][q] = GY[oy]; Wy[s2][q] = WY[oy];
          for (int r2 = 0; r2 < 2; ++r2) Wc[r2][s2][q] = WC[((size_t)(b + r2) * (w + 1) + (a + s2)) * nc + q];
        }
      update_cell(S, i0 + a, j0 + b, dt, Fx, Wx, Gy, Wy, Wc, r[0], r[1], r[2], r[3]);
      for (int f = 0; f < 4; ++f)
        for (int q = 0; q < nc; ++q) out[f * plane + ((size_t)q * h + b) * w + a] = r[f][q];
    }
}

// The same step for a list of cells only (each cell's own faces and corners): the updated
// W, V, Y, Z of cell k go to out[k*4*nc + field*nc + q].
void step2d_cells(const State& S, double dt, int ncells, const int32_t* ij, double* out) {
  const Problem& P = *S.P;
  const int nc = ncomp(P);
  for (int k = 0; k < ncells; ++k) {
    const int i = ij[2 * k], j = ij[2 * k + 1];
    double Fx[2][4], Wx[2][4], Gy[2][4], Wy[2][4], Wc[2][2][4];
    for (int s = 0; s < 2; ++s) {
      xface(S, i - 1 + s, j, dt, Fx[s], Wx[s]);
      yface(S, i, j - 1 + s, dt, Gy[s], Wy[s]);
      for (int r = 0; r < 2; ++r) corner(S, i - 1 + s, j - 1 + r, dt, Wc[r][s]);
    }
    double* o = out + (size_t)k * 4 * nc;
    update_cell(S, i, j, dt, Fx, Wx, Gy, Wy, Wc, o, o + nc, o + 2 * nc, o + 3 * nc);
  }
}

// ----------------------------------------------------------------------------------------
// Time step size from the CFL condition (Section 5 uses a fixed CFL number; the formula is
// the usual maximum characteristic speed over the cell averages).
// ----------------------------------------------------------------------------------------
double max_rate(const Problem& P, const double* W) {
  const size_t n = (size_t)P.nx * (P.dim == 2 ? P.ny : 1);
  const double g = P.gamma;
  double best = 0.0;
  for (size_t c = 0; c < n; ++c) {
    double r;
    if (P.eq == EQ_BURGERS) {
      double u = std::fabs(W[c]);
      r = P.dim == 1 ? u / P.dx : u / P.dx + u / P.dy;
    } else if (P.dim == 1) {
      double rho = W[c], u = W[n + c] / rho, E = W[2 * n + c];
      double p = (g - 1.0) * (E - 0.5 * rho * u * u);
      r = (std::fabs(u) + std::sqrt(g * p / rho)) / P.dx;
    } else {
      double rho = W[c], u = W[n + c] / rho, v = W[2 * n + c] / rho, E = W[3 * n + c];
      double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
      double cs = std::sqrt(g * p / rho);
      r = (std::fabs(u) + cs) / P.dx + (std::fabs(v) + cs) / P.dy;
    }
    if (std::isnan(r)) return r;  // a non-physical state poisons the step size
    if (r > best) best = r;
  }
  return best;
}

}  // namespace

// ========================================================================================
// C interface for the Python test harness (ctypes).
// ========================================================================================
extern "C" {

typedef Problem orc_problem;

// Section 2.4 reading: p1 coefficients, smoothness indicators, weights, combined polynomial.
// v = (h V_{-1}, h V_{+1}) for the quartic (reading R1); the *_deg forms take
// v = (h V_{-1}, h V_0, h V_{+1}) and quintic = 1 for reading R1'.  Coefficients c[0..5].
void orc_big_poly(const double* Wb, const double* v, double* c) {
  const double v3[3] = {v[0], 0.0, v[1]};
  double c6[6];
  big_poly(Wb, v3, 0, c6);
  for (int k = 0; k < 5; ++k) c[k] = c6[k];
}
void orc_big_poly_deg(const double* Wb, const double* v, int quintic, double* c) {
  big_poly(Wb, v, quintic, c);
}
double orc_smoothness(const double* c) {
  const double c6[6] = {c[0], c[1], c[2], c[3], c[4], 0.0};
  return smoothness(c6);
}
double orc_smoothness_deg(const double* c) { return smoothness(c); }
void orc_weights(const double* Wb, const double* v, int linear, double eps, const double* gam,
                 double* w) {
  const double v3[3] = {v[0], 0.0, v[1]};
  shweno_weights(Wb, v3, 0, linear, eps, gam, w);
}
void orc_recon(const double* Wb, const double* v, int linear, double eps, const double* gam,
               double xi, double* d) {
  const double v3[3] = {v[0], 0.0, v[1]};
  double w[3], c[6];
  shweno_weights(Wb, v3, 0, linear, eps, gam, w);
  shweno_poly(Wb, v3, 0, w, gam, c);
  poly_derivs(c, xi, d);
}
void orc_recon_deg(const double* Wb, const double* v, int quintic, int linear, double eps,
                   const double* gam, double xi, double* d) {
  double w[3], c[6];
  shweno_weights(Wb, v, quintic, linear, eps, gam, w);
  shweno_poly(Wb, v, quintic, w, gam, c);
  poly_derivs(c, xi, d);
}
void orc_quadrature(double* lob_nodes, double* lob_w, double* gauss_nodes, double* gauss_w) {
  lobatto4(lob_nodes, lob_w);
  gauss3(gauss_nodes, gauss_w);
}
double orc_burgers_godunov(double uL, double uR) { return burgers_godunov(uL, uR); }
void orc_hllc(const orc_problem* P, int dir, const double* WL, const double* WR, double* out) {
  hllc_state(*P, dir, WL, WR, out);
}
void orc_eigen(const orc_problem* P, int dir, const double* W, double* lam, double* R, double* L) {
  eigensystem(*P, dir, W, lam, R);
  invert(ncomp(*P), R, L);
}
void orc_upwind(const orc_problem* P, int dir, const double* Ws, const double* dL,
                const double* dR, double* out) {
  double lam[4], R[16], L[16];
  eigensystem(*P, dir, Ws, lam, R);
  invert(ncomp(*P), R, L);
  upwind(ncomp(*P), lam, wave_scale(*P, Ws, Ws[0], Ws[0]), R, L, dL, dR, out);
}
// CK on given spatial derivatives d[q][m][n] (= d^{m+n}W_q/dx^m dy^n, a 5x5 block per
// component); returns all mixed derivatives out[q][m][n][k] = d^{m+n+k} W_q/dx^m dy^n dt^k.
void orc_ck(const orc_problem* P, const double* d, double* out) {
  const int nc = ncomp(*P);
  Ser S[4];
  for (int q = 0; q < nc; ++q) {
    ser_zero(S[q]);
    for (int m = 0; m <= ORD; ++m)
      for (int n = 0; m + n <= ORD; ++n)
        S[q].c[m][n][0] = d[(q * 5 + m) * 5 + n] / (factorial(m) * factorial(n));
  }
  cauchy_kovalevskaya(*P, S);
  for (int q = 0; q < nc; ++q)
    for (int m = 0; m <= ORD; ++m)
      for (int n = 0; n <= ORD; ++n)
        for (int k = 0; k <= ORD; ++k)
          out[((q * 5 + m) * 5 + n) * 5 + k] =
              in_range(m, n, k) ? S[q].c[m][n][k] * factorial(m) * factorial(n) * factorial(k) : 0.0;
}
// Steps 3-4 at one point: one-sided derivatives dL, dR as [q][m][n]; returns the time-Taylor
// coefficients tc[q][k] = d^k W*/dt^k / k!.
void orc_grp_point(const orc_problem* P, int dir, const double* dL, const double* dR, double* tc) {
  Deriv a[4], b[4];
  std::memcpy(a, dL, sizeof(Deriv) * ncomp(*P));
  std::memcpy(b, dR, sizeof(Deriv) * ncomp(*P));
  double t[4][5];
  grp_point(*P, dir, a, b, t);
  for (int q = 0; q < ncomp(*P); ++q)
    for (int k = 0; k < 5; ++k) tc[q * 5 + k] = t[q][k];
}
double orc_max_rate(const orc_problem* P, const double* W) { return max_rate(*P, W); }

// One step of size dt from time t.  Arrays are [comp][ny][nx] (1D: [comp][nx]); Y, Z and their
// outputs are ignored in 1D.  flag: per-cell byte (nonzero = nonlinear weights) or null.
void orc_step(const orc_problem* P, const double* W, const double* V, const double* Y,
              const double* Z, const uint8_t* flag, double t, double dt, double* Wn, double* Vn,
              double* Yn, double* Zn) {
  State S{P, {W, V, Y, Z}, flag, t};
  if (P->dim == 1) step1d(*P, S, dt, Wn, Vn);
  else step2d(*P, S, dt, Wn, Vn, Yn, Zn);
}

// One 2D step restricted to the listed cells (ij = i0, j0, i1, j1, ...); out[k][field][q].
void orc_step2d_cells(const orc_problem* P, const double* W, const double* V, const double* Y,
                      const double* Z, const uint8_t* flag, double t, double dt, int ncells,
                      const int32_t* ij, double* out) {
  State S{P, {W, V, Y, Z}, flag, t};
  step2d_cells(S, dt, ncells, ij, out);
}

// ----- learned troubled-cell flag (not in the paper; the learned layer of the library) -----
// Label source: the largest relative deviation max_l |w_l - gamma_l| / gamma_l of the nonlinear
// weights of the 16 first-pass reconstructions anchored on cell (i, j) (y-pass on {W,Y} and
// {V,Z}, x-pass on {W,V} and {Y,Z}, four components) in the always-nonlinear scheme.
void orc_weight_deviation2d(const orc_problem* P, const double* W, const double* V, const double* Y,
                            const double* Z, double t, double* out) {
  State S{P, {W, V, Y, Z}, nullptr, t};
  const int nc = ncomp(*P);
  for (int j = 0; j < P->ny; ++j)
    for (int i = 0; i < P->nx; ++i) {
      double dev = 0.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int set = 0; set < 2; ++set)
          for (int q = 0; q < nc; ++q) {
            // pass 0: along y, sets {W,Y}, {V,Z}; pass 1: along x, sets {W,V}, {Y,Z}
            int fa = pass == 0 ? (set == 0 ? 0 : 1) : (set == 0 ? 0 : 2);
            int fd = pass == 0 ? (set == 0 ? 2 : 3) : (set == 0 ? 1 : 3);
            int di = pass == 1, dj = pass == 0;
            double h = pass == 0 ? P->dy : P->dx;
            double Wb[3] = {fetch(S, fa, q, i - di, j - dj), fetch(S, fa, q, i, j),
                            fetch(S, fa, q, i + di, j + dj)};
            double v[3] = {h * fetch(S, fd, q, i - di, j - dj), h * fetch(S, fd, q, i, j),
                           h * fetch(S, fd, q, i + di, j + dj)};
            double w[3];
            shweno_weights(Wb, v, P->quintic, 0, P->eps, P->gam, w);
            for (int l = 0; l < 3; ++l) dev = std::fmax(dev, std::fabs(w[l] - P->gam[l]) / P->gam[l]);
          }
      out[(size_t)j * P->nx + i] = dev;
    }
}

// Label source of the face-value form: the largest change the nonlinear weights make to the end
// values of the 16 first-pass reconstructions anchored on cell (i, j), relative to the range of
// the reconstruction's three cell averages:
//   max over reconstructions and xi = -1/2, +1/2 of |p(xi) - p1(xi)| / (max Wb - min Wb + f |W0| + 1e-300),
// where p is the SHWENO polynomial with the nonlinear weights and p1 the big-stencil polynomial
// (the reconstruction with the linear weights), both of reading R1, and f >= 1e-9 the caller's
// floor of the scale relative to the cell's own average (1e-9 keeps rounding, a few ulp of |W0|
// in p - p1 on constant data, near 1e-7; a larger f discounts changes small against |W0|).
double face_deviation(const double Wb[3], const double v[3], int quintic, double eps, const double gam[3],
                      double floor_rel) {
  double w[3], c[6], c1[6];
  shweno_weights(Wb, v, quintic, 0, eps, gam, w);
  shweno_poly(Wb, v, quintic, w, gam, c);
  big_poly(Wb, v, quintic, c1);
  const double mx = std::fmax(Wb[0], std::fmax(Wb[1], Wb[2])), mn = std::fmin(Wb[0], std::fmin(Wb[1], Wb[2]));
  const double scale = mx - mn + floor_rel * std::fabs(Wb[1]) + 1e-300;
  double dev = 0.0;
  for (double xi : {-0.5, 0.5}) {
    double d[5], d1[5];
    poly_derivs(c, xi, d);
    poly_derivs(c1, xi, d1);
    dev = std::fmax(dev, std::fabs(d[0] - d1[0]) / scale);
  }
  return dev;
}
void orc_face_deviation2d(const orc_problem* P, const double* W, const double* V, const double* Y,
                          const double* Z, double t, double floor_rel, double* out) {
  State S{P, {W, V, Y, Z}, nullptr, t};
  const int nc = ncomp(*P);
  for (int j = 0; j < P->ny; ++j)
    for (int i = 0; i < P->nx; ++i) {
      double dev = 0.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int set = 0; set < 2; ++set)
          for (int q = 0; q < nc; ++q) {
            // pass 0: along y, sets {W,Y}, {V,Z}; pass 1: along x, sets {W,V}, {Y,Z}
            int fa = pass == 0 ? (set == 0 ? 0 : 1) : (set == 0 ? 0 : 2);
            int fd = pass == 0 ? (set == 0 ? 2 : 3) : (set == 0 ? 1 : 3);
            int di = pass == 1, dj = pass == 0;
            double h = pass == 0 ? P->dy : P->dx;
            double Wb[3] = {fetch(S, fa, q, i - di, j - dj), fetch(S, fa, q, i, j),
                            fetch(S, fa, q, i + di, j + dj)};
            double v[3] = {h * fetch(S, fd, q, i - di, j - dj), h * fetch(S, fd, q, i, j),
                           h * fetch(S, fd, q, i + di, j + dj)};
            dev = std::fmax(dev, face_deviation(Wb, v, 0, P->eps, P->gam, floor_rel));  // reading R1's polynomials
          }
      out[(size_t)j * P->nx + i] = dev;
    }
}
double orc_face_deviation(const double* Wb, const double* v, double eps, const double* gam, double floor_rel) {
  const double v3[3] = {v[0], 0.0, v[1]};
  return face_deviation(Wb, v3, 0, eps, gam, floor_rel);
}

// Features of cell (i, j), 11 per variable for rho (component 0) and E (last component):
// the eight 3x3-stencil neighbours minus the centre and dx V, dy Y of the centre, all divided by
// s = (max - min over the stencil) + 1e-12 |centre| + 1e-300; then log10(range/(|centre| +
// 1e-30) + 1e-16) / 8.  Neighbour order: (-1,-1), (0,-1), (1,-1), (-1,0), (1,0), (-1,1), (0,1),
// (1,1) as (di, dj).  out[cell][22].
void orc_features2d(const orc_problem* P, const double* W, const double* V, const double* Y,
                    const double* Z, double t, double* out) {
  State S{P, {W, V, Y, Z}, nullptr, t};
  const int nc = ncomp(*P);
  const int comps[2] = {0, nc - 1};
  for (int j = 0; j < P->ny; ++j)
    for (int i = 0; i < P->nx; ++i) {
      double* f = out + ((size_t)j * P->nx + i) * 22;
      for (int a = 0; a < 2; ++a) {
        const int q = comps[a];
        double vals[3][3];
        double mn = 1e300, mx = -1e300;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            double x = fetch(S, 0, q, i + di, j + dj);
            vals[dj + 1][di + 1] = x;
            mn = std::fmin(mn, x);
            mx = std::fmax(mx, x);
          }
        const double c = vals[1][1];
        const double range = mx - mn;
        const double sc = range + 1e-12 * std::fabs(c) + 1e-300;
        int k = 0;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di)
            if (di != 0 || dj != 0) f[a * 11 + k++] = (vals[dj + 1][di + 1] - c) / sc;
        f[a * 11 + 8] = P->dx * fetch(S, 1, q, i, j) / sc;
        f[a * 11 + 9] = P->dy * fetch(S, 2, q, i, j) / sc;
        f[a * 11 + 10] = std::log10(range / (std::fabs(c) + 1e-30) + 1e-16) / 8.0;
      }
    }
}

// One 2D step restricted to a window of cells; out[field][comp][h][w].
void orc_step2d_window(const orc_problem* P, const double* W, const double* V, const double* Y,
                       const double* Z, const uint8_t* flag, double t, double dt, int i0, int j0,
                       int w, int h, double* out) {
  State S{P, {W, V, Y, Z}, flag, t};
  step2d_window(S, dt, i0, j0, w, h, out);
}

// Runs to t_final with dt = cfl / max_rate, the last step shortened to land on t_final.
// State arrays are updated in place.  Returns the number of steps; max_steps bounds the loop
// (a negative return means it was hit).  A step that leaves the physical range in some cell
// (Euler: rho <= 0, p <= 0 or a non-finite value; Burgers: a non-finite value) is not kept:
// the run stops at the state before it and *nonphysical is set to 1 (0 otherwise).
int64_t orc_run(const orc_problem* P, double* W, double* V, double* Y, double* Z,
                const uint8_t* flag, double t_final, double cfl, int64_t max_steps, double* t_out,
                int32_t* nonphysical) {
  const size_t n = (size_t)ncomp(*P) * P->nx * (P->dim == 2 ? P->ny : 1);
  const size_t cells = (size_t)P->nx * (P->dim == 2 ? P->ny : 1);
  std::vector<double> a(n), b(n), c(n), d(n);
  double t = 0.0;
  int64_t steps = 0;
  *nonphysical = 0;
  while (t < t_final) {
    if (steps >= max_steps) { *t_out = t; return -steps; }
    double dt = cfl / max_rate(*P, W);
    if (dt > t_final - t) dt = t_final - t;
    orc_step(P, W, V, Y, Z, flag, t, dt, a.data(), b.data(), c.data(), d.data());
    for (size_t k = 0; k < cells; ++k) {
      bool ok;
      if (P->eq == EQ_BURGERS) {
        ok = std::isfinite(a[k]);
      } else {
        const int nc = ncomp(*P);
        const double rho = a[k];
        double m2 = 0.0;
        for (int q = 1; q < nc - 1; ++q) m2 += a[q * cells + k] * a[q * cells + k];
        const double p = (P->gamma - 1.0) * (a[(nc - 1) * cells + k] - 0.5 * m2 / rho);
        ok = rho > 0.0 && p > 0.0 && std::isfinite(rho) && std::isfinite(p);
      }
      if (!ok) {
        *nonphysical = 1;
        *t_out = t;
        return steps;
      }
    }
    std::memcpy(W, a.data(), n * sizeof(double));
    std::memcpy(V, b.data(), n * sizeof(double));
    if (P->dim == 2) {
      std::memcpy(Y, c.data(), n * sizeof(double));
      std::memcpy(Z, d.data(), n * sizeof(double));
    }
    t += dt;
    ++steps;
  }
  *t_out = t;
  return steps;
}

}  // extern "C"
