// Generated by gen_tables.py -- exact rational constants of the SHWENO reconstruction.
// Do not edit by hand.
#pragma once
namespace shweno_tables {
// p1 monomial coefficients: c_k = sum of COEF_k_<v> * v over v in {W0, s, dv, a, sv}.
constexpr double P1_C0_W0 = (287.0 / 240.0);
constexpr double P1_C0_s = (-47.0 / 480.0);
constexpr double P1_C0_dv = (9.0 / 320.0);
constexpr double P1_C0_a = 0.0;
constexpr double P1_C0_sv = 0.0;
constexpr double P1_C1_W0 = 0.0;
constexpr double P1_C1_s = 0.0;
constexpr double P1_C1_dv = 0.0;
constexpr double P1_C1_a = (13.0 / 16.0);
constexpr double P1_C1_sv = (-5.0 / 16.0);
constexpr double P1_C2_W0 = (-5.0 / 2.0);
constexpr double P1_C2_s = (5.0 / 4.0);
constexpr double P1_C2_dv = (-3.0 / 8.0);
constexpr double P1_C2_a = 0.0;
constexpr double P1_C2_sv = 0.0;
constexpr double P1_C3_W0 = 0.0;
constexpr double P1_C3_s = 0.0;
constexpr double P1_C3_dv = 0.0;
constexpr double P1_C3_a = (-1.0 / 4.0);
constexpr double P1_C3_sv = (1.0 / 4.0);
constexpr double P1_C4_W0 = 1.0;
constexpr double P1_C4_s = (-1.0 / 2.0);
constexpr double P1_C4_dv = (1.0 / 4.0);
constexpr double P1_C4_a = 0.0;
constexpr double P1_C4_sv = 0.0;
// Taylor coefficient m (d^m p1/dxi^m / m!) at xi = +1/2 (P) and -1/2 (M):
// END_<P|M>[m][v] over the data v = (W-, W0, W+, v-, v+)
constexpr double END_P_0_0 = (-23.0 / 120.0);
constexpr double END_P_0_1 = (19.0 / 30.0);
constexpr double END_P_0_2 = (67.0 / 120.0);
constexpr double END_P_0_3 = (-3.0 / 40.0);
constexpr double END_P_0_4 = (-7.0 / 40.0);
constexpr double END_P_1_0 = (3.0 / 8.0);
constexpr double END_P_1_1 = -2.0;
constexpr double END_P_1_2 = (13.0 / 8.0);
constexpr double END_P_1_3 = (1.0 / 8.0);
constexpr double END_P_1_4 = (-3.0 / 8.0);
constexpr double END_P_2_0 = (7.0 / 8.0);
constexpr double END_P_2_1 = -1.0;
constexpr double END_P_2_2 = (1.0 / 8.0);
constexpr double END_P_2_3 = (3.0 / 8.0);
constexpr double END_P_2_4 = (3.0 / 8.0);
constexpr double END_P_3_0 = (-3.0 / 4.0);
constexpr double END_P_3_1 = 2.0;
constexpr double END_P_3_2 = (-5.0 / 4.0);
constexpr double END_P_3_3 = (-1.0 / 4.0);
constexpr double END_P_3_4 = (3.0 / 4.0);
constexpr double END_P_4_0 = (-1.0 / 2.0);
constexpr double END_P_4_1 = 1.0;
constexpr double END_P_4_2 = (-1.0 / 2.0);
constexpr double END_P_4_3 = (-1.0 / 4.0);
constexpr double END_P_4_4 = (1.0 / 4.0);
constexpr double END_M_0_0 = (67.0 / 120.0);
constexpr double END_M_0_1 = (19.0 / 30.0);
constexpr double END_M_0_2 = (-23.0 / 120.0);
constexpr double END_M_0_3 = (7.0 / 40.0);
constexpr double END_M_0_4 = (3.0 / 40.0);
constexpr double END_M_1_0 = (-13.0 / 8.0);
constexpr double END_M_1_1 = 2.0;
constexpr double END_M_1_2 = (-3.0 / 8.0);
constexpr double END_M_1_3 = (-3.0 / 8.0);
constexpr double END_M_1_4 = (1.0 / 8.0);
constexpr double END_M_2_0 = (1.0 / 8.0);
constexpr double END_M_2_1 = -1.0;
constexpr double END_M_2_2 = (7.0 / 8.0);
constexpr double END_M_2_3 = (-3.0 / 8.0);
constexpr double END_M_2_4 = (-3.0 / 8.0);
constexpr double END_M_3_0 = (5.0 / 4.0);
constexpr double END_M_3_1 = -2.0;
constexpr double END_M_3_2 = (3.0 / 4.0);
constexpr double END_M_3_3 = (3.0 / 4.0);
constexpr double END_M_3_4 = (-1.0 / 4.0);
constexpr double END_M_4_0 = (-1.0 / 2.0);
constexpr double END_M_4_1 = 1.0;
constexpr double END_M_4_2 = (-1.0 / 2.0);
constexpr double END_M_4_3 = (-1.0 / 4.0);
constexpr double END_M_4_4 = (1.0 / 4.0);
// dot product of row p of END_P (plus) or END_M with the data d[0..4]
template <bool PLUS>
__host__ __device__ __forceinline__ double end_dot(int p, const double d[5]) {
  switch (p) {
    case 0: return PLUS ? (END_P_0_0 * d[0] + END_P_0_1 * d[1] + END_P_0_2 * d[2] + END_P_0_3 * d[3] + END_P_0_4 * d[4]) : (END_M_0_0 * d[0] + END_M_0_1 * d[1] + END_M_0_2 * d[2] + END_M_0_3 * d[3] + END_M_0_4 * d[4]);
    case 1: return PLUS ? (END_P_1_0 * d[0] + END_P_1_1 * d[1] + END_P_1_2 * d[2] + END_P_1_3 * d[3] + END_P_1_4 * d[4]) : (END_M_1_0 * d[0] + END_M_1_1 * d[1] + END_M_1_2 * d[2] + END_M_1_3 * d[3] + END_M_1_4 * d[4]);
    case 2: return PLUS ? (END_P_2_0 * d[0] + END_P_2_1 * d[1] + END_P_2_2 * d[2] + END_P_2_3 * d[3] + END_P_2_4 * d[4]) : (END_M_2_0 * d[0] + END_M_2_1 * d[1] + END_M_2_2 * d[2] + END_M_2_3 * d[3] + END_M_2_4 * d[4]);
    case 3: return PLUS ? (END_P_3_0 * d[0] + END_P_3_1 * d[1] + END_P_3_2 * d[2] + END_P_3_3 * d[3] + END_P_3_4 * d[4]) : (END_M_3_0 * d[0] + END_M_3_1 * d[1] + END_M_3_2 * d[2] + END_M_3_3 * d[3] + END_M_3_4 * d[4]);
    case 4: return PLUS ? (END_P_4_0 * d[0] + END_P_4_1 * d[1] + END_P_4_2 * d[2] + END_P_4_3 * d[3] + END_P_4_4 * d[4]) : (END_M_4_0 * d[0] + END_M_4_1 * d[1] + END_M_4_2 * d[2] + END_M_4_3 * d[3] + END_M_4_4 * d[4]);
  }
  return 0.0;
}
// Even/odd parts of the end values: e_m(+1/2) = U_m + V_m, e_m(-1/2) = (-1)^m (U_m - V_m),
// U_m = ENDU_m_W0 W0 + ENDU_m_s s + ENDU_m_dv dv, V_m = ENDV_m_a a + ENDV_m_sv sv
// (R1'; QENDV_m_a a + QENDV_m_sv sv + QENDV_m_v0 v0; U_m is the same).
constexpr double ENDU_0_W0 = (19.0 / 30.0);
constexpr double ENDU_0_s = (11.0 / 60.0);
constexpr double ENDU_0_dv = (-1.0 / 20.0);
constexpr double ENDV_0_a = (3.0 / 8.0);
constexpr double ENDV_0_sv = (-1.0 / 8.0);
constexpr double ENDU_1_W0 = -2.0;
constexpr double ENDU_1_s = 1.0;
constexpr double ENDU_1_dv = (-1.0 / 4.0);
constexpr double ENDV_1_a = (5.0 / 8.0);
constexpr double ENDV_1_sv = (-1.0 / 8.0);
constexpr double ENDU_2_W0 = -1.0;
constexpr double ENDU_2_s = (1.0 / 2.0);
constexpr double ENDU_2_dv = 0.0;
constexpr double ENDV_2_a = (-3.0 / 8.0);
constexpr double ENDV_2_sv = (3.0 / 8.0);
constexpr double ENDU_3_W0 = 2.0;
constexpr double ENDU_3_s = -1.0;
constexpr double ENDU_3_dv = (1.0 / 2.0);
constexpr double ENDV_3_a = (-1.0 / 4.0);
constexpr double ENDV_3_sv = (1.0 / 4.0);
constexpr double ENDU_4_W0 = 1.0;
constexpr double ENDU_4_s = (-1.0 / 2.0);
constexpr double ENDU_4_dv = (1.0 / 4.0);
constexpr double ENDV_4_a = 0.0;
constexpr double ENDV_4_sv = 0.0;
constexpr double QENDV_0_a = 0.0;
constexpr double QENDV_0_sv = 0.0;
constexpr double QENDV_0_v0 = (1.0 / 2.0);
constexpr double QENDV_1_a = (3.0 / 4.0);
constexpr double QENDV_1_sv = (-1.0 / 6.0);
constexpr double QENDV_1_v0 = (-1.0 / 6.0);
constexpr double QENDV_2_a = (15.0 / 8.0);
constexpr double QENDV_2_sv = (-3.0 / 8.0);
constexpr double QENDV_2_v0 = -3.0;
constexpr double QENDV_3_a = 0.0;
constexpr double QENDV_3_sv = (1.0 / 6.0);
constexpr double QENDV_3_v0 = (-1.0 / 3.0);
constexpr double QENDV_4_a = (-15.0 / 8.0);
constexpr double QENDV_4_sv = (5.0 / 8.0);
constexpr double QENDV_4_v0 = (5.0 / 2.0);
// U_m(W0, s, dv) and V_m(a, sv) (R1) or V_m(a, sv, v0) (R1') of the end values
__host__ __device__ __forceinline__ double end_u(int m, double W0, double s, double dv) {
  switch (m) {
    case 0: return ENDU_0_W0 * W0 + ENDU_0_s * s + ENDU_0_dv * dv;
    case 1: return ENDU_1_W0 * W0 + ENDU_1_s * s + ENDU_1_dv * dv;
    case 2: return ENDU_2_W0 * W0 + ENDU_2_s * s;
    case 3: return ENDU_3_W0 * W0 + ENDU_3_s * s + ENDU_3_dv * dv;
    case 4: return ENDU_4_W0 * W0 + ENDU_4_s * s + ENDU_4_dv * dv;
  }
  return 0.0;
}
__host__ __device__ __forceinline__ double end_v(int m, double a, double sv) {
  switch (m) {
    case 0: return ENDV_0_a * a + ENDV_0_sv * sv;
    case 1: return ENDV_1_a * a + ENDV_1_sv * sv;
    case 2: return ENDV_2_a * a + ENDV_2_sv * sv;
    case 3: return ENDV_3_a * a + ENDV_3_sv * sv;
    case 4: return 0.0;
  }
  return 0.0;
}
__host__ __device__ __forceinline__ double qend_v(int m, double a, double sv, double v0) {
  switch (m) {
    case 0: return QENDV_0_v0 * v0;
    case 1: return QENDV_1_a * a + QENDV_1_sv * sv + QENDV_1_v0 * v0;
    case 2: return QENDV_2_a * a + QENDV_2_sv * sv + QENDV_2_v0 * v0;
    case 3: return QENDV_3_sv * sv + QENDV_3_v0 * v0;
    case 4: return QENDV_4_a * a + QENDV_4_sv * sv + QENDV_4_v0 * v0;
  }
  return 0.0;
}
// smoothness indicator of p1: beta1 = sum_{i<=j} B_ij c_i c_j (i, j >= 1)
constexpr double BETA_11 = 1.0;
constexpr double BETA_12 = 0.0;
constexpr double BETA_13 = (1.0 / 2.0);
constexpr double BETA_14 = 0.0;
constexpr double BETA_22 = (13.0 / 3.0);
constexpr double BETA_23 = 0.0;
constexpr double BETA_24 = (21.0 / 5.0);
constexpr double BETA_33 = (3129.0 / 80.0);
constexpr double BETA_34 = 0.0;
constexpr double BETA_44 = (87617.0 / 140.0);
// Reading R1' (quintic p1, data (W-, W0, W+, v-, v0, v+)): odd monomial coefficients
// c_k = QP1_C<k>_a a + QP1_C<k>_sv sv + QP1_C<k>_v0 v0 (k = 1, 3, 5); even ones as R1.
constexpr double QP1_C1_a = (-27.0 / 64.0);
constexpr double QP1_C1_sv = (19.0 / 192.0);
constexpr double QP1_C1_v0 = (79.0 / 48.0);
constexpr double QP1_C3_a = (15.0 / 8.0);
constexpr double QP1_C3_sv = (-11.0 / 24.0);
constexpr double QP1_C3_v0 = (-17.0 / 6.0);
constexpr double QP1_C5_a = (-3.0 / 4.0);
constexpr double QP1_C5_sv = (1.0 / 4.0);
constexpr double QP1_C5_v0 = 1.0;
// R1' Taylor coefficients at the ends over (W-, W0, W+, v-, v0, v+)
constexpr double QEND_P_0_0 = (11.0 / 60.0);
constexpr double QEND_P_0_1 = (19.0 / 30.0);
constexpr double QEND_P_0_2 = (11.0 / 60.0);
constexpr double QEND_P_0_3 = (1.0 / 20.0);
constexpr double QEND_P_0_4 = (1.0 / 2.0);
constexpr double QEND_P_0_5 = (-1.0 / 20.0);
constexpr double QEND_P_1_0 = (1.0 / 4.0);
constexpr double QEND_P_1_1 = -2.0;
constexpr double QEND_P_1_2 = (7.0 / 4.0);
constexpr double QEND_P_1_3 = (1.0 / 12.0);
constexpr double QEND_P_1_4 = (-1.0 / 6.0);
constexpr double QEND_P_1_5 = (-5.0 / 12.0);
constexpr double QEND_P_2_0 = (-11.0 / 8.0);
constexpr double QEND_P_2_1 = -1.0;
constexpr double QEND_P_2_2 = (19.0 / 8.0);
constexpr double QEND_P_2_3 = (-3.0 / 8.0);
constexpr double QEND_P_2_4 = -3.0;
constexpr double QEND_P_2_5 = (-3.0 / 8.0);
constexpr double QEND_P_3_0 = -1.0;
constexpr double QEND_P_3_1 = 2.0;
constexpr double QEND_P_3_2 = -1.0;
constexpr double QEND_P_3_3 = (-1.0 / 3.0);
constexpr double QEND_P_3_4 = (-1.0 / 3.0);
constexpr double QEND_P_3_5 = (2.0 / 3.0);
constexpr double QEND_P_4_0 = (11.0 / 8.0);
constexpr double QEND_P_4_1 = 1.0;
constexpr double QEND_P_4_2 = (-19.0 / 8.0);
constexpr double QEND_P_4_3 = (3.0 / 8.0);
constexpr double QEND_P_4_4 = (5.0 / 2.0);
constexpr double QEND_P_4_5 = (7.0 / 8.0);
constexpr double QEND_M_0_0 = (11.0 / 60.0);
constexpr double QEND_M_0_1 = (19.0 / 30.0);
constexpr double QEND_M_0_2 = (11.0 / 60.0);
constexpr double QEND_M_0_3 = (1.0 / 20.0);
constexpr double QEND_M_0_4 = (-1.0 / 2.0);
constexpr double QEND_M_0_5 = (-1.0 / 20.0);
constexpr double QEND_M_1_0 = (-7.0 / 4.0);
constexpr double QEND_M_1_1 = 2.0;
constexpr double QEND_M_1_2 = (-1.0 / 4.0);
constexpr double QEND_M_1_3 = (-5.0 / 12.0);
constexpr double QEND_M_1_4 = (-1.0 / 6.0);
constexpr double QEND_M_1_5 = (1.0 / 12.0);
constexpr double QEND_M_2_0 = (19.0 / 8.0);
constexpr double QEND_M_2_1 = -1.0;
constexpr double QEND_M_2_2 = (-11.0 / 8.0);
constexpr double QEND_M_2_3 = (3.0 / 8.0);
constexpr double QEND_M_2_4 = 3.0;
constexpr double QEND_M_2_5 = (3.0 / 8.0);
constexpr double QEND_M_3_0 = 1.0;
constexpr double QEND_M_3_1 = -2.0;
constexpr double QEND_M_3_2 = 1.0;
constexpr double QEND_M_3_3 = (2.0 / 3.0);
constexpr double QEND_M_3_4 = (-1.0 / 3.0);
constexpr double QEND_M_3_5 = (-1.0 / 3.0);
constexpr double QEND_M_4_0 = (-19.0 / 8.0);
constexpr double QEND_M_4_1 = 1.0;
constexpr double QEND_M_4_2 = (11.0 / 8.0);
constexpr double QEND_M_4_3 = (-7.0 / 8.0);
constexpr double QEND_M_4_4 = (-5.0 / 2.0);
constexpr double QEND_M_4_5 = (-3.0 / 8.0);
template <bool PLUS>
__host__ __device__ __forceinline__ double qend_dot(int p, const double d[6]) {
  switch (p) {
    case 0: return PLUS ? (QEND_P_0_0 * d[0] + QEND_P_0_1 * d[1] + QEND_P_0_2 * d[2] + QEND_P_0_3 * d[3] + QEND_P_0_4 * d[4] + QEND_P_0_5 * d[5]) : (QEND_M_0_0 * d[0] + QEND_M_0_1 * d[1] + QEND_M_0_2 * d[2] + QEND_M_0_3 * d[3] + QEND_M_0_4 * d[4] + QEND_M_0_5 * d[5]);
    case 1: return PLUS ? (QEND_P_1_0 * d[0] + QEND_P_1_1 * d[1] + QEND_P_1_2 * d[2] + QEND_P_1_3 * d[3] + QEND_P_1_4 * d[4] + QEND_P_1_5 * d[5]) : (QEND_M_1_0 * d[0] + QEND_M_1_1 * d[1] + QEND_M_1_2 * d[2] + QEND_M_1_3 * d[3] + QEND_M_1_4 * d[4] + QEND_M_1_5 * d[5]);
    case 2: return PLUS ? (QEND_P_2_0 * d[0] + QEND_P_2_1 * d[1] + QEND_P_2_2 * d[2] + QEND_P_2_3 * d[3] + QEND_P_2_4 * d[4] + QEND_P_2_5 * d[5]) : (QEND_M_2_0 * d[0] + QEND_M_2_1 * d[1] + QEND_M_2_2 * d[2] + QEND_M_2_3 * d[3] + QEND_M_2_4 * d[4] + QEND_M_2_5 * d[5]);
    case 3: return PLUS ? (QEND_P_3_0 * d[0] + QEND_P_3_1 * d[1] + QEND_P_3_2 * d[2] + QEND_P_3_3 * d[3] + QEND_P_3_4 * d[4] + QEND_P_3_5 * d[5]) : (QEND_M_3_0 * d[0] + QEND_M_3_1 * d[1] + QEND_M_3_2 * d[2] + QEND_M_3_3 * d[3] + QEND_M_3_4 * d[4] + QEND_M_3_5 * d[5]);
    case 4: return PLUS ? (QEND_P_4_0 * d[0] + QEND_P_4_1 * d[1] + QEND_P_4_2 * d[2] + QEND_P_4_3 * d[3] + QEND_P_4_4 * d[4] + QEND_P_4_5 * d[5]) : (QEND_M_4_0 * d[0] + QEND_M_4_1 * d[1] + QEND_M_4_2 * d[2] + QEND_M_4_3 * d[3] + QEND_M_4_4 * d[4] + QEND_M_4_5 * d[5]);
  }
  return 0.0;
}
// R1' smoothness indicator: beta1 = sum_{i<=j} QB_ij c_i c_j (i, j >= 1)
constexpr double QBETA_11 = 1.0;
constexpr double QBETA_12 = 0.0;
constexpr double QBETA_13 = (1.0 / 2.0);
constexpr double QBETA_14 = 0.0;
constexpr double QBETA_15 = (1.0 / 8.0);
constexpr double QBETA_22 = (13.0 / 3.0);
constexpr double QBETA_23 = 0.0;
constexpr double QBETA_24 = (21.0 / 5.0);
constexpr double QBETA_25 = 0.0;
constexpr double QBETA_33 = (3129.0 / 80.0);
constexpr double QBETA_34 = 0.0;
constexpr double QBETA_35 = (14127.0 / 224.0);
constexpr double QBETA_44 = (87617.0 / 140.0);
constexpr double QBETA_45 = 0.0;
constexpr double QBETA_55 = (252337135.0 / 16128.0);
// 3-point Gauss nodes on [-1/2, 1/2] (offset) and weights
constexpr double GAUSS_G = 0.38729833462074168852;  // sqrt(15)/10
constexpr double GAUSS_W0 = (5.0 / 18.0), GAUSS_W1 = (8.0 / 18.0);
// 4-point Gauss-Lobatto nodes and weights on [0, 1]
constexpr double LOB_L1 = 0.27639320225002103036;  // 1/2 - sqrt(5)/10
constexpr double LOB_L2 = 0.72360679774997896964;  // 1/2 + sqrt(5)/10
constexpr double LOB_W0 = (1.0 / 12.0), LOB_W1 = (5.0 / 12.0);
}  // namespace shweno_tables
