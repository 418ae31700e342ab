// Per-item device functions of the learned troubled-cell flag (features, network, flag
// dilation), shared by flagnet.cu and the batched persistent kernel (batch.cu).
#pragma once
#include "../../include/shweno.h"
#include "shweno_device.cuh"

namespace shweno {

constexpr int NIN = SHWENO_FLAG_FEATURES, NH = 32;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == SHWENO_FLAG_PARAMS, "parameter count");

// ------------------------------------------------------------------ features
__device__ __forceinline__ void cell_features(const Params& P, const double* st, int i, int j,
                                              double t, float f[NIN]) {
  const int comps[2] = {0, P.ncomp - 1};
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int q = comps[a];
    double v[3][3];
    double mn = 1e300, mx = -1e300;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const double x = fetch(P, st, 0, q, i + di, j + dj, t);
        v[dj + 1][di + 1] = x;
        mn = fmin(mn, x);
        mx = fmax(mx, x);
      }
    const double c = v[1][1], range = mx - mn;
    const double sc = range + 1e-12 * fabs(c) + 1e-300;
    const double is = 1.0 / sc;
    int k = 0;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di)
        if (di != 0 || dj != 0) f[a * 11 + k++] = (float)((v[dj + 1][di + 1] - c) * is);
    f[a * 11 + 8] = (float)(P.dx * fetch(P, st, 1, q, i, j, t) * is);
    f[a * 11 + 9] = (float)(P.dy * fetch(P, st, 2, q, i, j, t) * is);
    f[a * 11 + 10] = (float)(log10(range / (fabs(c) + 1e-30) + 1e-16) * 0.125);
  }
}

// ------------------------------------------------------------------ network
__device__ __forceinline__ float net_logit(const float* __restrict__ p, const float x[NIN]) {
  float h1[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    float z = p[OFF_B1 + i];
#pragma unroll
    for (int j = 0; j < NIN; ++j) z = fmaf(p[OFF_W1 + i * NIN + j], x[j], z);
    h1[i] = fmaxf(z, 0.f);
  }
  float out = p[OFF_B3];
#pragma unroll 4
  for (int i = 0; i < NH; ++i) {
    float z = p[OFF_B2 + i];
#pragma unroll
    for (int j = 0; j < NH; ++j) z = fmaf(p[OFF_W2 + i * NH + j], h1[j], z);
    out = fmaf(p[OFF_W3 + i], fmaxf(z, 0.f), out);
  }
  return out;
}

__device__ __forceinline__ void load_params(const float* __restrict__ g, float* s) {
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) s[k] = __ldcg(g + k);
  __syncthreads();
}

__device__ __forceinline__ int raw_flag(const Params& P, const uint8_t* raw, int i, int j) {
  if (i < 0 || i >= P.nx) {
    const int k = P.bc[i < 0 ? 0 : 1];
    if (k == BC_PERIODIC) i = ((i % P.nx) + P.nx) % P.nx;
    else if (k == BC_OUTFLOW) i = i < 0 ? 0 : P.nx - 1;
    else if (k == BC_REFLECTIVE) i = i < 0 ? -1 - i : 2 * P.nx - 1 - i;
    else return 1;
  }
  if (j < 0 || j >= P.ny) {
    const int k = P.bc[j < 0 ? 2 : 3];
    if (k == BC_PERIODIC) j = ((j % P.ny) + P.ny) % P.ny;
    else if (k == BC_OUTFLOW) j = j < 0 ? 0 : P.ny - 1;
    else if (k == BC_REFLECTIVE) j = j < 0 ? -1 - j : 2 * P.ny - 1 - j;
    else return 1;
  }
  return __ldcg(raw + (size_t)j * P.nx + i);
}

}  // namespace shweno
