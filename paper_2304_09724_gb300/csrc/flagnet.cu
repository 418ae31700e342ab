// Learned troubled-cell flag: a small MLP decides per cell whether the SHWENO reconstructions
// anchored on it need the nonlinear weights (flag 1) or may use the linear weights (flag 0),
// which makes them exactly the big-stencil polynomial p1 and skips the smoothness indicators.
// The paper has no such component; it is the learned layer put on top of the method.
//
//   features2d   22 inputs per cell from the committed state (FP64 arithmetic, stored FP32):
//                for rho and E, the eight 3x3 neighbours minus the centre and dx V, dy Y of the
//                centre, divided by (stencil range + 1e-12 |centre| + 1e-300), and
//                log10(range / (|centre| + 1e-30) + 1e-16) / 8.
//   wdev2d       label source: per cell, the largest relative deviation
//                max_l |w_l - gamma_l| / gamma_l of the 16 first-pass reconstructions anchored
//                on it (the plain scheme's own weights).
//   fdev2d       training label source: per cell, the largest change those weights make to the
//                reconstructions' end values, |p(+-1/2) - p1(+-1/2)|, relative to the range of the
//                reconstruction's three averages plus the caller's floor times |W0|.
//   mlp_forward / mlp_grad / mlp_adam   FP32 network 22 -> 32 -> 32 -> 1 (ReLU, ReLU, sigmoid),
//                binary cross-entropy with a positive-class weight, Adam.
//   infer2d + dilate2d   each step, before the reconstruction: flag = net(features) > threshold,
//                then dilated by one cell (3x3 OR), imposed-state ghost cells count as troubled.
#include <cuda_runtime.h>

#include "flagnet_items.cuh"
#include "shweno_kernels.h"

namespace shweno {

__global__ void features2d_kernel(Params P, const Ctl* __restrict__ ctl, const double* s0,
                                  const double* s1, float* __restrict__ out) {
  const size_t cells = (size_t)P.nx * P.ny;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const double* st = (ctl->nsteps & 1) ? s1 : s0;
  float f[NIN];
  cell_features(P, st, (int)(c % P.nx), (int)(c / P.nx), ctl->t, f);
#pragma unroll
  for (int k = 0; k < NIN; ++k) out[c * NIN + k] = f[k];
}

__global__ void wdev2d_kernel(Params P, const Ctl* __restrict__ ctl, const double* s0,
                              const double* s1, double* __restrict__ out) {
  const size_t cells = (size_t)P.nx * P.ny;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const double* st = (ctl->nsteps & 1) ? s1 : s0;
  const int i = (int)(c % P.nx), j = (int)(c / P.nx);
  const double t = ctl->t;
  double dev = 0.0;
  for (int pass = 0; pass < 2; ++pass)
    for (int set = 0; set < 2; ++set)
      for (int q = 0; q < P.ncomp; ++q) {
        const int fa = pass == 0 ? (set == 0 ? 0 : 1) : (set == 0 ? 0 : 2);
        const int fd = pass == 0 ? (set == 0 ? 2 : 3) : (set == 0 ? 1 : 3);
        const int di = pass == 1, dj = pass == 0;
        const double h = pass == 0 ? P.dy : P.dx;
        const double Wm = fetch(P, st, fa, q, i - di, j - dj, t), W0 = fetch(P, st, fa, q, i, j, t);
        const double Wp = fetch(P, st, fa, q, i + di, j + dj, t);
        double cf[5];
        p1_coeffs(Wm, W0, Wp, h * fetch(P, st, fd, q, i - di, j - dj, t), h * fetch(P, st, fd, q, i + di, j + dj, t), cf);
        const Mix m = shweno_mix(P, Wm, W0, Wp, cf, 1);
        // back from (A, B, C) to the weights: w1 = A g1, w2 = B + A g2, w3 = C + A g3
        const double w[3] = {m.A * P.gam[0], m.B + m.A * P.gam[1], m.C + m.A * P.gam[2]};
        for (int l = 0; l < 3; ++l) dev = fmax(dev, fabs(w[l] - P.gam[l]) / P.gam[l]);
      }
  out[c] = dev;
}

__global__ void fdev2d_kernel(Params P, const Ctl* __restrict__ ctl, const double* s0,
                              const double* s1, double floor_rel, double* __restrict__ out) {
  const size_t cells = (size_t)P.nx * P.ny;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const double* st = (ctl->nsteps & 1) ? s1 : s0;
  const int i = (int)(c % P.nx), j = (int)(c / P.nx);
  const double t = ctl->t;
  double dev = 0.0;
  for (int pass = 0; pass < 2; ++pass)
    for (int set = 0; set < 2; ++set)
      for (int q = 0; q < P.ncomp; ++q) {
        const int fa = pass == 0 ? (set == 0 ? 0 : 1) : (set == 0 ? 0 : 2);
        const int fd = pass == 0 ? (set == 0 ? 2 : 3) : (set == 0 ? 1 : 3);
        const int di = pass == 1, dj = pass == 0;
        const double h = pass == 0 ? P.dy : P.dx;
        const double Wm = fetch(P, st, fa, q, i - di, j - dj, t), W0 = fetch(P, st, fa, q, i, j, t);
        const double Wp = fetch(P, st, fa, q, i + di, j + dj, t);
        double cf[5];
        p1_coeffs(Wm, W0, Wp, h * fetch(P, st, fd, q, i - di, j - dj, t), h * fetch(P, st, fd, q, i + di, j + dj, t), cf);
        const Mix m = shweno_mix(P, Wm, W0, Wp, cf, 1);
        // p - p1 = (A - 1) p1 + B p2 + C p3 at xi = +-1/2 (p2 = W0 + (W0 - W-) xi, p3 = W0 + (W+ - W0) xi)
        const double even = cf[0] + 0.25 * cf[2] + 0.0625 * cf[4], odd = 0.5 * cf[1] + 0.125 * cf[3];
        const double s2 = 0.5 * (W0 - Wm), s3 = 0.5 * (Wp - W0);
        const double scale = fmax(Wm, fmax(W0, Wp)) - fmin(Wm, fmin(W0, Wp)) + floor_rel * fabs(W0) + 1e-300;
        const double dR = (m.A - 1.0) * (even + odd) + m.B * (W0 + s2) + m.C * (W0 + s3);
        const double dL = (m.A - 1.0) * (even - odd) + m.B * (W0 - s2) + m.C * (W0 - s3);
        dev = fmax(dev, fmax(fabs(dR), fabs(dL)) / scale);
      }
  out[c] = dev;
}

__global__ void mlp_forward_kernel(const float* __restrict__ params, const float* __restrict__ X,
                                   int64_t n, float* __restrict__ prob) {
  __shared__ float p[NPARAM];
  load_params(params, p);
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float x[NIN];
#pragma unroll
  for (int j = 0; j < NIN; ++j) x[j] = X[b * NIN + j];
  prob[b] = 1.f / (1.f + expf(-net_logit(p, x)));
}

// Gradient of mean BCE over n samples.  A CTA handles GB samples: each thread runs forward and
// backward for one sample into shared memory, then the CTA reduces every parameter's gradient
// over its samples and adds it to grad with one atomicAdd per parameter.
constexpr int GB = 128;
struct GradSmem {
  float p[NPARAM];
  float x[GB][NIN];
  float h1[GB][NH], h2[GB][NH], d1[GB][NH], d2[GB][NH];
  float d3[GB];
  float red[GB / 32];
};

__global__ void __launch_bounds__(GB) mlp_grad_kernel(const float* __restrict__ params,
                                                      const float* __restrict__ X,
                                                      const float* __restrict__ y, int64_t n,
                                                      float pw, float* __restrict__ grad,
                                                      float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char raw[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(raw);
  for (int k = threadIdx.x; k < NPARAM; k += GB) S.p[k] = params[k];
  __syncthreads();
  const int tid = threadIdx.x;
  const int64_t b = (int64_t)blockIdx.x * GB + tid;
  const float* p = S.p;
  float l = 0.f;
  if (b < n) {
    float x[NIN], z1[NH], h1[NH], z2[NH];
#pragma unroll
    for (int j = 0; j < NIN; ++j) x[j] = S.x[tid][j] = X[b * NIN + j];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      float z = p[OFF_B1 + i];
#pragma unroll
      for (int j = 0; j < NIN; ++j) z = fmaf(p[OFF_W1 + i * NIN + j], x[j], z);
      z1[i] = z;
      h1[i] = S.h1[tid][i] = fmaxf(z, 0.f);
    }
    float z3 = p[OFF_B3];
    for (int i = 0; i < NH; ++i) {
      float z = p[OFF_B2 + i];
#pragma unroll
      for (int j = 0; j < NH; ++j) z = fmaf(p[OFF_W2 + i * NH + j], h1[j], z);
      z2[i] = z;
      S.h2[tid][i] = fmaxf(z, 0.f);
      z3 = fmaf(p[OFF_W3 + i], fmaxf(z, 0.f), z3);
    }
    const float yy = y[b];
    const float sg = 1.f / (1.f + expf(-z3));
    // per-sample loss, stable: -pw y log(sig) - (1 - y) log(1 - sig)
    const float sp_neg = log1pf(expf(-fabsf(z3))) + fmaxf(-z3, 0.f);  // -log(sig(z))
    const float sp_pos = sp_neg + z3;                                    // -log(1 - sig(z))
    l = pw * yy * sp_neg + (1.f - yy) * sp_pos;
    const float d3 = (-pw * yy * (1.f - sg) + (1.f - yy) * sg) / (float)n;
    S.d3[tid] = d3;
    float d2[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) d2[i] = S.d2[tid][i] = z2[i] > 0.f ? d3 * p[OFF_W3 + i] : 0.f;
    for (int j = 0; j < NH; ++j) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < NH; ++i) s = fmaf(p[OFF_W2 + i * NH + j], d2[i], s);
      S.d1[tid][j] = z1[j] > 0.f ? s : 0.f;
    }
  } else {
    for (int j = 0; j < NIN; ++j) S.x[tid][j] = 0.f;
    for (int i = 0; i < NH; ++i) S.h1[tid][i] = S.h2[tid][i] = S.d1[tid][i] = S.d2[tid][i] = 0.f;
    S.d3[tid] = 0.f;
  }
  // loss: block sum, one atomic per CTA
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((tid & 31) == 0) S.red[tid >> 5] = l;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < GB / 32; ++w) s += S.red[w];
    atomicAdd(loss, s / (float)n);
  }
  // parameter gradients: sums over the CTA's samples
  for (int k = tid; k < NPARAM; k += GB) {
    float s = 0.f;
    if (k < OFF_B1) {
      const int i = k / NIN, j = k % NIN;
      for (int bb = 0; bb < GB; ++bb) s = fmaf(S.d1[bb][i], S.x[bb][j], s);
    } else if (k < OFF_W2) {
      const int i = k - OFF_B1;
      for (int bb = 0; bb < GB; ++bb) s += S.d1[bb][i];
    } else if (k < OFF_B2) {
      const int i = (k - OFF_W2) / NH, j = (k - OFF_W2) % NH;
      for (int bb = 0; bb < GB; ++bb) s = fmaf(S.d2[bb][i], S.h1[bb][j], s);
    } else if (k < OFF_W3) {
      const int i = k - OFF_B2;
      for (int bb = 0; bb < GB; ++bb) s += S.d2[bb][i];
    } else if (k < OFF_B3) {
      const int i = k - OFF_W3;
      for (int bb = 0; bb < GB; ++bb) s = fmaf(S.d3[bb], S.h2[bb][i], s);
    } else {
      for (int bb = 0; bb < GB; ++bb) s += S.d3[bb];
    }
    atomicAdd(&grad[k], s);
  }
}

__global__ void mlp_adam_kernel(float* __restrict__ params, const float* __restrict__ grad,
                                float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                float b2, float eps, float bc1, float bc2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float g = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  params[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
}

// ------------------------------------------------------------------ per-step inference
__global__ void infer2d_kernel(Params P, const Ctl* __restrict__ ctl, const double* s0,
                               const double* s1, const float* __restrict__ params, float logit_thr,
                               uint8_t* __restrict__ raw) {
  __shared__ float p[NPARAM];
  if (!ctl->active) return;
  load_params(params, p);
  const size_t cells = (size_t)P.nx * P.ny;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const double* st = (ctl->nsteps & 1) ? s1 : s0;
  float f[NIN];
  cell_features(P, st, (int)(c % P.nx), (int)(c / P.nx), ctl->t, f);
  raw[c] = net_logit(p, f) > logit_thr ? 1 : 0;
}

__global__ void dilate2d_kernel(Params P, const Ctl* __restrict__ ctl, const uint8_t* __restrict__ raw,
                                uint8_t* __restrict__ flags) {
  if (!ctl->active) return;
  const size_t cells = (size_t)P.nx * P.ny;
  const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const int i = (int)(c % P.nx), j = (int)(c / P.nx);
  int f = 0;
  for (int dj = -1; dj <= 1; ++dj)
    for (int di = -1; di <= 1; ++di) f |= raw_flag(P, raw, i + di, j + dj);
  flags[c] = (uint8_t)f;
}

// ------------------------------------------------------------------ host launchers
void launch_features2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                       float* out, cudaStream_t st) {
  const size_t cells = (size_t)P.nx * P.ny;
  features2d_kernel<<<(unsigned)((cells + 127) / 128), 128, 0, st>>>(P, ctl, s0, s1, out);
}
void launch_fdev2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                   double floor_rel, double* out, cudaStream_t st) {
  const size_t cells = (size_t)P.nx * P.ny;
  fdev2d_kernel<<<(unsigned)((cells + 127) / 128), 128, 0, st>>>(P, ctl, s0, s1, floor_rel, out);
}

void launch_wdev2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                   double* out, cudaStream_t st) {
  const size_t cells = (size_t)P.nx * P.ny;
  wdev2d_kernel<<<(unsigned)((cells + 127) / 128), 128, 0, st>>>(P, ctl, s0, s1, out);
}
void launch_infer2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                    const float* params, float logit_thr, uint8_t* raw, uint8_t* flags,
                    cudaStream_t st) {
  const size_t cells = (size_t)P.nx * P.ny;
  const unsigned g = (unsigned)((cells + 255) / 256);
  infer2d_kernel<<<g, 256, 0, st>>>(P, ctl, s0, s1, params, logit_thr, raw);
  dilate2d_kernel<<<g, 256, 0, st>>>(P, ctl, raw, flags);
}
void mlp_forward(const float* params, const float* X, int64_t n, float* prob, cudaStream_t st) {
  if (n > 0) mlp_forward_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, X, n, prob);
}
cudaError_t mlp_grad(const float* params, const float* X, const float* y, int64_t n, float pw,
                     float* grad, float* loss, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(GradSmem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), st);
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (n > 0)
    mlp_grad_kernel<<<(unsigned)((n + GB - 1) / GB), GB, sizeof(GradSmem), st>>>(params, X, y, n, pw, grad, loss);
  return cudaGetLastError();
}
void mlp_adam(float* params, const float* grad, float* m, float* v, float lr, float b1, float b2,
              float eps, float bc1, float bc2, cudaStream_t st) {
  mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(params, grad, m, v, lr, b1, b2, eps, bc1, bc2);
}

}  // namespace shweno
