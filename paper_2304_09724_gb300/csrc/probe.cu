// FP64 throughput probe: the denominator of the step kernels' roofline.
//
// The scheme runs in FP64 and its face kernels are bound by the FP64 pipe, whose rate the GPU's
// data sheet states only loosely for this part.  The probe measures it: every thread runs four
// independent chains of one FP64 operation -- fused multiply-add x <- x * b + c, multiply
// x <- x * b or add x <- x + c -- or of the three interleaved (two fused chains, one product,
// one sum), for `iters` iterations (b and c are kernel arguments, so nothing folds), one CTA of
// warps_per_sm warps per SM.  Thread 0 of CTA 0 reads the SM cycle
// counter around its loop, so the call also returns the rate per SM clock, which does not depend
// on the clock the GPU ran at.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/shweno.h"

namespace {

constexpr int kChains = 4;

__device__ double g_probe_sink;
__device__ long long g_probe_cycles;

template <int OP>  // 0: fma, 1: mul, 2: add, 3: fma, fma, mul, add
__global__ void fp64_probe_kernel(int64_t iters, double b, double c, double sentinel) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const double ca = c * 0x1p-20;  // the sum chains' increment
  const long long c0 = clock64();
  for (int64_t i = 0; i < iters; ++i) {
    if constexpr (OP == 3) {
      static_assert(kChains == 4, "the mixed stream interleaves four chains");
      x[0] = fma(x[0], b, c);
      x[1] = fma(x[1], b, c);
      x[2] = x[2] * b;
      x[3] = x[3] + ca;
    } else {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        if constexpr (OP == 0) x[k] = fma(x[k], b, c);
        else if constexpr (OP == 1) x[k] = x[k] * b;
        else x[k] = x[k] + ca;
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (threadIdx.x == 0 && blockIdx.x == 0) g_probe_cycles = clock64() - c0;
  if (s == sentinel) g_probe_sink = s;  // never true for the arguments the host passes
}

}  // namespace

extern "C" shweno_status shweno_fp64_probe(int32_t op, int32_t warps_per_sm, int64_t iters,
                                           void* cuda_stream, double* tflops_out,
                                           double* ops_per_clk_per_sm_out) {
  if (op < 0 || op > 3 || warps_per_sm < 1 || warps_per_sm > 32 || iters < 1 ||
      iters > (int64_t(1) << 24) || !tflops_out)
    return SHWENO_E_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SHWENO_E_CUDA;
  const int threads = 32 * warps_per_sm;
  // |x| stays near 1: with b = 1 - 2^-20 and c = 2^-20 the fused chain has the fixed point 1; the
  // product chain decays by 2^-20 and the sum chain grows by 2^-40 per iteration
  const double b = 1.0 - 0x1p-20, c = 0x1p-20;
  auto launch = [&](int64_t n) {
    if (op == 0) fp64_probe_kernel<0><<<sms, threads, 0, st>>>(n, b, c, -1.0);
    else if (op == 1) fp64_probe_kernel<1><<<sms, threads, 0, st>>>(n, b, c, -1.0);
    else if (op == 2) fp64_probe_kernel<2><<<sms, threads, 0, st>>>(n, b, c, -1.0);
    else fp64_probe_kernel<3><<<sms, threads, 0, st>>>(n, b, c, -1.0);
  };
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SHWENO_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SHWENO_E_CUDA;
  }
  launch(iters / 8 + 1);  // warm-up
  cudaEventRecord(e0, st);
  launch(iters);
  cudaEventRecord(e1, st);
  float ms = 0.0f;
  long long cycles = 0;
  cudaError_t err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaMemcpyFromSymbol(&cycles, g_probe_cycles, sizeof(cycles));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || ms <= 0.0f) return SHWENO_E_CUDA;
  const double ops = (double)sms * threads * kChains * (double)iters;
  const double flops_per_op = op == 0 ? 2.0 : (op == 3 ? 1.5 : 1.0);
  *tflops_out = flops_per_op * ops / (ms * 1e-3) / 1e12;
  if (ops_per_clk_per_sm_out)
    *ops_per_clk_per_sm_out = cycles > 0 ? (double)threads * kChains * (double)iters / (double)cycles : 0.0;
  return SHWENO_OK;
}
