// One ADER-SHWENO time step in two space dimensions (Section 3; Section 4 Steps 1-5).
//
// The SHWENO reconstruction runs dimension by dimension (Section 3.2): a first 1D pass along
// the face gives line averages of W and of its normal derivative as polynomials in the
// tangential coordinate, a second pass across the face gives all mixed derivatives
// d^{m+n}W/dx^m dy^n (m + n <= 4) on both sides of each face quadrature point.
//
//   coef2d   one thread per cell (ghost ring included): the first-pass polynomials of both
//            directions, y-pass on {W, Y} and {V, Z}, x-pass on {W, V} and {Y, Z}; the stencil
//            tile (4 fields x NC components with a one-cell halo) is staged in shared memory.
//   xface2d  one CTA per 128 x-faces of a row and one Gauss point (or the corner row): the CTA
//            evaluates the y-pass polynomials of the 131 columns it needs at eta_g into shared
//            memory, then each thread owns one face point: x-pass on both sides, leading term
//            (Eq. 3.6: HLLC, or the exact Burgers state), eigen-upwinded derivatives (Eq. 3.7),
//            Cauchy-Kovalevskaya (Section 3.1), Lobatto flux (Eq. 3.8) and W(t_{n+1})
//            (Eq. 3.11).  The corner row averages the y-pass traces of the rows below and above
//            and keeps only W(t_{n+1}).
//   yface2d  the same for y-faces, one CTA per 128 faces of a column.
//   update2d one thread per cell: Eq. (3.2) and Eq. (3.10), physical check, CFL rate.
// Every kernel is instantiated for NC = 1 (scalar Burgers) and NC = 4 (Euler), and for reading
// R1 (quartic p1) in step2d.cu and the R1' option (quintic p1) in step2d_quintic.cu, so the two
// translation units compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "shweno_kernels.h"
#include "step2d_items.cuh"

namespace shweno {

constexpr int TY = 8;  // coef2d tile height of the one-mesh kernel

template <int NC, bool Q>
__global__ void __launch_bounds__(TX * TY) coef2d_kernel(Params P, const Ctl* __restrict__ ctl,
                                                         const double* s0, const double* s1,
                                                         const uint8_t* __restrict__ flag,
                                                         double* __restrict__ ycoef,
                                                         double* __restrict__ xcoef) {
  __shared__ double tile[16][TY + 2][TX + 2];
  if (!ctl->active) return;
  coef2d_item<NC, TY, Q>(P, step_view(ctl), s0, s1, flag, ycoef, xcoef, blockIdx.x * TX - 2, blockIdx.y * TY - 2, tile,
                  threadIdx.x, threadIdx.y);
}

template <int NC, bool FLAGS, bool CHAR, bool Q>
__global__ void __launch_bounds__(SEG) xface2d_kernel(Params P, const Ctl* __restrict__ ctl,
                                                      const double* s0, const double* s1,
                                                      const double* __restrict__ ycoef,
                                                      const uint8_t* __restrict__ flag,
                                                      double* __restrict__ FX,
                                                      double* __restrict__ WX,
                                                      double* __restrict__ WC) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!ctl->active) return;
  const int slice = blockIdx.z;  // 0..2: Gauss point of the rows; 3: corner rows
  const int row = blockIdx.y;    // Gauss: cell row j; corner: corner row jc (y_{jc-1/2})
  if (slice < 3 && row >= P.ny) return;
  const StepView sv = step_view(ctl);
  xface_item<NC, FLAGS, CHAR, Q>(P, sv, sv.odd ? s1 : s0, ycoef, flag, FX, WX, WC, blockIdx.x * NFACE, row, slice,
                              smem_raw);
}

template <int NC, bool FLAGS, bool CHAR, bool Q>
__global__ void __launch_bounds__(SEG) yface2d_kernel(Params P, const Ctl* __restrict__ ctl,
                                                      const double* s0, const double* s1,
                                                      const double* __restrict__ xcoef,
                                                      const uint8_t* __restrict__ flag,
                                                      double* __restrict__ FY,
                                                      double* __restrict__ WY) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!ctl->active) return;
  const StepView sv = step_view(ctl);
  yface_item<NC, FLAGS, CHAR, Q>(P, sv, sv.odd ? s1 : s0, xcoef, flag, FY, WY, blockIdx.x * NFACE, blockIdx.y,
                              blockIdx.z, smem_raw);
}

template <int NC>
__global__ void __launch_bounds__(256) update2d_kernel(Params P, Ctl* __restrict__ ctl,
                                                       const double* s0, const double* s1,
                                                       double* o0, double* o1,
                                                       const double* __restrict__ FX,
                                                       const double* __restrict__ WX,
                                                       const double* __restrict__ FY,
                                                       const double* __restrict__ WY,
                                                       const double* __restrict__ WC) {
  __shared__ double red[32];
  if (!ctl->active) return;
  const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
  const StepView sv = step_view(ctl);
  double rate = 0.0;
  if (i < P.nx && j < P.ny) rate = update2d_cell<NC>(P, ctl, sv, sv.odd ? s1 : s0, sv.odd ? o0 : o1, FX, WX, FY, WY, WC, i, j);
  block_max_rate(rate, &ctl->rate_next, red);
}

// ------------------------------------------------------------------ host side (templates)
// Dynamic shared memory limits of the face kernels; returns the first failing call's status.
template <int NC, bool CHAR, bool Q>
static cudaError_t init_kernels2d_nc() {
  cudaError_t e = cudaSuccess;
  auto set = [&e](const void* f, size_t bytes) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = r;
  };
  set((const void*)xface2d_kernel<NC, false, CHAR, Q>, kFaceSmem);
  set((const void*)yface2d_kernel<NC, false, CHAR, Q>, kFaceSmem);
  set((const void*)xface2d_kernel<NC, true, CHAR, Q>, kFaceSmem);
  set((const void*)yface2d_kernel<NC, true, CHAR, Q>, kFaceSmem);
  return e;
}

// Attributes of every face kernel of one reading (Q = false: R1, true: R1').
template <bool Q>
static cudaError_t init_kernels2d_reading() {
  cudaError_t e = init_kernels2d_nc<1, false, Q>();
  if (e == cudaSuccess) e = init_kernels2d_nc<4, false, Q>();
  if (e == cudaSuccess) e = init_kernels2d_nc<4, true, Q>();
  return e;
}


// The two face kernels of a step (x-faces with the corner rows, then y-faces).
template <int NC, bool CHAR, bool Q>
static void launch_faces2d(const Params& P, Ctl* ctl, const double* s0, const double* s1,
                           const uint8_t* flag, const Scratch2D& S, cudaStream_t st, cudaEvent_t* ev) {
  dim3 xg((P.nx + 1 + NFACE - 1) / NFACE, P.ny + 1, 4);
  if (P.flag_mode == FLAG_ALL_NONLINEAR)
    xface2d_kernel<NC, false, CHAR, Q><<<xg, SEG, kFaceSmem, st>>>(P, ctl, s0, s1, S.ycoef, flag, S.FX, S.WX, S.WC);
  else
    xface2d_kernel<NC, true, CHAR, Q><<<xg, SEG, kFaceSmem, st>>>(P, ctl, s0, s1, S.ycoef, flag, S.FX, S.WX, S.WC);
  if (ev) cudaEventRecord(ev[2], st);
  dim3 yg((P.ny + 1 + NFACE - 1) / NFACE, P.nx, 3);
  if (P.flag_mode == FLAG_ALL_NONLINEAR)
    yface2d_kernel<NC, false, CHAR, Q><<<yg, SEG, kFaceSmem, st>>>(P, ctl, s0, s1, S.xcoef, flag, S.FY, S.WY);
  else
    yface2d_kernel<NC, true, CHAR, Q><<<yg, SEG, kFaceSmem, st>>>(P, ctl, s0, s1, S.xcoef, flag, S.FY, S.WY);
}

template <int NC, bool Q>
static void launch_step2d_nc(const Params& P, Ctl* ctl, const double* s0, const double* s1,
                             double* o0, double* o1, const uint8_t* flag, const Scratch2D& S,
                             cudaStream_t st, cudaEvent_t* ev) {
  dim3 cb(TX, TY), cg((P.nx + 4 + TX - 1) / TX, (P.ny + 4 + TY - 1) / TY);
  if (ev) cudaEventRecord(ev[0], st);
  coef2d_kernel<NC, Q><<<cg, cb, 0, st>>>(P, ctl, s0, s1, flag, S.ycoef, S.xcoef);
  if (ev) cudaEventRecord(ev[1], st);
  if constexpr (NC == 4) {
    if (P.charwise) launch_faces2d<NC, true, Q>(P, ctl, s0, s1, flag, S, st, ev);
    else launch_faces2d<NC, false, Q>(P, ctl, s0, s1, flag, S, st, ev);
  } else {
    launch_faces2d<NC, false, Q>(P, ctl, s0, s1, flag, S, st, ev);
  }
  if (ev) cudaEventRecord(ev[3], st);
  dim3 ug((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  update2d_kernel<NC><<<ug, cb, 0, st>>>(P, ctl, s0, s1, o0, o1, S.FX, S.WX, S.FY, S.WY, S.WC);
  if (ev) cudaEventRecord(ev[4], st);
}

// Both component counts of one reading.
template <bool Q>
static void launch_step2d_reading(const Params& P, Ctl* ctl, const double* s0, const double* s1,
                                  double* o0, double* o1, const uint8_t* flag, const Scratch2D& S,
                                  cudaStream_t st, cudaEvent_t* ev) {
  if (P.ncomp == 1) launch_step2d_nc<1, Q>(P, ctl, s0, s1, o0, o1, flag, S, st, ev);
  else launch_step2d_nc<4, Q>(P, ctl, s0, s1, o0, o1, flag, S, st, ev);
}

}  // namespace shweno
