// Host side of the 2D step, reading R1 (the kernels are in step2d_kernels.cuh; the R1' option
// is instantiated in step2d_quintic.cu).
#include <cuda_runtime.h>

#include "step2d_kernels.cuh"

namespace shweno {

// Coefficient tables hold 2 sets x ncomp x KC coefficients per cell, KC = 5 (R1) or 6 (R1').
size_t scratch2d_doubles(const Params& P) {
  const size_t nx = P.nx, ny = P.ny, nc = P.ncomp, kc = P.quintic ? 6 : 5;
  return 2 * kc * nc * (ny + 2) * (nx + 4) + 2 * kc * nc * nx * (ny + 4) + 2 * 3 * nc * ny * (nx + 1) +
         2 * 3 * nc * (ny + 1) * nx + nc * (ny + 1) * (nx + 1);
}

Scratch2D carve_scratch2d(const Params& P, double* base) {
  const size_t nx = P.nx, ny = P.ny, nc = P.ncomp, kc = P.quintic ? 6 : 5;
  Scratch2D S;
  S.ycoef = base; base += 2 * kc * nc * (ny + 2) * (nx + 4);
  S.xcoef = base; base += 2 * kc * nc * nx * (ny + 4);
  S.FX = base; base += 3 * nc * ny * (nx + 1);
  S.WX = base; base += 3 * nc * ny * (nx + 1);
  S.FY = base; base += 3 * nc * (ny + 1) * nx;
  S.WY = base; base += 3 * nc * (ny + 1) * nx;
  S.WC = base;
  return S;
}

cudaError_t init_kernels2d() {
  const cudaError_t e = init_kernels2d_reading<false>();
  return e != cudaSuccess ? e : init_kernels2d_quintic();
}

void launch_step2d(const Params& P, Ctl* ctl, const double* s0, const double* s1, double* o0,
                   double* o1, const uint8_t* flag, const Scratch2D& S, cudaStream_t st,
                   cudaEvent_t* ev) {
  if (P.quintic) launch_step2d_quintic(P, ctl, s0, s1, o0, o1, flag, S, st, ev);
  else launch_step2d_reading<false>(P, ctl, s0, s1, o0, o1, flag, S, st, ev);
}

}  // namespace shweno
