// The 2D step kernels of the R1' option (quintic p1 that also matches the cell's own derivative
// average), in a translation unit of their own so that they compile beside step2d.cu.
#include <cuda_runtime.h>

#include "step2d_kernels.cuh"

namespace shweno {

cudaError_t init_kernels2d_quintic() { return init_kernels2d_reading<true>(); }

void launch_step2d_quintic(const Params& P, Ctl* ctl, const double* s0, const double* s1,
                           double* o0, double* o1, const uint8_t* flag, const Scratch2D& S,
                           cudaStream_t st, cudaEvent_t* ev) {
  launch_step2d_reading<true>(P, ctl, s0, s1, o0, o1, flag, S, st, ev);
}

}  // namespace shweno
