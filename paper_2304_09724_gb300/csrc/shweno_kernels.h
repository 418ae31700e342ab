// Host-side launchers of the step kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "shweno_device.cuh"

namespace shweno {

// Scratch buffers of one 2D step (all device memory owned by the handle).
struct Scratch2D {
  double* ycoef;  // [2 sets][ncomp][KC coefs][ny+2][nx+4], KC = 5 (R1) or 6 (R1')
  double* xcoef;  // [2 sets][ncomp][KC coefs][nx][ny+4]
  double* FX;     // [3 gauss][ncomp][ny][nx+1]  time-averaged x-flux per Gauss point
  double* WX;     // [3 gauss][ncomp][ny][nx+1]  state at t_{n+1} per Gauss point
  double* FY;     // [3 gauss][ncomp][ny+1][nx]
  double* WY;     // [3 gauss][ncomp][ny+1][nx]
  double* WC;     // [ncomp][ny+1][nx+1]          state at t_{n+1} at cell corners
};

// ev: NULL, or events recorded before each kernel and after the last (kernels + 1 events).
constexpr int kKernels1D = 2;
constexpr int kKernels2D = 4;
void launch_step1d(const Params& P, Ctl* ctl, const double* s0, const double* s1, double* o0,
                   double* o1, const uint8_t* flag, double* FH, double* WE, cudaStream_t st,
                   cudaEvent_t* ev);
void launch_step2d(const Params& P, Ctl* ctl, const double* s0, const double* s1, double* o0,
                   double* o1, const uint8_t* flag, const Scratch2D& S, cudaStream_t st,
                   cudaEvent_t* ev);
size_t scratch2d_doubles(const Params& P);
// Kernel attributes (dynamic shared memory limits of the face kernels); call before any capture.
// Returns the first failing CUDA status.
cudaError_t init_kernels2d();
cudaError_t init_kernels2d_quintic();
void launch_step2d_quintic(const Params& P, Ctl* ctl, const double* s0, const double* s1,
                           double* o0, double* o1, const uint8_t* flag, const Scratch2D& S,
                           cudaStream_t st, cudaEvent_t* ev);
Scratch2D carve_scratch2d(const Params& P, double* base);
void launch_features2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                       float* out, cudaStream_t st);
void launch_wdev2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                   double* out, cudaStream_t st);
void launch_fdev2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                   double floor_rel, double* out, cudaStream_t st);
void launch_infer2d(const Params& P, const Ctl* ctl, const double* s0, const double* s1,
                    const float* params, float logit_thr, uint8_t* raw, uint8_t* flags,
                    cudaStream_t st);
void mlp_forward(const float* params, const float* X, int64_t n, float* prob, cudaStream_t st);
cudaError_t mlp_grad(const float* params, const float* X, const float* y, int64_t n, float pw,
                     float* grad, float* loss, cudaStream_t st);
void mlp_adam(float* params, const float* grad, float* m, float* v, float lr, float b1, float b2,
              float eps, float bc1, float bc2, cudaStream_t st);
// What the batch needs to know about a handle (filled by api.cu).
struct HandleView {
  Params P;
  Ctl* ctl;
  double* buf[2];
  const uint8_t* flags;
  Scratch2D S;
  const float* net;
  uint8_t* raw;
  uint8_t* flags_out;
  float logit_thr;
  int learned;
  cudaStream_t stream;
};
void launch_begin_step(Ctl* ctl, cudaStream_t st);
void launch_end_step(Ctl* ctl, cudaStream_t st);
void launch_rate(const Params& P, Ctl* ctl, const double* s0, const double* s1, cudaStream_t st);

}  // namespace shweno
