/*
 * shweno.h -- C ABI of the GB300 (sm_103a) FP64 library for the one-stage ADER-SHWENO scheme
 * of Luo, Li, Qiu, Zhu and Chen, "A compact simple HWENO scheme with ADER time discretization
 * for hyperbolic conservation laws I: structured meshes" (arXiv 2304.09724).
 *
 * Problem (Section 2, Eq. 2.1; Section 3, Eq. 3.1): W_t + F(W)_x (+ G(W)_y) = 0 on a uniform
 * Cartesian mesh, for scalar Burgers (F = G = W^2/2) or the compressible Euler equations of an
 * ideal gas (Eq. 5.1, 5.2; E = p/(gamma-1) + rho |u|^2/2).  The state of the method is, per cell,
 * the cell average W, the cell average V of W_x and, in 2D, the averages Y of W_y and Z of W_xy
 * (Section 2.5 Eq. 2.10; Section 3.2 Eq. 3.9).  One step is Section 4, Steps 1-5: SHWENO
 * reconstruction, Lax-Wendroff (Cauchy-Kovalevskaya) procedure, leading term and derivative
 * Riemann problems, Lobatto-in-time flux, update of W (Eq. 2.2 / 3.2) and of V, Y, Z
 * (Eq. 2.11 / 3.10).
 *
 * Layout of every state array: float64, component-major, x fastest, no ghost cells:
 *   1D: [ncomp][nx]          2D: [ncomp][ny][nx]
 * ncomp = 1 (Burgers), 3 (1D Euler: rho, rho u, E), 4 (2D Euler: rho, rho u, rho v, E).
 *
 * Conventions for every call:
 *  - Every call returns a shweno_status; nothing throws across the ABI.  On error the handle's
 *    message is available through shweno_last_error().
 *  - Pointers marked "device" must be device memory of the handle's GPU; "host" pointers are
 *    ordinary host memory.  Copies are ordered on the handle's CUDA stream; calls that return
 *    data to the host synchronise that stream.
 *  - The library owns its device buffers (two state buffers and the step scratch); callers keep
 *    ownership of everything they pass in.
 *  - One thread at a time per handle.
 */
#ifndef SHWENO_H
#define SHWENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SHWENO_OK = 0,
  SHWENO_E_INVALID = 1,      /* bad argument; nothing was changed */
  SHWENO_E_CUDA = 2,         /* a CUDA call failed; message in shweno_last_error() */
  SHWENO_E_NOMEM = 3,        /* device allocation failed */
  SHWENO_E_NONPHYSICAL = 4,  /* a step produced rho <= 0, p <= 0 or a NaN; that step was not
                                committed: the state and time are those before it */
  SHWENO_E_TIMEOUT = 5,      /* a bounded device-side wait gave up (batched runs) */
  SHWENO_E_STATE = 6         /* call not valid in the handle's current state */
} shweno_status;

typedef enum { SHWENO_BURGERS = 0, SHWENO_EULER = 1 } shweno_eq;

/* Boundary conditions (Section 5 examples).  Ghost cells are never stored; they are mapped
 * on load.  OUTFLOW copies every cell quantity of the boundary cell (zero-order extrapolation,
 * the non-reflecting (outflow) sides of Examples 5.3, 5.9, 5.10).  REFLECTIVE mirrors the
 * state with the normal momentum and the derivatives normal to the wall changing sign
 * (Example 5.6).  INFLOW imposes the conserved state inflow[side] with zero derivatives.
 * DMR_BOTTOM / DMR_TOP are the lower and upper sides of the double Mach reflection problem
 * (Example 5.10): exact post-shock state for x < 1/6 and a wall beyond; exact position of the
 * Mach 10 shock at the current time, sampled at ghost-cell centres. */
typedef enum {
  SHWENO_BC_PERIODIC = 0,
  SHWENO_BC_OUTFLOW = 1,
  SHWENO_BC_REFLECTIVE = 2,
  SHWENO_BC_INFLOW = 3,
  SHWENO_BC_DMR_BOTTOM = 4,  /* Euler only, y-low side */
  SHWENO_BC_DMR_TOP = 5      /* Euler only, y-high side */
} shweno_bc_kind;

typedef struct {
  int32_t dim;        /* 1 or 2 */
  int32_t eq;         /* shweno_eq */
  int64_t nx, ny;     /* cells per direction (ny ignored in 1D); each >= 4 */
  double x0, x1;      /* domain [x0, x1] */
  double y0, y1;      /* domain [y0, y1] (2D) */
} shweno_grid;

typedef struct {
  int32_t kind[4];        /* shweno_bc_kind for x-low, x-high, y-low, y-high */
  double inflow[4][4];    /* conserved state of an INFLOW side, by side */
} shweno_bc;

/* Reconstruction options.  Defaults (opts == NULL): nonlinear weights everywhere,
 * eps = 1e-6, linear weights gamma = (0.994, 0.003, 0.003) (Section 2.4), componentwise
 * reconstruction of the conserved variables (the paper's). */
typedef struct {
  int32_t flag_mode;  /* 0: nonlinear weights in every cell; 1: linear weights in every cell;
                         2: per-cell troubled flags (shweno_set_flags) */
  double eps;         /* epsilon of the nonlinear weights */
  double gam[3];      /* linear weights, positive, summing to 1 */
  int32_t charwise;   /* not in the paper.  0: componentwise; 1 (Euler): each reconstruction
                         across a face runs in the characteristic fields of the flux Jacobian
                         along the face normal at the mean of the two adjacent states (1D: the
                         two cell averages; 2D: the two order-0 values of the pass along the
                         face at that point), projected with the left eigenvectors and mapped
                         back with the right ones; no effect for Burgers */
  int32_t quintic;    /* not in the paper's text, which omits the procedure.  0: reading R1, the
                         quartic p1 matching the three cell averages and the outer derivative
                         averages; 1: reading R1', a quintic p1 that also matches the cell's own
                         derivative average (Section 2.4) */
} shweno_opts;

typedef struct shweno_handle shweno_handle;

/* Creates a solver for one mesh on the current CUDA device.  gamma: ratio of specific heats
 * (Euler; ignored for Burgers).  cuda_stream: a cudaStream_t on which every operation of the
 * handle is ordered; NULL makes the handle create its own stream (one that synchronises with the
 * legacy default stream).  The initial state is zero, t = 0.
 * Errors: INVALID (bad grid, BC or options), NOMEM, CUDA. */
shweno_status shweno_create(const shweno_grid* grid, double gamma, const shweno_bc* bc,
                            const shweno_opts* opts, void* cuda_stream, shweno_handle** out);

/* Copies a state in (W, V and, in 2D, Y, Z; each [ncomp][ny][nx]).  on_device = 1: device
 * pointers, 0: host pointers.  Sets the time to t and the step count to 0.
 * Errors: INVALID (null pointer), CUDA. */
shweno_status shweno_set_state(shweno_handle* h, const double* W, const double* V,
                               const double* Y, const double* Z, double t, int on_device);

/* Copies the committed state out (same layouts; Y, Z ignored in 1D).  Synchronises. */
shweno_status shweno_get_state(shweno_handle* h, double* W, double* V, double* Y, double* Z,
                               int on_device);

/* One step of size dt > 0 from the current time (Section 4 Steps 1-5).  Synchronises to check
 * the new state; NONPHYSICAL leaves the state and time of before the step. */
shweno_status shweno_step(shweno_handle* h, double dt);

/* Advances to t_final with dt = cfl / max over cells of the characteristic rate
 * ((|u|+c)/dx + (|v|+c)/dy; Burgers |u| instead of |u|+c), the last step shortened to land on
 * t_final.  The step size is computed and applied on the device (CUDA graph of several steps);
 * the host only polls for completion.  t_out / nsteps_out (may be NULL) receive the final time
 * and the number of steps taken by this call.  NONPHYSICAL: stops at the last good state. */
shweno_status shweno_run(shweno_handle* h, double t_final, double cfl, double* t_out,
                         int64_t* nsteps_out);

/* Enqueues exactly nsteps CFL steps (dt = cfl / rate, no end time) and returns without waiting.
 * Groups of four steps go out as one CUDA graph (captured on first use and kept); the remaining
 * steps, and calls for fewer than four, go out as plain launches.  A non-physical step stops the
 * sequence on the device (the last good state stays committed); the error is reported by the next
 * shweno_sync.  Used for throughput measurement. */
shweno_status shweno_advance(shweno_handle* h, int64_t nsteps, double cfl);

/* Waits for the handle's stream; returns NONPHYSICAL if a step since the last call failed. */
shweno_status shweno_sync(shweno_handle* h);

/* Per-kernel timing (profiling).  While enabled, every step records CUDA events on the handle's
 * stream around each of its kernels (steps are then launched one by one instead of as a graph).
 * shweno_get_timing synchronises, writes the accumulated milliseconds of kernel k to ms[k]
 * (k < max_kernels), the kernel count to *nkernels and the number of timed steps to *nsteps, and
 * clears the totals.  shweno_kernel_name(h, k) names kernel k of the handle's step. */
shweno_status shweno_set_timing(shweno_handle* h, int enable);
shweno_status shweno_get_timing(shweno_handle* h, double* ms, int max_kernels, int* nkernels,
                                int64_t* nsteps);
const char* shweno_kernel_name(const shweno_handle* h, int k);

/* Step size the CFL rule would take now: dt = cfl / rate (rate_out may be NULL). */
shweno_status shweno_cfl_dt(shweno_handle* h, double cfl, double* dt_out, double* rate_out);

/* Current time and committed step count. */
shweno_status shweno_get_time(shweno_handle* h, double* t_out, int64_t* nsteps_out);

/* Per-cell troubled flags for flag_mode 2 ([ny][nx] bytes, nonzero = nonlinear weights;
 * device or host pointer).  A reconstruction anchored on a cell with flag 0 uses the linear
 * weights, which makes it exactly the big-stencil polynomial p1. */
shweno_status shweno_set_flags(shweno_handle* h, const uint8_t* flags, int on_device);

shweno_status shweno_destroy(shweno_handle* h);

/* Message of the last failed call on h ("" if none); h may be NULL for create errors. */
const char* shweno_last_error(const shweno_handle* h);

/* Device allocation hook: every device buffer of every handle created afterwards comes from
 * alloc(bytes, ctx) and goes back through release(ptr, ctx).  NULL restores cudaMalloc/cudaFree.
 * alloc returns NULL on failure (create then fails with NOMEM). */
typedef void* (*shweno_alloc_fn)(size_t bytes, void* ctx);
typedef void (*shweno_free_fn)(void* ptr, void* ctx);
shweno_status shweno_set_allocator(shweno_alloc_fn alloc, shweno_free_fn release, void* ctx);

/* ---------------------------------------------------------------- learned troubled-cell flag
 * Not in the paper: a small network decides per cell whether the reconstructions anchored on it
 * need the nonlinear SHWENO weights (flag 1) or may use the linear weights (flag 0, which makes
 * them exactly the big-stencil quartic p1 of Section 2.4 and skips the smoothness indicators).
 * Network: SHWENO_FLAG_FEATURES inputs -> 32 (ReLU) -> 32 (ReLU) -> 1 (sigmoid), FP32, parameters
 * packed W1[32][22], b1[32], W2[32][32], b2[32], w3[32], b3 (SHWENO_FLAG_PARAMS floats).
 * Features of a cell (2D Euler): for rho and E, the eight 3x3 neighbours minus the centre and
 * dx*V, dy*Y of the centre, each divided by (stencil range + 1e-12 |centre| + 1e-300), and
 * log10(range / (|centre| + 1e-30) + 1e-16) / 8; neighbour order (-1,-1), (0,-1), (1,-1), (-1,0),
 * (1,0), (-1,1), (0,1), (1,1) as (di, dj).  All pointers of this group are device pointers. */
#define SHWENO_FLAG_FEATURES 22
#define SHWENO_FLAG_PARAMS 1825

/* Features of the committed state: out[cells][SHWENO_FLAG_FEATURES] (2D Euler handles). */
shweno_status shweno_flag_features(shweno_handle* h, float* out);

/* Training-label source: per cell, max over its 16 first-pass reconstructions (y-pass on {W,Y}
 * and {V,Z}, x-pass on {W,V} and {Y,Z}, every component) of max_l |w_l - gamma_l| / gamma_l, the
 * relative deviation of the plain scheme's nonlinear weights from the linear ones.  out[cells]. */
shweno_status shweno_weight_deviation(shweno_handle* h, double* out);

/* Training-label source of the face-value form: per cell, the largest change the plain scheme's
 * nonlinear weights make to the end values of those 16 first-pass reconstructions (reading R1),
 *   max over reconstructions and xi = -1/2, +1/2 of |p(xi) - p1(xi)| / (max - min of the
 *   reconstruction's three averages + floor_rel |W0| + 1e-300),
 * with p the SHWENO polynomial and p1 the big-stencil quartic (Section 2.4).  floor_rel >= 1e-9
 * (1e-9: relative to the local range; larger values discount changes that are small against the
 * cell's own average).  out[cells].  Errors: INVALID (floor_rel), STATE (not 2D Euler). */
shweno_status shweno_face_deviation(shweno_handle* h, double floor_rel, double* out);

/* Network on n samples: prob[b] = sigmoid(net(x[b])).  x: [n][SHWENO_FLAG_FEATURES]. */
shweno_status shweno_mlp_forward(const float* params, const float* x, int64_t n, float* prob,
                                 void* cuda_stream);

/* Gradient of the mean weighted binary cross-entropy
 *   L = mean_b( -pos_weight y_b log(sig(z_b)) - (1 - y_b) log(1 - sig(z_b)) ),  y_b in {0, 1},
 * written to grad[SHWENO_FLAG_PARAMS] (overwritten) and L to *loss. */
shweno_status shweno_mlp_grad(const float* params, const float* x, const float* y, int64_t n,
                              float pos_weight, float* grad, float* loss, void* cuda_stream);

/* One Adam step (bias-corrected; step counts from 1) on params with moment buffers m, v. */
shweno_status shweno_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t step,
                              float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* Puts a flag_mode-2 handle in learned mode: from now on every step first evaluates the network
 * on every cell of the committed state, sets flag = (probability > threshold), dilates the flags
 * by one cell (3x3 OR; imposed-state ghost cells count as troubled), then steps with those flags.
 * params: SHWENO_FLAG_PARAMS floats (device if on_device, else host).  Errors: STATE if the
 * handle was not created with flag_mode 2 or is 1D. */
shweno_status shweno_set_flag_net(shweno_handle* h, const float* params, double threshold,
                                  int on_device);

/* Flags used by the last step (after dilation), [ny][nx] bytes. */
shweno_status shweno_get_flags(shweno_handle* h, uint8_t* out, int on_device);

/* ---------------------------------------------------------------- batched launches
 * Not in the paper: many independent problems (existing handles, 1D and 2D mixed, uneven sizes,
 * each with its own CFL time step and end time) advanced together.  Two modes:
 *  - persistent: one persistent kernel, launched from a CUDA graph.  Work items (problem, phase,
 *    index) flow through a device queue; the CTA that finishes a problem's last item of a phase
 *    enqueues the next phase or commits the step.  The only device-side wait is for an empty
 *    queue; it is bounded (about a second by default, shweno_batch_set), after which the run
 *    returns SHWENO_E_TIMEOUT.
 *  - lockstep: rounds of one launch per phase kind over the items of every running problem,
 *    then a commit of every running problem's step (one round = one step of each); the host
 *    reads the running count every 4 rounds.  No device-side wait.  Each CTA does one item, so
 *    the 2D face items run at the one-mesh kernels' register budget without spilling.
 * Both modes run the same items and the same step commit: the same step counts and times, states
 * equal to round-off (the compiler may fuse a product into a multiply-add differently in the two
 * kernels).  Each step is committed on the problem's own control block, so every handle stays
 * usable on its own afterwards.  The handles must outlive the batch and must not be used on their own
 * while a batch run is in flight. */
typedef struct shweno_batch shweno_batch;

/* Run modes (shweno_batch_set_mode).  AUTO: lockstep when every problem is 2D (their items are
 * large enough that a launch per phase costs little), persistent otherwise. */
enum { SHWENO_BATCH_AUTO = 0, SHWENO_BATCH_PERSISTENT = 1, SHWENO_BATCH_LOCKSTEP = 2 };

/* Groups n handles.  cuda_stream: stream of the batch's work (NULL: its own).
 * Errors: INVALID (null or bad handle; a 2D handle created with charwise = 1 or any handle
 * created with quintic = 1, whose items the persistent kernel does not carry), STATE (a
 * per-cell-flag handle without flags or flag network), NOMEM (device memory for the queue and
 * the problem table), CUDA (stream creation or set-up upload failed). */
shweno_status shweno_batch_create(shweno_handle* const* hs, int n, void* cuda_stream,
                                  shweno_batch** out);

/* Advances every problem p to t_final[p] (host array) with dt = cfl / rate, or by at most
 * max_steps steps when max_steps > 0.  per_problem (may be NULL) receives each problem's status
 * (OK, NONPHYSICAL: stopped at its last good state, TIMEOUT).  Returns TIMEOUT if a device-side
 * wait ran out, CUDA on a CUDA error, otherwise OK (even if some problems are NONPHYSICAL). */
shweno_status shweno_batch_run(shweno_batch* b, const double* t_final, double cfl, int64_t max_steps,
                               shweno_status* per_problem);

/* Autotuner: times the candidate launch shapes of the persistent kernel (1D tile of 128..1024
 * cells; 1 or 2 CTAs per SM, or 2..4 when every problem is 1D and the lighter 1D-only kernel
 * runs) on trial_steps steps of the actual problems, restoring every state afterwards, and keeps
 * the fastest; the choice is written to tile1d_out / ctas_per_sm_out (may be NULL).  The mode is
 * left as it is (a lockstep run uses only the 1D tile); a batch of 2D problems in lockstep mode
 * has nothing to tune, and the call returns the current settings without running anything. */
shweno_status shweno_batch_autotune(shweno_batch* b, const double* t_final, double cfl,
                                    int64_t trial_steps, int* tile1d_out, int* ctas_per_sm_out);

/* Sets the launch shape by hand and the bound of the empty-queue wait (values <= 0 keep the
 * current setting).  tile1d: power of 2 in [128, 1024]; ctas_per_sm: 1 or 2 (1..4 for a batch
 * of 1D problems only).  Errors: INVALID (out of range). */
shweno_status shweno_batch_set(shweno_batch* b, int tile1d, int ctas_per_sm, int64_t spin_limit);

/* Sets the run mode (SHWENO_BATCH_AUTO, _PERSISTENT or _LOCKSTEP; the default is AUTO).
 * Errors: INVALID (another value). */
shweno_status shweno_batch_set_mode(shweno_batch* b, int mode);

/* The mode the next run takes (SHWENO_BATCH_PERSISTENT or _LOCKSTEP; -1 for a null batch). */
int shweno_batch_get_mode(const shweno_batch* b);

shweno_status shweno_batch_destroy(shweno_batch* b);
const char* shweno_batch_last_error(const shweno_batch* b);

/* Allocation-free single 1D step.  The paper has no counterpart: this is a convenience for
 * callers that cannot allocate device memory when they step -- real-time loops that cannot take
 * an allocation's latency or the device-wide synchronisation that freeing memory implies, and
 * frameworks that own all device memory through their own pool.  It advances one 1D state by dt
 * with the same kernels as shweno_step, without any allocation: the step's scratch (per-face
 * fluxes and states and the kernels' control block) lives in one fixed __device__ array of
 * 256 bytes + 48 (nx_max + 1) bytes (about 3.1 MB) that every GPU loading this library holds
 * until exit.
 *   eq, nx (4 <= nx <= SHWENO_NOALLOC_MAX_NX), [x0, x1], gamma, bc_kind[2] (x-low, x-high;
 *   PERIODIC, OUTFLOW, REFLECTIVE or INFLOW; periodic on both sides or on neither),
 *   inflow[2][4] (the conserved state of an INFLOW side; may be NULL only when no side is
 *   INFLOW), flag_mode 0 (nonlinear weights in every cell) or 1 (linear weights in every cell);
 *   state_in / state_out: device pointers to [2][ncomp][nx] float64 (W then V), not
 *   overlapping; t: time of state_in; dt > 0; cuda_stream: the stream the work is ordered on.
 * The call waits for the step (it synchronises cuda_stream) and returns NONPHYSICAL if the new
 * state has rho <= 0, p <= 0 or a NaN (state_out then holds that state; state_in is untouched).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it for the process, so it should come before any stream
 * capture, and no call may follow a cudaDeviceReset of that device.  All calls share the one
 * array: calls that overlap on the GPU race.  Sizes beyond the maximum and any other bad
 * argument return INVALID. */
#define SHWENO_NOALLOC_MAX_NX 65536
shweno_status shweno_step1d_noalloc(int32_t eq, int64_t nx, double x0, double x1, double gamma,
                                    const int32_t bc_kind[2], const double inflow[2][4],
                                    int32_t flag_mode, const double* state_in, double* state_out,
                                    double t, double dt, void* cuda_stream);

/* FP64 throughput probe (not part of the scheme): the roofline denominator of the step kernels,
 * which are bound by the FP64 pipe.  Launches one CTA of warps_per_sm (1..32) warps on every SM
 * of the current device, on cuda_stream; each thread runs four independent chains of one FP64
 * operation, op = 0 fused multiply-add, 1 multiply, 2 add, or 3 the three interleaved (two
 * fused chains, one product, one sum), for iters (1..2^24) iterations.  Waits for the launch and
 * writes the rate in TFLOP/s (a fused multiply-add counts 2) to *tflops_out and, if
 * ops_per_clk_per_sm_out is not NULL, the operations per SM clock per SM (from the SM cycle
 * counter of one CTA).  Errors: INVALID (out of range, NULL tflops_out), CUDA. */
shweno_status shweno_fp64_probe(int32_t op, int32_t warps_per_sm, int64_t iters, void* cuda_stream,
                                double* tflops_out, double* ops_per_clk_per_sm_out);

#ifdef __cplusplus
}
#endif

#endif /* SHWENO_H */
