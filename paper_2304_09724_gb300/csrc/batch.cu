// Batched persistent launch: many independent problems of uneven sizes (1D and/or 2D handles),
// each with its own time step and end time, advanced by one persistent kernel.
//
// Work is cut into items (problem, phase, index).  The phases of one step of a problem are
//   1D: tiles of `tile1d` cells (faces of the tile into shared memory, then the tile's update);
//   2D: [flag inference, flag dilation,] first-pass tiles, face segments (x-face Gauss points,
//       corner points and y-face Gauss points), update segments.
// A device queue holds the items that are ready: a ring of slots with published sequence
// numbers; a CTA takes a ticket (atomicAdd on the head) and waits for that slot to be published.
// The CTA that completes the last item of a phase pushes the next phase's items, or, after the
// last phase, commits the step on the problem's own control block (t, step count, CFL rate --
// exactly what end_step/begin_step do for one mesh) and pushes the next step.  Items of a
// problem are never in flight in two phases at once, so no CTA ever waits for another CTA's
// item: the only wait is for an empty queue.  That wait is bounded (spin_limit iterations of
// a short sleep); when it runs out the CTA raises the batch's timeout word and returns, and the
// host reports SHWENO_E_TIMEOUT.  A problem whose step turns non-physical stops at its last
// good state (status NONPHYSICAL) while the others continue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/shweno.h"
#include "flagnet_items.cuh"
#include "shweno_kernels.h"
#include "step1d_items.cuh"
#include "step2d_items.cuh"

namespace shweno {

constexpr int BT = 128;       // threads per CTA of the persistent kernel
constexpr int TYB = 4;        // first-pass tile height in the batch (32 x 4 = 128 cells)
enum { PH_INFER = 0, PH_DILATE = 1, PH_COEF = 2, PH_FACE = 3, PH_UPDATE = 4, PH_TILE1D = 5 };

struct BatchProblem {
  Params P;
  Ctl* ctl;
  double* s0;
  double* s1;
  const uint8_t* flag;
  Scratch2D S;
  const float* net;
  uint8_t* raw;
  uint8_t* flags;
  float logit_thr;
  int32_t nphase;
  int32_t phase_kind[5];
  int32_t nitems[5];
  int32_t tile1d;
  int32_t nsegx, nsegy, ncx, ncy, nsegu, nxitems;
  int64_t max_steps;  // stop after this many committed steps (in this run)
  int64_t step0;      // committed steps at the start of the run
};

struct BatchCtl {
  unsigned long long head;  // next ticket
  unsigned long long tail;  // next free slot
  int active;               // problems still running
  int timeout;              // a wait ran out
};

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kBatchSmem1D = sizeof(double) * 2 * 3 * (1024 + 1);  // F-hat and W(t+dt) of a tile
// the largest item: a face segment, a first-pass tile (16 fields with halo) or a 1D tile
constexpr size_t kBatchSmem = cmax(cmax(kFaceSmem, sizeof(double) * 16 * (TYB + 2) * (TX + 2)), kBatchSmem1D);

__device__ __forceinline__ long long enc(int p, int ph, long long idx) {
  return ((long long)p << 40) | ((long long)ph << 36) | idx;
}

// Reserves n slots and publishes the items (p, phase, 0..n-1).  Called by one thread.
__device__ void push_items(BatchCtl* bc, long long* items, unsigned long long* seq, unsigned long long mask,
                           int p, int ph, int n) {
  const unsigned long long j = atomicAdd(&bc->tail, (unsigned long long)n);
  for (int k = 0; k < n; ++k) items[(j + k) & mask] = enc(p, ph, k);
  __threadfence();
  for (int k = 0; k < n; ++k) atomicExch(&seq[(j + k) & mask], j + k + 1);  // +1: 0 means empty
}

// Start of a step for problem p (begin_step of one mesh): returns false when the problem is done.
__device__ bool begin_problem_step(const BatchProblem& B) {
  volatile Ctl* c = B.ctl;
  if (c->err != ERR_NONE) { c->active = 0; return false; }
  if (c->nsteps - B.step0 >= B.max_steps) { c->active = 0; return false; }
  double dt;
  if (c->mode == 0) {
    dt = c->dt_fixed;
  } else {
    if (!(c->t < c->t_final)) { c->active = 0; return false; }
    const double rate = __longlong_as_double((long long)c->rate_cur);
    dt = c->cfl / rate;
    if (!(dt <= c->t_final - c->t)) dt = c->t_final - c->t;
  }
  c->dt = dt;
  c->rate_next = 0ull;
  c->active = 1;
  return true;
}

// End of a step for problem p (end_step of one mesh): a step that raised an error is not
// committed (the state stays the last good one); otherwise t, the step count and the CFL rate
// advance and the next step begins.  Returns false when the problem is done.
__device__ bool commit_problem_step(const BatchProblem& B) {
  volatile Ctl* c = B.ctl;
  if (c->err != ERR_NONE) {
    c->err_step = c->nsteps;
    c->active = 0;
    return false;
  }
  c->t = c->t + c->dt;
  c->nsteps += 1;
  c->rate_cur = c->rate_next;
  return begin_problem_step(B);
}

// ------------------------------------------------------------------ the work of one item
// HAS2D = false: a batch of 1D problems only; the 2D items are left out of the kernel, which
// then needs about half the registers and runs more CTAs per SM.
template <bool HAS2D>
__device__ __forceinline__ void item_body(const BatchProblem& B, int kind, long long idx, unsigned char* smem) {
  const Params& P = B.P;
  Ctl* ctl = B.ctl;
  const StepView sv = step_view(ctl);
  __shared__ double red[BT / 32];
  if (!HAS2D) kind = PH_TILE1D;
  switch (kind) {
    case PH_TILE1D: {  // 1D: faces of the tile into shared memory, then the cells' update
      const int c0 = (int)idx * B.tile1d;
      const int nc = min(B.tile1d, P.nx - c0);
      double* FH = reinterpret_cast<double*>(smem);
      double* WE = FH + 3 * (B.tile1d + 1);
      const double* st = sv.odd ? B.s1 : B.s0;
      double* out = sv.odd ? B.s0 : B.s1;
      for (int k = threadIdx.x; k <= nc; k += BT) {
        double Fh[3], We[3];
        if (P.ncomp == 1) face1d_point<1, false>(P, st, B.flag, c0 + k, sv.t, sv.dt, Fh, We);
        else face1d_point<3, false>(P, st, B.flag, c0 + k, sv.t, sv.dt, Fh, We);
        for (int q = 0; q < P.ncomp; ++q) { FH[q * (B.tile1d + 1) + k] = Fh[q]; WE[q * (B.tile1d + 1) + k] = We[q]; }
      }
      __syncthreads();
      double rate = 0.0;
      for (int k = threadIdx.x; k < nc; k += BT) {
        const int j = c0 + k;
        double Wn[4];
        for (int q = 0; q < P.ncomp; ++q) {
          const int fo = q * (B.tile1d + 1) + k;
          Wn[q] = __ldcg(st + (size_t)q * P.nx + j) - sv.dt / P.dx * (FH[fo + 1] - FH[fo]);
          out[(size_t)q * P.nx + j] = Wn[q];
          out[(size_t)(P.ncomp + q) * P.nx + j] = (WE[fo + 1] - WE[fo]) * P.idx;
        }
        if (!cell_physical(P, Wn)) atomicCAS(&ctl->err, ERR_NONE, ERR_NONPHYSICAL);
        else rate = fmax(rate, cell_rate(P, Wn));
      }
      block_max_rate(rate, &ctl->rate_next, red);
      break;
    }
  }
  if constexpr (HAS2D) switch (kind) {
    case PH_INFER: {
      float* p = reinterpret_cast<float*>(smem);
      load_params(B.net, p);
      const size_t c = (size_t)idx * BT + threadIdx.x;
      if (c < (size_t)P.nx * P.ny) {
        const double* st = sv.odd ? B.s1 : B.s0;
        float f[NIN];
        cell_features(P, st, (int)(c % P.nx), (int)(c / P.nx), sv.t, f);
        B.raw[c] = net_logit(p, f) > B.logit_thr ? 1 : 0;
      }
      break;
    }
    case PH_DILATE: {
      const size_t c = (size_t)idx * BT + threadIdx.x;
      if (c < (size_t)P.nx * P.ny) {
        const int i = (int)(c % P.nx), j = (int)(c / P.nx);
        int f = 0;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) f |= raw_flag(P, B.raw, i + di, j + dj);
        B.flags[c] = (uint8_t)f;
      }
      break;
    }
    case PH_COEF: {
      const int bxi = (int)(idx % B.ncx), byi = (int)(idx / B.ncx);
      auto tile = reinterpret_cast<double(*)[TYB + 2][TX + 2]>(smem);
      if (P.ncomp == 1)
        coef2d_item<1, TYB>(P, sv, B.s0, B.s1, B.flag, B.S.ycoef, B.S.xcoef, bxi * TX - 2, byi * TYB - 2,
                            tile, threadIdx.x % TX, threadIdx.x / TX);
      else
        coef2d_item<4, TYB>(P, sv, B.s0, B.s1, B.flag, B.S.ycoef, B.S.xcoef, bxi * TX - 2, byi * TYB - 2,
                            tile, threadIdx.x % TX, threadIdx.x / TX);
      break;
    }
    case PH_FACE: {
      const bool flags = P.flag_mode != FLAG_ALL_NONLINEAR;
      if (idx < B.nxitems) {
        const int seg = (int)(idx % B.nsegx), r = (int)(idx / B.nsegx);
        const int slice = r < 3 * P.ny ? r / P.ny : 3;
        const int row = r < 3 * P.ny ? r % P.ny : r - 3 * P.ny;
        const int f0 = seg * NFACE;
        if (P.ncomp == 1) {
          if (flags) xface_item<1, true>(P, sv, sv.odd ? B.s1 : B.s0, B.S.ycoef, B.flag, B.S.FX, B.S.WX, B.S.WC, f0, row, slice, smem);
          else xface_item<1, false>(P, sv, sv.odd ? B.s1 : B.s0, B.S.ycoef, B.flag, B.S.FX, B.S.WX, B.S.WC, f0, row, slice, smem);
        } else {
          if (flags) xface_item<4, true>(P, sv, sv.odd ? B.s1 : B.s0, B.S.ycoef, B.flag, B.S.FX, B.S.WX, B.S.WC, f0, row, slice, smem);
          else xface_item<4, false>(P, sv, sv.odd ? B.s1 : B.s0, B.S.ycoef, B.flag, B.S.FX, B.S.WX, B.S.WC, f0, row, slice, smem);
        }
      } else {
        const long long k = idx - B.nxitems;
        const int seg = (int)(k % B.nsegy), r = (int)(k / B.nsegy);
        const int slice = r / P.nx, col = r % P.nx;
        const int f0 = seg * NFACE;
        if (P.ncomp == 1) {
          if (flags) yface_item<1, true>(P, sv, sv.odd ? B.s1 : B.s0, B.S.xcoef, B.flag, B.S.FY, B.S.WY, f0, col, slice, smem);
          else yface_item<1, false>(P, sv, sv.odd ? B.s1 : B.s0, B.S.xcoef, B.flag, B.S.FY, B.S.WY, f0, col, slice, smem);
        } else {
          if (flags) yface_item<4, true>(P, sv, sv.odd ? B.s1 : B.s0, B.S.xcoef, B.flag, B.S.FY, B.S.WY, f0, col, slice, smem);
          else yface_item<4, false>(P, sv, sv.odd ? B.s1 : B.s0, B.S.xcoef, B.flag, B.S.FY, B.S.WY, f0, col, slice, smem);
        }
      }
      break;
    }
    case PH_UPDATE: {
      const int seg = (int)(idx % B.nsegu), j = (int)(idx / B.nsegu);
      const int i = seg * BT + threadIdx.x;
      double rate = 0.0;
      if (i < P.nx) {
        const double* st = sv.odd ? B.s1 : B.s0;
        double* out = sv.odd ? B.s0 : B.s1;
        rate = P.ncomp == 1
                   ? update2d_cell<1>(P, ctl, sv, st, out, B.S.FX, B.S.WX, B.S.FY, B.S.WY, B.S.WC, i, j)
                   : update2d_cell<4>(P, ctl, sv, st, out, B.S.FX, B.S.WX, B.S.FY, B.S.WY, B.S.WC, i, j);
      }
      block_max_rate(rate, &ctl->rate_next, red);
      break;
    }
  }
}

// The persistent kernel's call (left to the compiler's inlining choice: forcing it makes the
// kernel spill far more).
template <bool HAS2D>
__device__ void do_item(const BatchProblem& B, int kind, long long idx, unsigned char* smem) {
  item_body<HAS2D>(B, kind, idx, smem);
}

// ------------------------------------------------------------------ persistent kernel
template <bool HAS2D>
__global__ void __launch_bounds__(BT, HAS2D ? 1 : 4) batch_kernel(const BatchProblem* __restrict__ probs, int* pstate,
                                                   BatchCtl* bc, long long* items, unsigned long long* seq,
                                                   unsigned long long mask, long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_state;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long ticket = atomicAdd(&bc->head, 1ull);
      volatile unsigned long long* vs = seq;
      volatile int* vb = &bc->active;
      volatile int* vt = &bc->timeout;
      long long spins = 0;
      int state = 0;
      for (;;) {
        if (vs[ticket & mask] == ticket + 1) {
          __threadfence();
          s_item = __ldcg(&items[ticket & mask]);
          state = 1;
          break;
        }
        if (*vb == 0 || *vt != 0) { state = 2; break; }
        if (++spins > spin_limit) { atomicExch(&bc->timeout, 1); state = 2; break; }
        __nanosleep(256);
      }
      s_state = state;
    }
    __syncthreads();
    if (s_state != 1) return;
    const long long item = s_item;
    const int p = (int)(item >> 40), ph = (int)((item >> 36) & 15);
    const long long idx = item & ((1ll << 36) - 1);
    const BatchProblem& B = probs[p];
    do_item<HAS2D>(B, B.phase_kind[ph], idx, smem);
    __threadfence();  // this thread's results visible device-wide before the item counts as done
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const int done = atomicAdd(&pstate[p], 1) + 1;
      if (done == B.nitems[ph]) {
        pstate[p] = 0;
        __threadfence();
        int next = ph + 1;
        if (next == B.nphase) {  // end of the step: commit (end_step) and start the next one
          const bool go = commit_problem_step(B);
          next = 0;
          if (!go) {
            __threadfence();
            atomicSub(&bc->active, 1);
            next = -1;
          }
        }
        if (next >= 0) push_items(bc, items, seq, mask, p, next, B.nitems[next]);
      }
    }
    __syncthreads();
  }
}

// Seeds the queue: first step of every problem (rates are already in rate_cur).
__global__ void batch_seed_kernel(const BatchProblem* __restrict__ probs, int n, BatchCtl* bc,
                                  long long* items, unsigned long long* seq, unsigned long long mask) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const BatchProblem& B = probs[p];
  if (begin_problem_step(B)) push_items(bc, items, seq, mask, p, 0, B.nitems[0]);
  else atomicSub(&bc->active, 1);
}

__global__ void batch_reset_kernel(BatchCtl* bc, int n, unsigned long long* seq, unsigned long long cap,
                                   int* pstate) {
  const unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < cap) seq[k] = 0ull;
  if (k < (unsigned long long)n) pstate[k] = 0;
  if (k == 0) { bc->head = 0; bc->tail = 0; bc->active = n; bc->timeout = 0; }
}

// Per-problem CFL rate of the committed state: blocks over (problem, chunk of cells).
__global__ void batch_rate_kernel(const BatchProblem* __restrict__ probs, const int* chunk0, int n) {
  __shared__ double red[32];
  // find the problem of this block: chunk0 is the prefix sum of chunks per problem
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (chunk0[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
  }
  const BatchProblem& B = probs[lo];
  const Params& P = B.P;
  const size_t cells = (size_t)P.nx * P.ny;
  const size_t c = (size_t)(blockIdx.x - chunk0[lo]) * blockDim.x + threadIdx.x;
  const double* st = (B.ctl->nsteps & 1) ? B.s1 : B.s0;
  double r = 0.0;
  if (c < cells) {
    double W[4];
    for (int q = 0; q < P.ncomp; ++q) W[q] = st[q * cells + c];
    if (!cell_physical(P, W)) atomicCAS(&B.ctl->err, ERR_NONE, ERR_NONPHYSICAL);
    else r = cell_rate(P, W);
  }
  block_max_rate(r, &B.ctl->rate_cur, red);
}

__global__ void batch_config_kernel(const BatchProblem* __restrict__ probs, int n, const double* t_final,
                                    double cfl) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  volatile Ctl* c = probs[p].ctl;
  c->mode = 1;
  c->t_final = t_final[p];
  c->cfl = cfl;
  c->err = ERR_NONE;
  c->active = 0;
  c->rate_cur = 0ull;
}

// ------------------------------------------------------------------ lockstep launches
// The other way to run a batch: rounds of one launch per phase kind over the items of every
// problem still running, then one thread per problem commits its step and begins the next (one
// round = one step of every running problem).  Block b of the launch of kind k does item
// b - start[p] of the problem p with start[p] <= b < start[p + 1] (start: prefix sums of the
// problems' item counts of that kind).  Each CTA does one item and exits, so the face item
// compiles as in the one-mesh kernels; in the persistent kernel's loop it does not fit in 255
// registers and spills.  Items, step commit and step begin are the persistent kernel's, so the
// two modes take the same steps; their states agree to round-off (the same functions inlined
// into different kernels may contract a product into a fused multiply-add differently).
constexpr int kLockKinds[] = {PH_INFER, PH_DILATE, PH_COEF, PH_FACE, PH_UPDATE, PH_TILE1D};
constexpr int kNumLockKinds = 6;

template <int KIND>
__global__ void __launch_bounds__(BT) lockstep_kernel(const BatchProblem* __restrict__ probs,
                                                      const int* __restrict__ start, int n) {
  extern __shared__ __align__(16) unsigned char smem[];
  int lo = 0, hi = n;  // the last problem whose first block is at or before this one
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= (int)blockIdx.x) lo = mid;
    else hi = mid;
  }
  const BatchProblem& B = probs[lo];
  if (!((const volatile Ctl*)B.ctl)->active) return;  // done, or stopped: its blocks idle
  item_body<true>(B, KIND, (long long)blockIdx.x - __ldg(start + lo), smem);
}

// One thread per problem: commits the round's step of every running problem and counts the
// problems that go on (bc->active, zeroed before the launch).
__global__ void lockstep_commit_kernel(const BatchProblem* __restrict__ probs, int n, BatchCtl* bc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const BatchProblem& B = probs[p];
  if (!((const volatile Ctl*)B.ctl)->active) return;
  if (commit_problem_step(B)) atomicAdd(&bc->active, 1);
}

// First step of every problem in lockstep mode (rates are already in rate_cur).
__global__ void lockstep_seed_kernel(const BatchProblem* __restrict__ probs, int n, BatchCtl* bc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (begin_problem_step(probs[p])) atomicAdd(&bc->active, 1);
}

}  // namespace shweno

// ======================================================================== host side
struct shweno_handle;
namespace shweno {
bool handle_view(shweno_handle* h, HandleView* v);  // api.cu
}  // namespace shweno

struct shweno_batch {
  std::vector<shweno::HandleView> views;
  std::vector<shweno::BatchProblem> host_probs;
  shweno::BatchProblem* probs = nullptr;
  int* pstate = nullptr;
  shweno::BatchCtl* bc = nullptr;
  long long* items = nullptr;
  unsigned long long* seq = nullptr;
  unsigned long long cap = 0;
  int* chunk0 = nullptr;
  int nchunks = 0;
  double* t_final = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int tile1d = 512;
  int ctas_per_sm = 2;
  bool has2d = true;  // false: every problem is 1D (the lighter kernel, up to 4 CTAs per SM)
  int grid = 0;
  long long spin_limit = 4000000;  // x ~256 ns sleeps: about a second
  std::string err;
  cudaGraphExec_t graph = nullptr;
  std::vector<double> tuned;  // autotuner timings (ms) per candidate
  int mode = SHWENO_BATCH_AUTO;  // SHWENO_BATCH_AUTO / _PERSISTENT / _LOCKSTEP
  int* lstart = nullptr;         // lockstep block tables: [kind][problem + 1] prefix sums
  std::vector<int> lstart_host;
  int ltotal[shweno::kNumLockKinds] = {};
};

namespace {

shweno_status bfail(shweno_batch* b, shweno_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

void fill_problem(shweno_batch* b, int p) {
  using namespace shweno;
  const HandleView& v = b->views[p];
  BatchProblem& B = b->host_probs[p];
  std::memset(&B, 0, sizeof(B));
  B.P = v.P;
  B.ctl = v.ctl;
  B.s0 = v.buf[0];
  B.s1 = v.buf[1];
  B.flag = v.learned ? v.flags_out : v.flags;
  B.S = v.S;
  B.net = v.net;
  B.raw = v.raw;
  B.flags = v.flags_out;
  B.logit_thr = v.logit_thr;
  B.max_steps = INT64_MAX;
  if (v.P.dim == 1) {
    B.tile1d = b->tile1d;
    B.nphase = 1;
    B.phase_kind[0] = PH_TILE1D;
    B.nitems[0] = (v.P.nx + b->tile1d - 1) / b->tile1d;
  } else {
    const int nx = v.P.nx, ny = v.P.ny;
    const int cells_items = (int)(((size_t)nx * ny + BT - 1) / BT);
    B.ncx = (nx + 4 + TX - 1) / TX;
    B.ncy = (ny + 4 + TYB - 1) / TYB;
    B.nsegx = (nx + 1 + NFACE - 1) / NFACE;
    B.nsegy = (ny + 1 + NFACE - 1) / NFACE;
    B.nsegu = (nx + BT - 1) / BT;
    B.nxitems = B.nsegx * (3 * ny + ny + 1);
    int k = 0;
    if (v.learned) {
      B.phase_kind[k] = PH_INFER; B.nitems[k++] = cells_items;
      B.phase_kind[k] = PH_DILATE; B.nitems[k++] = cells_items;
    }
    B.phase_kind[k] = PH_COEF; B.nitems[k++] = B.ncx * B.ncy;
    B.phase_kind[k] = PH_FACE; B.nitems[k++] = B.nxitems + B.nsegy * nx * 3;
    B.phase_kind[k] = PH_UPDATE; B.nitems[k++] = B.nsegu * ny;
    B.nphase = k;
  }
}

}  // namespace

extern "C" {

shweno_status shweno_batch_create(shweno_handle* const* hs, int n, void* cuda_stream, shweno_batch** out) {
  using namespace shweno;
  if (!hs || n <= 0 || !out || n >= (1 << 23)) return SHWENO_E_INVALID;
  *out = nullptr;
  shweno_batch* b = new shweno_batch();
  b->views.resize(n);
  b->host_probs.resize(n);
  size_t cap_need = 0;
  for (int p = 0; p < n; ++p) {
    if (!hs[p] || !handle_view(hs[p], &b->views[p])) { delete b; return SHWENO_E_INVALID; }
    // the persistent kernel carries reading R1 and the componentwise 2D face items only
    if ((b->views[p].P.dim == 2 && b->views[p].P.charwise) || b->views[p].P.quintic) {
      delete b;
      return SHWENO_E_INVALID;
    }
    if (b->views[p].P.flag_mode == FLAG_PER_CELL && !b->views[p].flags && !b->views[p].learned) {
      delete b;
      return SHWENO_E_STATE;
    }
  }
  b->has2d = false;
  for (int p = 0; p < n; ++p) b->has2d |= b->views[p].P.dim == 2;
  if (!b->has2d) b->ctas_per_sm = 4;
  if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
  else {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      cudaGetLastError();
      b->stream = nullptr;
      delete b;
      return SHWENO_E_CUDA;
    }
    b->own_stream = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = sms * b->ctas_per_sm;
  // chunks of the rate kernel
  std::vector<int> ch(n);
  int acc = 0;
  for (int p = 0; p < n; ++p) {
    ch[p] = acc;
    acc += (int)(((size_t)b->views[p].P.nx * b->views[p].P.ny + 255) / 256);
  }
  b->nchunks = acc;
  // queue capacity: the largest phase of every problem in flight at once, plus one ticket per CTA
  for (int p = 0; p < n; ++p) {
    fill_problem(b, p);
    int mx = 0;
    for (int k = 0; k < b->host_probs[p].nphase; ++k) mx = std::max(mx, b->host_probs[p].nitems[k]);
    // 1D problems may be re-tiled by the autotuner down to 128 cells per item
    if (b->views[p].P.dim == 1) mx = std::max(mx, (b->views[p].P.nx + 127) / 128);
    cap_need += mx;
  }
  cap_need += 4 * (size_t)sms * 8 + 1;
  b->cap = 1;
  while (b->cap < cap_need) b->cap <<= 1;
  bool ok = cudaMalloc(&b->probs, n * sizeof(BatchProblem)) == cudaSuccess &&
            cudaMalloc(&b->pstate, n * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->bc, sizeof(BatchCtl)) == cudaSuccess &&
            cudaMalloc(&b->items, b->cap * sizeof(long long)) == cudaSuccess &&
            cudaMalloc(&b->seq, b->cap * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&b->chunk0, n * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->t_final, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->lstart, (size_t)kNumLockKinds * (n + 1) * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    shweno_batch_destroy(b);
    return SHWENO_E_NOMEM;
  }
  if (cudaMemcpy(b->chunk0, ch.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaFuncSetAttribute(batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) != cudaSuccess ||
      cudaFuncSetAttribute(batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem1D) != cudaSuccess ||
      cudaFuncSetAttribute(lockstep_kernel<PH_FACE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFaceSmem) != cudaSuccess ||
      cudaFuncSetAttribute(lockstep_kernel<PH_TILE1D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem1D) != cudaSuccess) {
    cudaGetLastError();
    shweno_batch_destroy(b);
    return SHWENO_E_CUDA;
  }
  *out = b;
  return SHWENO_OK;
}

shweno_status shweno_batch_destroy(shweno_batch* b) {
  if (!b) return SHWENO_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->probs);
  cudaFree(b->pstate);
  cudaFree(b->bc);
  cudaFree(b->items);
  cudaFree(b->seq);
  cudaFree(b->chunk0);
  cudaFree(b->t_final);
  cudaFree(b->lstart);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return SHWENO_OK;
}

const char* shweno_batch_last_error(const shweno_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

namespace {

// Enqueues one batch run (config, rates, seed, persistent kernel) on b->stream.
void enqueue_batch(shweno_batch* b, double cfl) {
  using namespace shweno;
  const int n = (int)b->views.size();
  const unsigned long long cap = b->cap;
  batch_config_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(b->probs, n, b->t_final, cfl);
  batch_reset_kernel<<<(unsigned)((std::max<unsigned long long>(cap, n) + 255) / 256), 256, 0, b->stream>>>(
      b->bc, n, b->seq, cap, b->pstate);
  batch_rate_kernel<<<b->nchunks, 256, 0, b->stream>>>(b->probs, b->chunk0, n);
  batch_seed_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(b->probs, n, b->bc, b->items, b->seq, cap - 1);
  if (b->has2d)
    batch_kernel<true><<<b->grid, BT, kBatchSmem, b->stream>>>(b->probs, b->pstate, b->bc, b->items, b->seq,
                                                               cap - 1, b->spin_limit);
  else
    batch_kernel<false><<<b->grid, BT, kBatchSmem1D, b->stream>>>(b->probs, b->pstate, b->bc, b->items, b->seq,
                                                                  cap - 1, b->spin_limit);
}

// Problem table, start step counts and end times of one run, uploaded on b->stream.
shweno_status prepare_run(shweno_batch* b, const double* t_final, int64_t max_steps) {
  using namespace shweno;
  const int n = (int)b->views.size();
  for (int p = 0; p < n; ++p) {
    fill_problem(b, p);
    b->host_probs[p].max_steps = max_steps > 0 ? max_steps : INT64_MAX;
  }
  // step counts at the start (for max_steps)
  std::vector<Ctl> ctl(n);
  for (int p = 0; p < n; ++p)
    if (cudaMemcpyAsync(&ctl[p], b->views[p].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return bfail(b, SHWENO_E_CUDA, "reading a control block failed");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, SHWENO_E_CUDA, "stream sync failed");
  for (int p = 0; p < n; ++p) b->host_probs[p].step0 = ctl[p].nsteps;
  if (cudaMemcpyAsync(b->probs, b->host_probs.data(), n * sizeof(BatchProblem), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->t_final, t_final, n * sizeof(double), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return bfail(b, SHWENO_E_CUDA, "upload failed");
  return SHWENO_OK;
}

// One persistent-kernel run (from the cached graph when `graph`).
shweno_status run_once(shweno_batch* b, const double* t_final, double cfl, int64_t max_steps, bool graph) {
  using namespace shweno;
  const shweno_status ps = prepare_run(b, t_final, max_steps);
  if (ps != SHWENO_OK) return ps;
  if (graph) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(b, SHWENO_E_CUDA, "capture failed");
      enqueue_batch(b, cfl);
      if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess) return bfail(b, SHWENO_E_CUDA, "capture failed");
      cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(b, SHWENO_E_CUDA, "graph instantiation failed");
    }
    if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return bfail(b, SHWENO_E_CUDA, "graph launch failed");
  } else {
    enqueue_batch(b, cfl);
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, SHWENO_E_CUDA, std::string("batch kernel: ") + cudaGetErrorString(e));
  BatchCtl bc;
  if (cudaMemcpy(&bc, b->bc, sizeof(BatchCtl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, SHWENO_E_CUDA, "reading the batch control failed");
  if (bc.timeout) return bfail(b, SHWENO_E_TIMEOUT, "a device-side wait of the batch ran out");
  return SHWENO_OK;
}

// Dynamic shared memory of a lockstep launch of one kind.
size_t lock_smem(const shweno_batch* b, int kind) {
  using namespace shweno;
  switch (kind) {
    case PH_INFER: return sizeof(float) * NPARAM;
    case PH_COEF: return sizeof(double) * 16 * (TYB + 2) * (TX + 2);
    case PH_FACE: return kFaceSmem;
    case PH_TILE1D: return sizeof(double) * 2 * 3 * (b->tile1d + 1);
    default: return 0;
  }
}

void launch_lock(shweno_batch* b, int kind, const int* start, int grid) {
  using namespace shweno;
  const int n = (int)b->views.size();
  const size_t sm = lock_smem(b, kind);
  switch (kind) {
    case PH_INFER: lockstep_kernel<PH_INFER><<<grid, BT, sm, b->stream>>>(b->probs, start, n); break;
    case PH_DILATE: lockstep_kernel<PH_DILATE><<<grid, BT, sm, b->stream>>>(b->probs, start, n); break;
    case PH_COEF: lockstep_kernel<PH_COEF><<<grid, BT, sm, b->stream>>>(b->probs, start, n); break;
    case PH_FACE: lockstep_kernel<PH_FACE><<<grid, BT, sm, b->stream>>>(b->probs, start, n); break;
    case PH_UPDATE: lockstep_kernel<PH_UPDATE><<<grid, BT, sm, b->stream>>>(b->probs, start, n); break;
    default: lockstep_kernel<PH_TILE1D><<<grid, BT, sm, b->stream>>>(b->probs, start, n); break;
  }
}

// One lockstep run: rates and first steps, then rounds of (one launch per phase kind with work,
// the commit) until no problem runs, reading the running count back every few rounds.
shweno_status run_lockstep(shweno_batch* b, const double* t_final, double cfl, int64_t max_steps) {
  using namespace shweno;
  const shweno_status ps = prepare_run(b, t_final, max_steps);
  if (ps != SHWENO_OK) return ps;
  const int n = (int)b->views.size();
  // block tables: start[k][p] = first block of problem p in the launch of kind k
  b->lstart_host.assign((size_t)kNumLockKinds * (n + 1), 0);
  for (int k = 0; k < kNumLockKinds; ++k) {
    long long acc = 0;
    for (int p = 0; p < n; ++p) {
      b->lstart_host[(size_t)k * (n + 1) + p] = (int)acc;
      const BatchProblem& B = b->host_probs[p];
      for (int f = 0; f < B.nphase; ++f)
        if (B.phase_kind[f] == kLockKinds[k]) acc += B.nitems[f];
      if (acc > INT32_MAX) return bfail(b, SHWENO_E_INVALID, "too many items for one lockstep launch");
    }
    b->lstart_host[(size_t)k * (n + 1) + n] = (int)acc;
    b->ltotal[k] = (int)acc;
  }
  if (cudaMemcpyAsync(b->lstart, b->lstart_host.data(), b->lstart_host.size() * sizeof(int), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess)
    return bfail(b, SHWENO_E_CUDA, "upload failed");
  int* active = &b->bc->active;
  batch_config_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(b->probs, n, b->t_final, cfl);
  batch_rate_kernel<<<b->nchunks, 256, 0, b->stream>>>(b->probs, b->chunk0, n);
  cudaMemsetAsync(b->bc, 0, sizeof(BatchCtl), b->stream);
  lockstep_seed_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(b->probs, n, b->bc);
  const int kChunk = 4;  // rounds between two reads of the running count
  int64_t rounds = 0;
  for (;;) {
    int running = 0;
    if (cudaMemcpyAsync(&running, active, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return bfail(b, SHWENO_E_CUDA, "reading the running count failed");
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SHWENO_E_CUDA, std::string("lockstep round: ") + cudaGetErrorString(e));
    if (running == 0 || (max_steps > 0 && rounds >= max_steps)) break;
    int64_t r = kChunk;
    if (max_steps > 0) r = std::min<int64_t>(r, max_steps - rounds);
    for (int64_t i = 0; i < r; ++i) {
      for (int k = 0; k < kNumLockKinds; ++k)
        if (b->ltotal[k] > 0) launch_lock(b, kLockKinds[k], b->lstart + (size_t)k * (n + 1), b->ltotal[k]);
      cudaMemsetAsync(active, 0, sizeof(int), b->stream);
      lockstep_commit_kernel<<<(n + 127) / 128, 128, 0, b->stream>>>(b->probs, n, b->bc);
    }
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return bfail(b, SHWENO_E_CUDA, std::string("lockstep launch: ") + cudaGetErrorString(le));
    rounds += r;
  }
  return SHWENO_OK;
}

// The mode a run takes: lockstep when set, or in auto mode when every problem is 2D.
bool use_lockstep(const shweno_batch* b) {
  if (b->mode == SHWENO_BATCH_LOCKSTEP) return true;
  if (b->mode == SHWENO_BATCH_PERSISTENT) return false;
  for (const auto& v : b->views)
    if (v.P.dim != 2) return false;
  return true;
}

}  // namespace

extern "C" {

shweno_status shweno_batch_run(shweno_batch* b, const double* t_final, double cfl, int64_t max_steps,
                               shweno_status* per_problem) {
  using namespace shweno;
  if (!b || !t_final || !(cfl > 0.0)) return bfail(b, SHWENO_E_INVALID, "invalid argument");
  const int n = (int)b->views.size();
  // the cached graph bakes in the cfl; rebuild when it changes
  static thread_local double last_cfl = -1.0;
  if (b->graph && cfl != last_cfl) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  last_cfl = cfl;
  shweno_status s = use_lockstep(b) ? run_lockstep(b, t_final, cfl, max_steps)
                                    : run_once(b, t_final, cfl, max_steps, max_steps <= 0);
  if (per_problem) {
    for (int p = 0; p < n; ++p) {
      Ctl c;
      if (cudaMemcpy(&c, b->views[p].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) {
        per_problem[p] = SHWENO_E_CUDA;
        continue;
      }
      per_problem[p] = c.err == ERR_NONPHYSICAL ? SHWENO_E_NONPHYSICAL : (s == SHWENO_E_TIMEOUT && c.t < t_final[p] ? SHWENO_E_TIMEOUT : SHWENO_OK);
    }
  }
  return s;
}

// Autotuner: times each candidate (1D tile size, CTAs per SM) on a bounded number of steps of
// the actual problems, restoring every problem's state and control block after each trial, and
// keeps the fastest.  Returns the choice through tile1d / ctas_per_sm.
shweno_status shweno_batch_autotune(shweno_batch* b, const double* t_final, double cfl, int64_t trial_steps,
                                    int* tile1d_out, int* ctas_per_sm_out) {
  using namespace shweno;
  if (!b || !t_final || trial_steps <= 0) return bfail(b, SHWENO_E_INVALID, "invalid argument");
  const int n = (int)b->views.size();
  bool any1d = false;
  for (auto& v : b->views) any1d |= v.P.dim == 1;
  if (!any1d && use_lockstep(b)) {  // lockstep rounds of 2D problems have no launch shape to tune
    b->tuned.clear();
    if (tile1d_out) *tile1d_out = b->tile1d;
    if (ctas_per_sm_out) *ctas_per_sm_out = b->ctas_per_sm;
    return SHWENO_OK;
  }
  // backups of the states and control blocks
  std::vector<double*> bk(n, nullptr);
  std::vector<Ctl> cbk(n);
  for (int p = 0; p < n; ++p) {
    const auto& P = b->views[p].P;
    const size_t d = (size_t)(P.dim == 2 ? 4 : 2) * P.ncomp * P.nx * P.ny;
    if (cudaMalloc(&bk[p], 2 * d * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      for (double* q : bk) cudaFree(q);
      return bfail(b, SHWENO_E_NOMEM, "no room for the autotuner's backups");
    }
    cudaMemcpyAsync(bk[p], b->views[p].buf[0], d * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(bk[p] + d, b->views[p].buf[1], d * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(&cbk[p], b->views[p].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream);
  }
  cudaStreamSynchronize(b->stream);
  auto restore = [&]() {
    for (int p = 0; p < n; ++p) {
      const auto& P = b->views[p].P;
      const size_t d = (size_t)(P.dim == 2 ? 4 : 2) * P.ncomp * P.nx * P.ny;
      cudaMemcpyAsync(b->views[p].buf[0], bk[p], d * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
      cudaMemcpyAsync(b->views[p].buf[1], bk[p] + d, d * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
      cudaMemcpyAsync(b->views[p].ctl, &cbk[p], sizeof(Ctl), cudaMemcpyHostToDevice, b->stream);
    }
    cudaStreamSynchronize(b->stream);
  };
  std::vector<int> tiles = any1d ? std::vector<int>{128, 256, 512, 1024} : std::vector<int>{b->tile1d};
  std::vector<int> occ = b->has2d ? std::vector<int>{1, 2} : std::vector<int>{2, 3, 4};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int bt = b->tile1d, bo = b->ctas_per_sm;
  b->tuned.clear();
  shweno_status st = SHWENO_OK;
  for (int t : tiles) {
    for (int o : occ) {
      b->tile1d = t;
      b->ctas_per_sm = o;
      b->grid = sms * o;
      cudaEventRecord(e0, b->stream);
      st = run_once(b, t_final, cfl, trial_steps, false);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      restore();
      b->tuned.push_back(ms);
      if (st != SHWENO_OK) break;
      if (ms < best) { best = ms; bt = t; bo = o; }
    }
    if (st != SHWENO_OK) break;  // a failed trial ends the search; the states are restored
  }
  b->tile1d = bt;
  b->ctas_per_sm = bo;
  b->grid = sms * bo;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  for (double* q : bk) cudaFree(q);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tile1d_out) *tile1d_out = bt;
  if (ctas_per_sm_out) *ctas_per_sm_out = bo;
  return st;
}

shweno_status shweno_batch_set(shweno_batch* b, int tile1d, int ctas_per_sm, int64_t spin_limit) {
  if (!b) return SHWENO_E_INVALID;
  if (tile1d > 0) {
    if (tile1d < 128 || tile1d > 1024 || (tile1d & (tile1d - 1))) return bfail(b, SHWENO_E_INVALID, "tile1d must be 128..1024, a power of 2");
    b->tile1d = tile1d;
  }
  if (ctas_per_sm > 0) {
    if (ctas_per_sm > (b->has2d ? 2 : 4))
      return bfail(b, SHWENO_E_INVALID, "ctas_per_sm must be 1..2 (1..4 for a batch of 1D problems)");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->ctas_per_sm = ctas_per_sm;
    b->grid = sms * ctas_per_sm;
  }
  if (spin_limit > 0) b->spin_limit = spin_limit;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return SHWENO_OK;
}

shweno_status shweno_batch_set_mode(shweno_batch* b, int mode) {
  if (!b) return SHWENO_E_INVALID;
  if (mode != SHWENO_BATCH_AUTO && mode != SHWENO_BATCH_PERSISTENT && mode != SHWENO_BATCH_LOCKSTEP)
    return bfail(b, SHWENO_E_INVALID, "mode must be SHWENO_BATCH_AUTO, _PERSISTENT or _LOCKSTEP");
  b->mode = mode;
  return SHWENO_OK;
}

int shweno_batch_get_mode(const shweno_batch* b) {
  if (!b) return -1;
  return use_lockstep(b) ? SHWENO_BATCH_LOCKSTEP : SHWENO_BATCH_PERSISTENT;
}

}  // extern "C"
