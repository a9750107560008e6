// mqo_step.cuh -- the fused descent step (one tick of gradient work): the
// arguments, the per-element tail and the counter flush shared by the two
// step kernels (mqo_step.cu: shared-memory staged; mqo_step_generic.cu:
// global-memory gathers).
//
// For every node v and trajectory b of a stepping trajectory:
//   (A x)_vb  = sum over the CSR row of v, in row order, of w_vu x_ub (float32)
//   grad      = 1 - gamma (A x)_vb              (h, Eq. 3)
//             | -lambda - 2 (A x)_vb            (f_B, Eq. 7)
//             | or the gradient of f_L, f_P, f_A (Sec. 3), selected by
//               `objective`; f_L and f_P also use the weighted degree d_v
//   V'        = mu V + alpha grad               (momentum ascent, Sec. 5)
//   x'        = Pi_box(x + V')                  (projection of Sec. 3)
// and, from the same neighbour gather, the exact evaluation of the rounded
// incoming point z = [x > 0.5] (MIS) or [x > 0] (MaxCut): set size,
// conflicting and uncovered nodes (checker, Eq. 8), or cut,
// nodes violating the fixed-point condition of the selected relaxation and
// positive-gain nodes.
// The rounding of x' is written next to x' (ZX), so the next step and the
// acceptance of this step's point read it without recomputing.
//
// Thread mapping: a row group of LPR = B/VEC lanes handles one node; lane l
// owns trajectories l*VEC .. l*VEC+VEC-1 and accumulates them sequentially
// over the row, so every (v,b) sum is in CSR order.  Column indices are
// loaded LPR at a time with one coalesced load and broadcast by shuffles.
// One CTA per item (a range of at most 256 nodes of one member graph), or
// several per item for the global-memory kernel when there are few items.
//
// k_step_g: generic; neighbour rows of x are gathered from global memory.
// k_step_s: member graphs small enough for shared memory: the CTA first
//   copies its graph's block of x (and, for MIS, of the rounding bits) to
//   shared memory; every neighbour gather then hits shared memory, and the
//   MIS checker ORs whole 32-trajectory words of neighbour bits.  Several
//   rows per warp share each shuffle and shared-memory instruction.
#pragma once

#include <type_traits>

#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

// Staged-gather step kernel (mqo_step_staged.cu): CTAs of kStagedThreads
// threads, one Slice each (mqo_dev.cuh).
constexpr int kStagedThreads = 256;

// Byte offsets of the staged kernel's shared memory: counters, slice row
// pointers, column indices, weights, own rows of x and V, gathered rows.
struct StagedLayout {
  size_t cnt, rp, col, w, xo, vo, nb, total;
};
__host__ __device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ __forceinline__ StagedLayout staged_layout(int B, int sx, int sv, int cols, int rows,
                                                                bool weighted) {
  StagedLayout L;
  L.cnt = 0;
  L.rp = L.cnt + align16((size_t)3 * B * 8);
  L.col = L.rp + align16((size_t)(rows + 1) * 4);
  L.w = L.col + align16((size_t)cols * 4);
  L.xo = L.w + (weighted ? align16((size_t)cols) : 0);
  L.vo = L.xo + align16((size_t)rows * B * sx);
  L.nb = L.vo + align16((size_t)rows * B * sv);
  L.total = L.nb + align16((size_t)cols * B * sx);
  return L;
}

struct StepArgs {
  GraphDev g;
  int32_t B, Bw, R, problem, objective;
  int32_t split;  // generic kernel: CTAs per item, each taking a contiguous slice of its rows
  const Slice* slices;  // staged kernel: its slices, their count, and the most rows and CSR entries of one
  int32_t num_slices, slice_rows, slice_cols;
  float alpha, momentum, gamma, lambda_;
  void* X0;
  void* X1;
  void* V;
  uint32_t* ZX0;
  uint32_t* ZX1;
  Counters* cnt;
  const int32_t* act;         // nullptr: every trajectory steps
  const int32_t* gflag_step;  // nullptr: every member graph
  const int64_t* tick;
};

// Per-element tail of the step: evaluation of z(x), momentum update,
// projection, storage rounding.  `nb` is the neighbour information of the
// element: MIS any-neighbour-in-set flag, MaxCut weighted count P of
// neighbours with z = 1 (wsum = weighted degree).  OBJ >= 0 fixes the MaxCut
// relaxation at compile time (the f_B instances of the global-memory
// kernels); -1 reads it from the arguments.
template <typename TX, typename TV, int OBJ = -1>
__device__ __forceinline__ void step_element(const StepArgs& a, bool mis, float thr, float lo, TX xin, TV vin,
                                             float acc, int nb, int wsum, bool stepping, TX& xout, TV& vout,
                                             bool& znew, int& c0, int& c1, int& c2) {
  const float x = to_f(xin);
  const float vold = to_f(vin);
  const bool z = x > thr;
  const int obj = OBJ >= 0 ? OBJ : a.objective;
  if (mis) {
    const bool any = nb != 0;
    c0 += z;
    c1 += z && any;
    c2 += !z && !any;
  } else {
    const int as = 2 * nb - wsum;
    c0 += z ? (wsum - nb) : nb;
    const bool fixed = cut_fixed(obj, a.lambda_, z, as, wsum);
    c1 += !fixed;
    const int gn = z ? as : -as;
    c2 += gn > 0;
  }
  float grad;
  if (mis) {
    const float tt = a.gamma * acc;
    grad = 1.0f - tt;
  } else {
    grad = cut_grad(obj, a.lambda_, x, acc, wsum);
  }
  const float m1 = a.momentum * vold;
  const float m2 = a.alpha * grad;
  const float vn = m1 + m2;
  const float xn = clamp_box(x + vn, lo, 1.0f);
  if (stepping) {
    xout = from_f<TX>(xn);
    vout = from_f<TV>(vn);
  } else {
    xout = xin;
    vout = vin;
  }
  znew = to_f(xout) > thr;
}

// flush per-lane counters of an item: shared-memory reduction, then one
// atomic per trajectory and counter into replica (item % R)
template <int VEC>
__device__ __forceinline__ void flush_step_counters(const StepArgs& a, unsigned long long* s_cnt, int g, int it,
                                                    int b0, int lpr, int* c0, int* c1, int* c2,
                                                    uint32_t stepm) {
  // the 32/lpr row groups of a warp hold the same trajectories: sum them
  // by shuffles first, so one lane per trajectory issues the atomics
#pragma unroll
  for (int e = 0; e < VEC; ++e)
    for (int o = lpr; o < 32; o <<= 1) {
      c0[e] += __shfl_xor_sync(0xffffffffu, c0[e], o);
      c1[e] += __shfl_xor_sync(0xffffffffu, c1[e], o);
      c2[e] += __shfl_xor_sync(0xffffffffu, c2[e], o);
    }
  if ((threadIdx.x & 31) < lpr) {
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      if (!((stepm >> e) & 1u)) continue;
      if (c0[e]) atomicAdd(&s_cnt[3 * (b0 + e) + 0], (unsigned long long)(long long)c0[e]);
      if (c1[e]) atomicAdd(&s_cnt[3 * (b0 + e) + 1], (unsigned long long)(long long)c1[e]);
      if (c2[e]) atomicAdd(&s_cnt[3 * (b0 + e) + 2], (unsigned long long)(long long)c2[e]);
    }
  }
  __syncthreads();
  const int B = a.B;
  const int rep = it % a.R;
  for (int i = threadIdx.x; i < 3 * B; i += blockDim.x) {
    const unsigned long long val = s_cnt[i];
    if (val) {
      const int bb = i / 3, k = i - 3 * bb;
      Counters* c = a.cnt + ((int64_t)g * B + bb) * a.R + rep;
      unsigned long long* dst = k == 0 ? &c->value : (k == 1 ? &c->a : &c->b);
      atomicAdd(dst, val);
    }
  }
}

// the global-memory step kernel (mqo_step_generic.cu) for the given storage
// types and trajectories per lane
cudaError_t launch_step_generic(const StepArgs& a, int vec, int x_dtype, int v_dtype, int grid, cudaStream_t s);
// the staged-gather step kernel (mqo_step_staged.cu), `smem` bytes of
// dynamic shared memory (staged_layout(...).total)
cudaError_t launch_step_staged(const StepArgs& a, int vec, int x_dtype, int v_dtype, size_t smem, cudaStream_t s);
bool staged_vec_ok(int B, int x_dtype, int vec);
int default_staged_vec(int B, int x_dtype);

}  // namespace mqo
