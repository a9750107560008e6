// mqo_dev.cuh -- device-side types and helpers of the mQO CUDA library.
//
// Everything here is written for sm_103a and compiled with --fmad=false:
// every float expression rounds once per operation, exactly as written, so
// that the descent arithmetic is reproducible operation by operation.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace mqo {

enum : int { PROB_MIS = 0, PROB_MAXCUT = 1 };
enum : int { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2 };
// MaxCut relaxations of Sec. 3: f_B (Eq. 7, the default),
// f_L (Eq. 4), f_P (perturbed Laplacian), f_A (adjacency form)
enum : int { OBJ_FB = 0, OBJ_FL = 1, OBJ_FP = 2, OBJ_FA = 3 };
// PH_WAIT (pool mode): the trajectory holds a finished set until every
// trajectory of its graph has one (the batch of Alg. 3/4 steps 3-4)
enum : int { PH_DESCENT = 0, PH_REPAIR = 1, PH_LS = 2, PH_WAIT = 3 };
// graph-wide decisions of the pool machine for one tick
enum : int { DEC_NONE = 0, DEC_NEXT = 1, DEC_LS = 2, DEC_OUTER = 3 };
enum : int { EP_DESCENT = 0, EP_LS = 1 };
constexpr int kPoolMax = 128;  // largest pool size K
enum : int {
  RD_NONE = -1,
  RD_COUNT = 0,
  RD_DROP = 1,
  RD_COMPLETE = 2,
  RD_SWAP = 3,
  RD_FLIP1 = 4,
  RD_FLIP2 = 5
};
// per-trajectory actions decided by the control kernel for one tick
enum : int {
  ACT_STEP = 1,        // take a descent step this tick
  ACT_ACC_ZX = 2,      // best <- z of the x evaluated by the last step
  ACT_ACC_WORK = 4,    // best <- work set (repaired / locally searched)
  ACT_RESET = 8,       // x <- best set with R zeroed, V <- 0 (Alg. 1 steps 6-8)
  ACT_INIT = 16,       // x <- fresh initialisation, V <- 0 (Alg. 1 step 2)
  ACT_WORK_ZX = 32,    // work set <- z of the last step (repair entry)
  ACT_WORK_BEST = 64,  // work set <- best set (local-search entry)
  ACT_POOL = 128,      // pool mode: RESET / WORK_BEST take pool slot pbase[t] (empty set if < 0) as base
  ACT_APPLY_MASK = ACT_ACC_ZX | ACT_ACC_WORK | ACT_RESET | ACT_INIT | ACT_WORK_ZX | ACT_WORK_BEST
};

struct Params {
  int32_t problem, B, x_dtype, v_dtype;
  float alpha, momentum, gamma, lambda_;
  double rho;
  float sigma;
  int32_t t_gs, cap, init_kind, local_search, repair;
  uint64_t seed;
  int32_t objective;  // MaxCut relaxation (OBJ_*)
  int32_t pool_k;     // 0: independent trajectories; K >= 1: pmQO pool of K sets per graph
};

// One trajectory of the tick machine (field meanings as mqo_traj_info).
struct __align__(16) TrajState {
  int32_t phase, s, r, o;
  int64_t best, ticks;
  int32_t last_round, round;  // round: discrete round of the current tick
  int64_t last_commits;
  int64_t ev_value, ev_a, ev_b;
  int64_t accepts, descents;
  int32_t act, ls_done;
  uint32_t rkeys[6];
  int64_t rk;
  int64_t held;  // pool mode: value of the held set (INT64_MIN: none, or not a candidate)
  // gains breakdown: the first accepted value (end of the first descent's
  // gradient updates), then the strict improvements accepted from later
  // descents (global resets, restarts) and from local search
  int64_t first_value, gain_descent, gain_ls;
  int64_t steps;  // descent steps taken in all
};

// book a strict improvement of st.best to `value` by its source
__device__ __forceinline__ void credit_gain(TrajState& st, int64_t value, bool from_ls) {
  if (st.best == (int64_t)(-9223372036854775807LL - 1)) st.first_value = value;
  else if (from_ls) st.gain_ls += value - st.best;
  else st.gain_descent += value - st.best;
}

// Per member graph state of the pool machine (pmQO, Alg. 3/4).
struct PoolState {
  int32_t epoch;    // EP_DESCENT: trajectories finish descents; EP_LS: local searches
  int32_t count;    // pool members (<= K)
  int64_t best;     // value of the graph's best set (INT64_MIN before the first)
  int64_t merges;   // pool merges so far
  int32_t dec;      // decision of the current tick (DEC_*)
  int32_t best_src; // best set replaced this tick from: 0 the new pool slot 0, K + b trajectory b's work set, -1 no
  int32_t merged;   // 1 if the pool was rewritten this tick (psrc holds the sources of slots 0..count-1)
  int32_t stamp;    // tick + 1 when pool bits or the best set must be rewritten this tick
};

// Per-trajectory integer sums produced by one tick (value of MaxCut is 2*cut).
struct Counters {
  unsigned long long value, a, b, commits;
};

// A contiguous node range inside one member graph.
constexpr int kItemMaxNodes = 256;  // nodes of one work item (a node range of one member graph)

struct Item {
  int32_t g, v0, v1, pad;
};

// A node range [v0, v1) inside work item `it` of member graph g, CSR
// entries [j0, j1): the unit of the staged-gather step kernels (at most
// slice_rows rows whose CSR rows hold at most slice_cols entries together).
struct __align__(16) Slice {
  int32_t g, it, v0, v1, j0, j1, pad0, pad1;
};

struct GraphDev {
  int32_t n, num_graphs;
  int64_t nnz;
  const int32_t* row_ptr;   // n+1
  const int32_t* col;       // nnz, global ids
  const uint16_t* col16;    // nnz, member-local ids (every member graph below 65536 nodes), else nullptr
  const int8_t* w;          // nnz or nullptr
  const int32_t* node_off;  // num_graphs+1
  const int32_t* dmax;      // num_graphs
  const Item* items;
  const int32_t* order;     // n: the rows of each item [v0,v1) by decreasing degree
  int32_t num_items;
};

struct SolverDev {
  GraphDev g;
  Params p;
  int32_t B, Bw;
  int32_t R;        // counter replicas per trajectory (item i adds into replica i % R)
  int32_t step_vec; // trajectories per lane of the global-memory step kernel (0: B/32 or 1)
  int32_t step_wide; // shared-memory step kernel with 16-byte lanes
  int32_t step_c16;  // shared-memory step kernel reads the 16-bit member-local column indices
  int32_t split;    // CTAs per item of the node-parallel kernels (several when there are few items)
  int32_t step_staged;  // 1: staged-gather step kernel (when the shared-memory one is not used)
  const Slice* slices;  // its slices, their count, and the most rows / CSR entries of one slice
  int32_t num_slices, slice_rows, slice_cols;
  void* X0;         // relaxed x: tick t reads X[t&1] and writes X[(t+1)&1]
  void* X1;
  void* V;          // momentum
  uint32_t* ZX0;    // ZX[k] = threshold rounding of X[k], node-major bits
  uint32_t* ZX1;
  uint32_t* Zbest;  // best set
  uint32_t* Zwork;  // work set of repair / local search
  uint32_t* Zaux;   // tight (MIS) / positive-gain (MaxCut) bits
  uint32_t* Zfree;  // free (uncovered) bits
  uint32_t* Zdrop;  // drop decisions of a repair round
  int32_t* owner;   // [n*B] move ownership marks
  int32_t* pa;      // [n*B] proposal endpoint a
  int32_t* pb;      // [n*B] proposal endpoint b
  int32_t* gain;    // [n*B] 1-flip gains (MaxCut)
  TrajState* st;    // [G*B]
  int32_t* act;     // [G*B] actions of the current tick (compact copy)
  int32_t* rnd;     // [G*B] discrete round of the current tick (compact copy)
  Counters* cnt;    // [G*B*R]
  int64_t* tick;    // current tick number
  int32_t* gflag;   // [3*G] tick stamps: any apply / any discrete / any step
  int32_t* any;     // [4] per-tick "any trajectory" stamps (apply, disc, step)
  int64_t* bestv;   // [G*B] best value of each trajectory (compact copy for readout)
  // pool mode (p.pool_k = K > 0)
  int32_t K, Kw;    // pool size, pool bit words per node
  uint32_t* Pool;   // [n*Kw] pool sets, node-major: slot k of node v = bit k%32 of word v*Kw + k/32
  PoolState* pool;  // [G]
  int32_t* psrc;    // [G*K] source of new slot s of a merge: j < K old slot j, K + b trajectory b's work set
  int64_t* pval;    // [G*K] values of the pool members, best first
  int32_t* pbase;   // [G*B] pool slot a trajectory resets / searches from (-1: the empty set)
};

// The item of this CTA and its slice of the item's nodes when each item is
// split over S.split CTAs (CTA c takes slice c % split); false if the slice
// is empty.
__device__ __forceinline__ bool item_slice(const SolverDev& S, int& it, Item& item) {
  it = blockIdx.x / S.split;
  item = S.g.items[it];
  const int part = blockIdx.x - it * S.split;
  const int per = (item.v1 - item.v0 + S.split - 1) / S.split;
  const int r0 = item.v0 + part * per;
  item.v1 = item.v1 < r0 + per ? item.v1 : r0 + per;
  item.v0 = r0;
  return item.v0 < item.v1;
}

// sum of the R replicas of a trajectory's counters
__device__ __forceinline__ Counters sum_replicas(const Counters* c, int64_t tau, int R) {
  Counters s{0ull, 0ull, 0ull, 0ull};
  for (int r = 0; r < R; ++r) {
    const Counters x = c[tau * R + r];
    s.value += x.value;
    s.a += x.a;
    s.b += x.b;
    s.commits += x.commits;
  }
  return s;
}

// --------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11), device version.
// --------------------------------------------------------------------------
struct U64x4 {
  uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                               uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t h0 = __umul64hi(M0, c0), l0 = M0 * c0;
    const uint64_t h1 = __umul64hi(M1, c2), l1 = M1 * c2;
    const uint64_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
    c0 = n0;
    c1 = l1;
    c2 = n2;
    c3 = l0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  U64x4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

constexpr uint64_t TAG_INIT = 1ULL;
constexpr uint64_t TAG_RESET = 2ULL;

__device__ __forceinline__ float unit24(uint64_t w) { return (float)(w >> 40) * (1.0f / 16777216.0f); }

// --------------------------------------------------------------------------
// Keyed permutation of {0..n-1}: Feistel network on ceil(log2 n) bits with
// alternating half widths, lowbias32 round function, cycle walking.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ uint32_t feistel_once(uint32_t v, int d, const uint32_t* k) {
  int wl = d >> 1, wr = d - wl;
  uint32_t L = v >> wr, R = v & ((1u << wr) - 1u);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const uint32_t f = mix32(R ^ k[i]) & ((1u << wl) - 1u);
    const uint32_t nl = R, nr = L ^ f;
    const int t = wl;
    wl = wr;
    wr = t;
    L = nl;
    R = nr;
  }
  return (L << wr) | R;
}

// sigma(v) for 0 <= v < n; the walk ends within 2^d steps (d <= 31).
__device__ __forceinline__ uint32_t feistel_sigma(uint32_t n, const uint32_t* k, uint32_t v) {
  if (n <= 1u) return v;
  int d = 32 - __clz(n - 1u);
  if (d < 2) d = 2;
  uint32_t y = feistel_once(v, d, k);
  for (uint32_t it = 0; y >= n && it < (1u << d); ++it) y = feistel_once(y, d, k);
  return y;
}

// --------------------------------------------------------------------------
// Storage types
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// VEC consecutive elements of T loaded / stored as one aligned access.
template <typename T, int VEC>
struct alignas(sizeof(T) * VEC) Pack {
  T e[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ Pack<T, VEC> ld_pack(const T* p) {
  return *reinterpret_cast<const Pack<T, VEC>*>(p);
}
template <typename T, int VEC>
__device__ __forceinline__ Pack<T, VEC> ld_pack_stream(const T* p) {
  Pack<T, VEC> r;
  if constexpr (sizeof(Pack<T, VEC>) == 16) {
    int4 t = __ldcs(reinterpret_cast<const int4*>(p));
    r = *reinterpret_cast<Pack<T, VEC>*>(&t);
  } else if constexpr (sizeof(Pack<T, VEC>) == 8) {
    int2 t = __ldcs(reinterpret_cast<const int2*>(p));
    r = *reinterpret_cast<Pack<T, VEC>*>(&t);
  } else if constexpr (sizeof(Pack<T, VEC>) == 4) {
    int t = __ldcs(reinterpret_cast<const int*>(p));
    r = *reinterpret_cast<Pack<T, VEC>*>(&t);
  } else {
    r = *reinterpret_cast<const Pack<T, VEC>*>(p);
  }
  return r;
}
template <typename T, int VEC>
__device__ __forceinline__ void st_pack(T* p, const Pack<T, VEC>& v) {
  *reinterpret_cast<Pack<T, VEC>*>(p) = v;
}

// VEC elements of T at p (aligned to VEC*sizeof(T)) as floats, read with one
// vector load.  bfloat16 -> float is exact: the 16 bits become the high half
// of the float's bits; binary16 goes through the half2 conversion.
template <typename T, int VEC>
__device__ __forceinline__ void load_unpack(const unsigned char* p, float* f);
template <>
__device__ __forceinline__ void load_unpack<__nv_bfloat16, 4>(const unsigned char* p, float* f) {
  const uint2 r = *reinterpret_cast<const uint2*>(p);
  f[0] = __uint_as_float(r.x << 16);
  f[1] = __uint_as_float(r.x & 0xffff0000u);
  f[2] = __uint_as_float(r.y << 16);
  f[3] = __uint_as_float(r.y & 0xffff0000u);
}
template <>
__device__ __forceinline__ void load_unpack<__nv_bfloat16, 8>(const unsigned char* p, float* f) {
  const uint4 r = *reinterpret_cast<const uint4*>(p);
  f[0] = __uint_as_float(r.x << 16);
  f[1] = __uint_as_float(r.x & 0xffff0000u);
  f[2] = __uint_as_float(r.y << 16);
  f[3] = __uint_as_float(r.y & 0xffff0000u);
  f[4] = __uint_as_float(r.z << 16);
  f[5] = __uint_as_float(r.z & 0xffff0000u);
  f[6] = __uint_as_float(r.w << 16);
  f[7] = __uint_as_float(r.w & 0xffff0000u);
}
template <>
__device__ __forceinline__ void load_unpack<__half, 8>(const unsigned char* p, float* f) {
  const uint4 r = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
    f[2 * k] = a.x;
    f[2 * k + 1] = a.y;
  }
}
template <>
__device__ __forceinline__ void load_unpack<__half, 4>(const unsigned char* p, float* f) {
  const uint2 r = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
  f[0] = a.x;
  f[1] = a.y;
  f[2] = b.x;
  f[3] = b.y;
}
template <>
__device__ __forceinline__ void load_unpack<__nv_bfloat16, 2>(const unsigned char* p, float* f) {
  const uint32_t r = *reinterpret_cast<const uint32_t*>(p);
  f[0] = __uint_as_float(r << 16);
  f[1] = __uint_as_float(r & 0xffff0000u);
}
template <>
__device__ __forceinline__ void load_unpack<__half, 2>(const unsigned char* p, float* f) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(p));
  f[0] = a.x;
  f[1] = a.y;
}
template <>
__device__ __forceinline__ void load_unpack<float, 2>(const unsigned char* p, float* f) {
  const float2 r = *reinterpret_cast<const float2*>(p);
  f[0] = r.x;
  f[1] = r.y;
}
template <>
__device__ __forceinline__ void load_unpack<float, 4>(const unsigned char* p, float* f) {
  const float4 r = *reinterpret_cast<const float4*>(p);
  f[0] = r.x;
  f[1] = r.y;
  f[2] = r.z;
  f[3] = r.w;
}

// (a, b) += (x, y) with one packed FP32 add (sm_100 family): each element
// is an IEEE round-to-nearest addition, bit-identical to a + x and b + y
__device__ __forceinline__ void add_f32x2(float& a, float& b, float x, float y) {
  asm("{\n\t.reg .b64 p, q;\n\t"
      "mov.b64 p, {%0, %1};\n\t"
      "mov.b64 q, {%2, %3};\n\t"
      "add.rn.f32x2 p, p, q;\n\t"
      "mov.b64 {%0, %1}, p;\n\t}"
      : "+f"(a), "+f"(b)
      : "f"(x), "f"(y));
}

// acc[e] += widened bfloat16 e of the VEC-element row at p (8 or 16 bytes,
// aligned), one add.rn.f32.bf16 (sm_100 family) per element: the bfloat16
// operand converts to float32 exactly and the sum rounds once to nearest,
// bit-identical to widening first and adding in float32.
__device__ __forceinline__ void add_bf16x2_word(float& a, float& b, uint32_t w) {
  asm("{\n\t.reg .b16 lo, hi;\n\t"
      "mov.b32 {lo, hi}, %2;\n\t"
      "add.rn.f32.bf16 %0, lo, %0;\n\t"
      "add.rn.f32.bf16 %1, hi, %1;\n\t}"
      : "+f"(a), "+f"(b)
      : "r"(w));
}
template <int VEC>
__device__ __forceinline__ void add_bf16_row(float* acc, const unsigned char* p);
template <>
__device__ __forceinline__ void add_bf16_row<4>(float* acc, const unsigned char* p) {
  const uint2 r = *reinterpret_cast<const uint2*>(p);
  add_bf16x2_word(acc[0], acc[1], r.x);
  add_bf16x2_word(acc[2], acc[3], r.y);
}
template <>
__device__ __forceinline__ void add_bf16_row<8>(float* acc, const unsigned char* p) {
  const uint4 r = *reinterpret_cast<const uint4*>(p);
  add_bf16x2_word(acc[0], acc[1], r.x);
  add_bf16x2_word(acc[2], acc[3], r.y);
  add_bf16x2_word(acc[4], acc[5], r.z);
  add_bf16x2_word(acc[6], acc[7], r.w);
}
template <>
__device__ __forceinline__ void add_bf16_row<2>(float* acc, const unsigned char* p) {
  add_bf16x2_word(acc[0], acc[1], *reinterpret_cast<const uint32_t*>(p));
}

__device__ __forceinline__ float clamp_box(float v, float lo, float hi) {
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

// Ascent direction of a MaxCut relaxation at x given acc = (Ax)_v (float32,
// CSR order) and the weighted degree d: f_B -lambda - 2 acc, f_A -2 acc,
// f_L 1/2 (d x - acc), f_P 2 ((d x - acc) + lambda x); one rounding per
// operation, as written (the gradients of Sec. 3's definitions).
__device__ __forceinline__ float cut_grad(int obj, float lambda_, float x, float acc, int d) {
  if (obj == OBJ_FB || obj == OBJ_FA) {
    const float t = 2.0f * acc;
    return obj == OBJ_FB ? -lambda_ - t : -t;
  }
  const float t1 = (float)d * x;
  const float t2 = t1 - acc;
  if (obj == OBJ_FL) return 0.5f * t2;
  const float t3 = lambda_ * x;
  const float t4 = t2 + t3;
  return 2.0f * t4;
}

// Is the binary point fixed at node v under a PGA step of the relaxation?
// s_v = +1 (z) is fixed iff the gradient there is >= 0, s_v = -1 iff <= 0,
// with as = (As)_v and d the weighted degree (integers):
//   f_B: grad = -lambda - 2 as (0 < lambda < 2, integer weights, Thm 3.6)
//   f_L: grad = 1/2 (d s_v - as);  f_P: grad = 2 (d s_v - as + lambda s_v);
//   f_A: grad = -2 as.  |as - d| < 2^24, so the f_P comparison is exact in float.
__device__ __forceinline__ bool cut_fixed(int obj, float lambda_, bool z, int as, int d) {
  switch (obj) {
    case OBJ_FL: return z ? (as <= d) : (as >= -d);
    case OBJ_FP: return z ? ((float)(as - d) <= lambda_) : ((float)(-(as + d)) <= lambda_);
    case OBJ_FA: return z ? (as <= 0) : (as >= 0);
    default: return z ? (as <= -1) : (as >= 0);
  }
}

// --------------------------------------------------------------------------
// Bit words: node-major, Bw words per node, trajectory b -> bit b%32 of
// word b/32.  In the (node, trajectory) thread mapping used by the pair
// kernels (trajectory fastest, blockDim a multiple of max(32, B)), every
// word of a node is owned by the lanes of one warp, so word updates are
// aggregated with ballots and written by one lane.
// --------------------------------------------------------------------------
__device__ __forceinline__ bool get_bit(const uint32_t* words, int64_t v, int Bw, int b) {
  return (words[v * Bw + (b >> 5)] >> (b & 31)) & 1u;
}

// Update the calling lane's bit in word `words[v*Bw + b/32]` to `val` where
// `active`; all 32 lanes must call this together.
__device__ __forceinline__ void update_word(uint32_t* words, int64_t v, int Bw, int b, int B, bool val, bool active) {
  const unsigned full = 0xffffffffu;
  const unsigned mv = __ballot_sync(full, val && active);
  const unsigned ma = __ballot_sync(full, active);
  const int lane = threadIdx.x & 31;
  const int G = B < 32 ? B : 32;
  const int gbase = lane & ~(G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const unsigned gv = (mv >> gbase) & gmask, ga = (ma >> gbase) & gmask;
  if (lane == gbase && ga) {
    uint32_t* wp = words + v * Bw + (b >> 5);
    *wp = (*wp & ~ga) | (gv & ga);
  }
}

// As update_word, but safe against concurrent atomic writers of other bits
// of the same word (used where cross-node commits run in the same pass).
__device__ __forceinline__ void update_word_atomic(uint32_t* words, int64_t v, int Bw, int b, int B, bool val,
                                                   bool active) {
  const unsigned full = 0xffffffffu;
  const unsigned mv = __ballot_sync(full, val && active);
  const unsigned ma = __ballot_sync(full, active);
  const int lane = threadIdx.x & 31;
  const int G = B < 32 ? B : 32;
  const int gbase = lane & ~(G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const unsigned gv = (mv >> gbase) & gmask, ga = (ma >> gbase) & gmask;
  if (lane == gbase && ga) {
    uint32_t* wp = words + v * Bw + (b >> 5);
    if (ga & ~gv) atomicAnd(wp, ~(ga & ~gv));
    if (gv) atomicOr(wp, gv);
  }
}

__device__ __forceinline__ bool sorted_contains(const int32_t* col, int32_t lo, int32_t hi, int32_t key) {
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    const int32_t c = col[mid];
    if (c == key) return true;
    if (c < key) lo = mid + 1;
    else hi = mid;
  }
  return false;
}

}  // namespace mqo
