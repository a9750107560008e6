// mqo_pool.cu -- the graph-wide part of pmQO (Alg. 3 for MIS, Alg. 4 for
// MaxCut): the B trajectories of a member graph share a pool P_K of the K
// best sets found so far.
//
// A trajectory whose descent (or the repair of a capped MIS descent, or a
// local search) is over holds its set and waits (PH_WAIT).  At the start of
// the tick after every trajectory of the graph waits, k_pool_ctrl (one CTA
// per member graph) merges the held sets into the pool -- P_K <- TopK(P_K U
// batch), steps 4 and 11, a stable selection of the K largest values with
// pool members first (pool order) and then the batch (trajectory order) --
// replaces the graph's best set by the pool's first member if that is
// strictly better (steps 5 and 12), and decides what every trajectory does
// next:
//   DEC_NEXT   another reset round (steps 6-10): trajectory b restarts from
//              pool member k_b drawn uniformly (step 7) with its reset set R
//              zeroed (steps 8-9)
//   DEC_LS     after T_gs rounds, local search (step 13): OneTwoSwap on the
//              best set (MIS, one trajectory), OneTwoFlip on every pool
//              member (MaxCut, trajectory b searches member b)
//   DEC_OUTER  a new outer iteration with fresh initialisations (step 2)
// At the end of a local-search epoch the best search result replaces the
// best set if it is strictly better.  k_pool_apply then rewrites the pool
// bits and the best sets node by node (one CTA per item).  The per
// trajectory part of the decision is taken by the control kernel.
#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

constexpr uint64_t TAG_POOL = 3ULL;
constexpr int kPoolThreads = 256;
constexpr int64_t kNoValue = (int64_t)(-9223372036854775807LL - 1);

// Step 7: a pool index uniform in [0, count): the high 64 bits of u * count
// for the first 64-bit Philox word u keyed (seed, trajectory), counter
// (TAG_POOL, outer iteration, round).
__device__ __forceinline__ int32_t pool_pick(uint64_t seed, int64_t tau, int32_t o, int32_t r, int32_t count) {
  if (count <= 0) return -1;
  const U64x4 w = philox4x64_10(TAG_POOL, (uint64_t)o, (uint64_t)r, 0ULL, seed, (uint64_t)tau);
  return (int32_t)__umul64hi(w.v[0], (uint64_t)count);
}

__global__ void __launch_bounds__(kPoolThreads) k_pool_ctrl(SolverDev S) {
  __shared__ int64_t s_v[kPoolMax + 128];  // candidate values
  __shared__ int32_t s_c[kPoolMax + 128];  // candidate sources
  __shared__ int64_t s_h[128];             // held values of the batch
  __shared__ int32_t s_wait, s_nh;
  __shared__ int64_t s_first;  // value of the new first pool member
  const int g = blockIdx.x;
  const int B = S.B, K = S.K;
  const int tid = threadIdx.x;
  const int64_t t = *S.tick;
  PoolState ps = S.pool[g];  // read by every thread before thread 0 writes it
  if (tid == 0) {
    s_wait = 1;
    s_nh = 0;
  }
  __syncthreads();
  for (int b = tid; b < B; b += blockDim.x) {
    const TrajState& st = S.st[(int64_t)g * B + b];
    if (st.phase != PH_WAIT) s_wait = 0;
    s_h[b] = st.held;
  }
  __syncthreads();
  if (!s_wait) {
    if (tid == 0) {
      ps.dec = DEC_NONE;
      ps.best_src = -1;
      ps.merged = 0;
      S.pool[g] = ps;
    }
    return;
  }
  if (ps.epoch == EP_LS) {
    // end of step 13: the best search result replaces the best set if it
    // is strictly better (the first trajectory on ties)
    if (tid == 0) {
      int win = -1;
      int64_t bv = ps.best;
      for (int b = 0; b < B; ++b)
        if (s_h[b] != kNoValue && s_h[b] > bv) {
          bv = s_h[b];
          win = b;
        }
      ps.best_src = -1;
      ps.merged = 0;
      if (win >= 0) {
        ps.best = bv;
        ps.best_src = K + win;
        ps.stamp = (int32_t)(t + 1);
      }
      ps.epoch = EP_DESCENT;
      ps.dec = DEC_OUTER;
      S.pool[g] = ps;
    }
    return;
  }
  // steps 4 / 11: candidates are the pool members (pool order), then the
  // held sets that are candidates (trajectory order)
  const int count = ps.count;
  for (int j = tid; j < count; j += blockDim.x) {
    s_v[j] = S.pval[(int64_t)g * K + j];
    s_c[j] = j;
  }
  for (int b = tid; b < B; b += blockDim.x) {
    if (s_h[b] == kNoValue) continue;
    int pos = 0;
    for (int q = 0; q < b; ++q) pos += s_h[q] != kNoValue;
    s_v[count + pos] = s_h[b];
    s_c[count + pos] = K + b;
    atomicAdd(&s_nh, 1);
  }
  __syncthreads();
  const int nc = count + s_nh;
  const int keep = nc < K ? nc : K;
  // stable descending order: the rank of candidate i counts the larger
  // values and the equal values before it
  int64_t myv[2];
  int32_t myc[2], myr[2];
  int mine = 0;
  for (int i = tid; i < nc; i += blockDim.x) {
    const int64_t v = s_v[i];
    int rank = 0;
    for (int j = 0; j < nc; ++j) {
      const int64_t u = s_v[j];
      rank += (u > v) || (u == v && j < i);
    }
    myv[mine] = v;
    myc[mine] = s_c[i];
    myr[mine] = rank;
    ++mine;
  }
  __syncthreads();  // every candidate read before the pool values are rewritten
  for (int k = 0; k < mine; ++k)
    if (myr[k] < K) {
      S.pval[(int64_t)g * K + myr[k]] = myv[k];
      S.psrc[(int64_t)g * K + myr[k]] = myc[k];
      if (myr[k] == 0) s_first = myv[k];
    }
  __syncthreads();
  const int64_t first = keep > 0 ? s_first : kNoValue;
  // the decision reads the round counters of trajectory 0 (all trajectories
  // of a graph advance r and o together in pool mode)
  const TrajState& s0 = S.st[(int64_t)g * B];
  const int32_t r0 = s0.r, o0 = s0.o;
  int dec;
  if (r0 < S.p.t_gs) dec = DEC_NEXT;
  else if (S.p.local_search) dec = DEC_LS;
  else dec = DEC_OUTER;
  const bool mis = S.p.problem == PROB_MIS;
  for (int b = tid; b < B; b += blockDim.x) {
    const int64_t tau = (int64_t)g * B + b;
    int32_t base = -1;
    if (dec == DEC_NEXT) base = pool_pick(S.p.seed, tau, o0, r0 + 1, keep);
    else if (dec == DEC_LS && !mis) base = b < keep ? b : -1;
    S.pbase[tau] = base;
  }
  if (tid == 0) {
    ps.count = keep;
    ps.merges += 1;
    ps.merged = 1;
    ps.best_src = -1;
    if (keep > 0 && first > ps.best) {  // steps 5 / 12
      ps.best = first;
      ps.best_src = 0;
    }
    ps.stamp = (int32_t)(t + 1);
    ps.dec = dec;
    if (dec == DEC_LS) ps.epoch = EP_LS;
    S.pool[g] = ps;
  }
}

// Rewrite the pool bits of a merge and the best sets of a replacement, node
// by node; the sources are read before any word of the node is written.
__global__ void __launch_bounds__(kPoolThreads) k_pool_apply(SolverDev S) {
  __shared__ int32_t s_src[kPoolMax];
  const Item item = S.g.items[blockIdx.x];
  const int g = item.g;
  const int64_t t = *S.tick;
  const PoolState ps = S.pool[g];
  if (ps.stamp != (int32_t)(t + 1)) return;
  const int K = S.K, Kw = S.Kw, B = S.B, Bw = S.Bw;
  if (ps.merged)
    for (int k = threadIdx.x; k < ps.count; k += blockDim.x) s_src[k] = S.psrc[(int64_t)g * K + k];
  __syncthreads();
  const uint32_t full = B >= 32 ? 0xffffffffu : ((1u << B) - 1u);
  for (int64_t v = item.v0 + threadIdx.x; v < item.v1; v += blockDim.x) {
    uint32_t w[kPoolMax / 32];
#pragma unroll
    for (int k = 0; k < kPoolMax / 32; ++k) w[k] = k < Kw ? S.Pool[v * Kw + k] : 0u;
    if (ps.merged) {
      uint32_t nw[kPoolMax / 32] = {0u, 0u, 0u, 0u};
      for (int s = 0; s < ps.count; ++s) {
        const int src = s_src[s];
        const uint32_t bit = src < K ? (w[src >> 5] >> (src & 31)) & 1u : (uint32_t)get_bit(S.Zwork, v, Bw, src - K);
        nw[s >> 5] |= bit << (s & 31);
      }
#pragma unroll
      for (int k = 0; k < kPoolMax / 32; ++k) {
        w[k] = nw[k];
        if (k < Kw) S.Pool[v * Kw + k] = nw[k];
      }
    }
    if (ps.best_src >= 0) {
      const bool bit = ps.best_src < K ? (w[0] & 1u) : get_bit(S.Zwork, v, Bw, ps.best_src - K);
      for (int k = 0; k < Bw; ++k) S.Zbest[v * Bw + k] = bit ? full : 0u;
    }
  }
}

cudaError_t launch_pool_ctrl(const SolverDev& S, cudaStream_t stream) {
  k_pool_ctrl<<<S.g.num_graphs, kPoolThreads, 0, stream>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_pool_apply(const SolverDev& S, cudaStream_t stream) {
  k_pool_apply<<<S.g.num_items, kPoolThreads, 0, stream>>>(S);
  return cudaGetLastError();
}

}  // namespace mqo
