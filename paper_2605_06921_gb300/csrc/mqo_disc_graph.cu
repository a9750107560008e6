// mqo_disc_graph.cu -- the discrete passes of a tick (repair and local
// search rounds, then the counts of the work set) fused into one kernel for
// member graphs that fit in shared memory: one CTA per member graph stages
// the graph's bit words (work set, tight / positive-gain bits, free bits,
// drop bits) in shared memory and runs pass A (decide / propose), pass B
// (commit) and pass C (count) with block barriers in between, then writes
// the words back.  Same rounds and results as the three k_disc launches
// (see mqo_tick.cu): repair = Def. 2.1 feasibility + maximality; rounds of
// (1,2)-swaps (Def. 2.3), 1-flips (Def. 2.4) and 2-flips (Def. 2.5).
//
// Mapping: B >= 32 (Bw = B/32 words per node).  Warp w always handles word
// w % Bw of its nodes, so lane l always owns trajectory (w % Bw)*32 + l and
// keeps its counters in registers.  Whole-word set logic (ORs over smaller
// neighbours, once/twice counts) is computed by the warp's 32 lanes
// together from shared memory.
#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

namespace {

constexpr int kDgThreads = 1024;  // one CTA per SM: 32 warps overlap their neighbour-list loads

__device__ __forceinline__ bool sbit(const uint32_t* words, int u, int Bw, int b) {
  return (words[u * Bw + (b >> 5)] >> (b & 31)) & 1u;
}

// A node's neighbour list held in registers: lane l holds entries
// rs + l + 32k (k < kNb) as local ids, -1 past the end.  The loads of a list
// are independent, so one list costs one memory latency; longer rows keep
// their tail (entries past rs + 32 kNb) in memory.
constexpr int kNb = 5;
// tight neighbours a set node keeps in registers for its swap search; a
// longer list falls back to the sequential scan
constexpr int kTight = 8;

struct NbList {
  int32_t u[kNb];
  int32_t rs, re;
};

// member-local id of entry j: the 16-bit copy where the graph has one (half
// the bytes, and it was just streamed by the step kernel of the same tick)
__device__ __forceinline__ int32_t local_col(const int32_t* col, const uint16_t* col16, int32_t off, int32_t j) {
  return col16 ? (int32_t)col16[j] : col[j] - off;
}

__device__ __forceinline__ void nb_load(NbList& L, const int32_t* s_rp, const int32_t* col, const uint16_t* col16,
                                        int32_t off, int vl) {
  const int lane = threadIdx.x & 31;
  L.rs = s_rp[vl];
  L.re = s_rp[vl + 1];
#pragma unroll
  for (int k = 0; k < kNb; ++k) {
    const int32_t j = L.rs + lane + 32 * k;
    L.u[k] = j < L.re ? local_col(col, col16, off, j) : -1;
  }
}

// OR over the list (only u < vl if `less`) of word wk of `words`
__device__ __forceinline__ uint32_t nb_or(const NbList& L, const uint32_t* words, const int32_t* col,
                                          const uint16_t* col16, int32_t off, int Bw, int wk, int vl, bool less) {
  const int lane = threadIdx.x & 31;
  uint32_t r = 0u;
#pragma unroll
  for (int k = 0; k < kNb; ++k) {
    const int32_t u = L.u[k];
    if (u >= 0 && (!less || u < vl)) r |= words[u * Bw + wk];
  }
  for (int32_t j = L.rs + 32 * kNb + lane; j < L.re; j += 32) {
    const int32_t u = local_col(col, col16, off, j);
    if (!less || u < vl) r |= words[u * Bw + wk];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r |= __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// bits set in at least one / at least two neighbours' word wk
__device__ __forceinline__ void nb_once_twice(const NbList& L, const uint32_t* words, const int32_t* col,
                                              const uint16_t* col16, int32_t off, int Bw, int wk, uint32_t& once,
                                              uint32_t& twice) {
  const int lane = threadIdx.x & 31;
  once = 0u;
  twice = 0u;
#pragma unroll
  for (int k = 0; k < kNb; ++k) {
    const int32_t u = L.u[k];
    const uint32_t w = u >= 0 ? words[u * Bw + wk] : 0u;
    twice |= once & w;
    once |= w;
  }
  for (int32_t j = L.rs + 32 * kNb + lane; j < L.re; j += 32) {
    const uint32_t w = words[local_col(col, col16, off, j) * Bw + wk];
    twice |= once & w;
    once |= w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t o2 = __shfl_xor_sync(0xffffffffu, once, o);
    const uint32_t t2 = __shfl_xor_sync(0xffffffffu, twice, o);
    twice = twice | t2 | (once & o2);
    once |= o2;
  }
}

}  // namespace

__global__ void __launch_bounds__(kDgThreads) k_disc_graph(SolverDev S) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int g = blockIdx.x;
  const int64_t t = *S.tick;
  if (S.any[1] != (int32_t)(t + 1)) return;
  const int G = S.g.num_graphs;
  if (S.gflag[G + g] != (int32_t)(t + 1)) return;
  const int B = S.B, Bw = S.Bw;
  const bool mis = S.p.problem == PROB_MIS;
  const int32_t off = S.g.node_off[g];
  const int32_t ng = S.g.node_off[g + 1] - off;
  const int32_t* rp = S.g.row_ptr;
  const int32_t* col = S.g.col;
  const uint16_t* col16 = S.g.col16;
  const int8_t* wts = S.g.w;
  const int nw = ng * Bw;
  uint32_t* sW = reinterpret_cast<uint32_t*>(smem);  // work set
  uint32_t* sA = sW + nw;                            // tight / positive gain
  uint32_t* sF = sA + nw;                            // free
  uint32_t* sD = sF + nw;                            // drop decisions
  int* s_rnd = reinterpret_cast<int*>(sD + nw);      // round of each trajectory
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_rnd + ((B + 1) & ~1));
  int32_t* s_rp = reinterpret_cast<int32_t*>(s_cnt + 4 * B);  // row pointers of the graph

  for (int i = threadIdx.x; i < nw; i += blockDim.x) {
    const int64_t gi = (int64_t)off * Bw + i;
    sW[i] = S.Zwork[gi];
    sA[i] = S.Zaux[gi];
    sF[i] = S.Zfree[gi];
    sD[i] = 0u;
  }
  for (int i = threadIdx.x; i < B; i += blockDim.x) s_rnd[i] = S.rnd[(int64_t)g * B + i];
  for (int i = threadIdx.x; i < 4 * B; i += blockDim.x) s_cnt[i] = 0ull;
  for (int i = threadIdx.x; i <= ng; i += blockDim.x) s_rp[i] = rp[off + i];
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;  // a multiple of Bw (Bw <= 4)
  const int wk = warp % Bw;
  const int b = wk * 32 + lane;
  const int round = s_rnd[b];
  const uint32_t bit = 1u << lane;
  const int vstep = nwarps / Bw;
  long long acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;

  // the 32 trajectories of a warp are fixed, so what a pass needs is too
  const bool w_drop = __any_sync(0xffffffffu, round == RD_DROP);
  const bool w_comp = __any_sync(0xffffffffu, round == RD_COMPLETE);
  const bool w_flip = __any_sync(0xffffffffu, round == RD_FLIP1);
  const bool w_lane = __any_sync(0xffffffffu, round == RD_SWAP || round == RD_FLIP2);
  const bool w_swap = __any_sync(0xffffffffu, round == RD_SWAP);
  const bool w_words = w_drop || w_comp || w_flip;
  const bool w_act = __any_sync(0xffffffffu, round != RD_NONE);
  const int vfirst = warp / Bw;

  // ---------------- pass A: decisions on the snapshot
  NbList cur, nxt;
  if ((w_words || w_lane) && vfirst < ng && w_words) nb_load(cur, s_rp, col, col16, off, vfirst);
  for (int vl = vfirst; (w_words || w_lane) && vl < ng; vl += vstep) {
    if (w_words && vl + vstep < ng) nb_load(nxt, s_rp, col, col16, off, vl + vstep);
    const int64_t v = off + vl;
    const int32_t rs = s_rp[vl], re = s_rp[vl + 1];
    const int64_t e = v * B + b;
    const bool zv = sbit(sW, vl, Bw, b);
    bool dropv = false, addv = false, flipv = false;
    if (w_drop) {
      const uint32_t o = nb_or(cur, sW, col, col16, off, Bw, wk, vl, true);
      dropv = round == RD_DROP && zv && (o & bit);
    }
    if (w_comp) {
      const uint32_t o = nb_or(cur, sF, col, col16, off, Bw, wk, vl, true);
      addv = round == RD_COMPLETE && sbit(sF, vl, Bw, b) && !(o & bit);
    }
    if (w_flip) {
      const uint32_t o = nb_or(cur, sA, col, col16, off, Bw, wk, vl, true);
      flipv = round == RD_FLIP1 && sbit(sA, vl, Bw, b) && !(o & bit);
    }
    if (w_words) cur = nxt;
    const unsigned md = __ballot_sync(0xffffffffu, dropv);
    const unsigned mc = __ballot_sync(0xffffffffu, addv || flipv);
    if (lane == 0) {
      sD[vl * Bw + wk] = md;
      if (mc) sW[vl * Bw + wk] ^= mc;  // complete sets clear bits, flip1 toggles
    }
    acc3 += dropv + addv + flipv;
    if (w_swap) {
      // (1,2)-swap proposal of a set node v (Def. 2.3): the first pair, in
      // CSR order of N(v), of non-adjacent tight neighbours.  The warp first
      // lists each lane's tight neighbours together: a 32-entry chunk of
      // N(v) is loaded at once, and only entries whose tight word has a bit
      // of a proposing lane are broadcast; the pairs of the (short) lists
      // are then tested per lane.
      const unsigned need = __ballot_sync(0xffffffffu, round == RD_SWAP && zv);
      int32_t fa = -1, fb = -1;
      if (need) {
        int32_t tl[kTight];
        int ntl = 0;
        for (int32_t c0 = rs; c0 < re; c0 += 32) {
          const int32_t j = c0 + lane;
          const int32_t u = j < re ? col[j] : -1;
          const uint32_t tw = u >= 0 ? sA[(u - off) * Bw + wk] & need : 0u;
          unsigned m = __ballot_sync(0xffffffffu, tw != 0u);
          while (m) {
            const int i = __ffs(m) - 1;
            m &= m - 1u;
            const int32_t uu = __shfl_sync(0xffffffffu, u, i);
            const uint32_t ww = __shfl_sync(0xffffffffu, tw, i);
            if (ww & bit) {
              if (ntl < kTight) tl[ntl] = uu;
              ++ntl;
            }
          }
        }
        if ((need & bit) && ntl <= kTight) {
          for (int x = 0; x < ntl && fa < 0; ++x)
            for (int y = x + 1; y < ntl; ++y)
              if (!sorted_contains(col, rp[tl[x]], rp[tl[x] + 1], tl[y])) {
                fa = tl[x];
                fb = tl[y];
                break;
              }
        } else if (need & bit) {  // a long tight list: the sequential scan
          for (int32_t i = rs; i < re && fa < 0; ++i) {
            const int32_t a = col[i];
            if (!sbit(sA, a - off, Bw, b)) continue;
            for (int32_t j = i + 1; j < re; ++j) {
              const int32_t cc = col[j];
              if (!sbit(sA, cc - off, Bw, b)) continue;
              if (!sorted_contains(col, rp[a], rp[a + 1], cc)) {
                fa = a;
                fb = cc;
                break;
              }
            }
          }
        }
      }
      if (round == RD_SWAP) {
        S.pa[e] = fa;
        S.pb[e] = fb;
        if (fa >= 0) {
          S.owner[(int64_t)fa * B + b] = (int32_t)v;
          S.owner[(int64_t)fb * B + b] = (int32_t)v;
        }
      }
    }
    if (round == RD_FLIP2) {
      int32_t fb = -1;
      const int32_t ga = S.gain[e];
      for (int32_t j = rs; j < re; ++j) {
        const int32_t u = col[j];
        if (u <= v) continue;
        if (sbit(sW, u - off, Bw, b) == zv) continue;
        const int w = wts ? (int)wts[j] : 1;
        if (ga + S.gain[(int64_t)u * B + b] + 2 * w > 0) {
          fb = u;
          break;
        }
      }
      S.pb[e] = fb;
      if (fb >= 0) {
        atomicMin(&S.owner[e], (int32_t)v);
        atomicMin(&S.owner[(int64_t)fb * B + b], (int32_t)v);
      }
    }
  }
  __syncthreads();

  // ---------------- pass B: commits
  // A proposal commits if no neighbour of its two new nodes (swap) or of
  // its two flipped nodes (2-flip) is claimed by a smaller proposer.  The
  // warp checks one proposing lane at a time, its 32 lanes scanning the two
  // neighbour lists together.
  const bool w_flip2 = __any_sync(0xffffffffu, round == RD_FLIP2);
  for (int vl = vfirst; (w_drop || w_lane) && vl < ng; vl += vstep) {
    const int64_t v = off + vl;
    const int64_t e = v * B + b;
    const unsigned md = sD[vl * Bw + wk];
    if (lane == 0 && md) atomicAnd(&sW[vl * Bw + wk], ~md);
    if (w_swap) {
      const int32_t fa = round == RD_SWAP ? S.pa[e] : -1;
      const int32_t fb = fa >= 0 ? S.pb[e] : -1;
      bool ok = false;
      unsigned pm = __ballot_sync(0xffffffffu, fa >= 0);
      while (pm) {
        const int i = __ffs(pm) - 1;
        pm &= pm - 1u;
        const int32_t ends[2] = {__shfl_sync(0xffffffffu, fa, i), __shfl_sync(0xffffffffu, fb, i)};
        const int bi = wk * 32 + i;
        bool bad = false;
        for (int k = 0; k < 2; ++k)
          for (int32_t j = rp[ends[k]] + lane; j < rp[ends[k] + 1]; j += 32)
            bad |= S.owner[(int64_t)col[j] * B + bi] < (int32_t)v;
        bad = __any_sync(0xffffffffu, bad);
        if (lane == i) ok = !bad;
      }
      if (fa >= 0 && ok) {
        atomicAnd(&sW[vl * Bw + wk], ~bit);
        atomicOr(&sW[(fa - off) * Bw + wk], bit);
        atomicOr(&sW[(fb - off) * Bw + wk], bit);
        acc3 += 1;
      }
    }
    if (w_flip2) {
      const int32_t fb = round == RD_FLIP2 ? S.pb[e] : -1;
      bool ok = fb >= 0 && S.owner[e] == (int32_t)v && S.owner[(int64_t)fb * B + b] == (int32_t)v;
      unsigned pm = __ballot_sync(0xffffffffu, ok);
      while (pm) {
        const int i = __ffs(pm) - 1;
        pm &= pm - 1u;
        const int32_t f = __shfl_sync(0xffffffffu, fb, i);
        const int32_t ends[2] = {(int32_t)v, f};
        const int bi = wk * 32 + i;
        bool bad = false;
        for (int k = 0; k < 2; ++k)
          for (int32_t j = rp[ends[k]] + lane; j < rp[ends[k] + 1]; j += 32) {
            const int32_t y = col[j];
            if (y != (int32_t)v && y != f) bad |= S.owner[(int64_t)y * B + bi] < (int32_t)v;
          }
        bad = __any_sync(0xffffffffu, bad);
        if (lane == i) ok = !bad;
      }
      if (ok) {
        atomicXor(&sW[vl * Bw + wk], bit);
        atomicXor(&sW[(fb - off) * Bw + wk], bit);
        acc3 += 1;
      }
    }
  }
  __syncthreads();

  // ---------------- pass C: counts of the (new) work set
  const bool act = round != RD_NONE;
  if (w_act && mis && vfirst < ng) nb_load(cur, s_rp, col, col16, off, vfirst);
  for (int vl = vfirst; w_act && vl < ng; vl += vstep) {
    if (mis && vl + vstep < ng) nb_load(nxt, s_rp, col, col16, off, vl + vstep);
    const int64_t v = off + vl;
    const int32_t rs = s_rp[vl], re = s_rp[vl + 1];
    const int64_t e = v * B + b;
    const bool zv = sbit(sW, vl, Bw, b);
    bool aux = false, fr = false;
    if (act) S.owner[e] = 0x7fffffff;
    if (mis) {
      uint32_t once, twice;
      nb_once_twice(cur, sW, col, col16, off, Bw, wk, once, twice);
      cur = nxt;
      if (act) {
        const bool one = (once & bit) != 0, two = (twice & bit) != 0;
        acc0 += zv;
        acc1 += zv && one;
        fr = !zv && !one;
        acc2 += fr;
        aux = !zv && one && !two;
      }
    } else if (act) {
      int P = 0, W = 0;
      for (int32_t j = rs; j < re; ++j) {
        const int w = wts ? (int)wts[j] : 1;
        W += w;
        if (sbit(sW, local_col(col, col16, off, j), Bw, b)) P += w;
      }
      const int as = 2 * P - W;
      acc0 += zv ? (W - P) : P;
      acc1 += !(zv ? (as <= -1) : (as >= 0));  // f_B rule (Thm 3.6), any objective
      const int gn = zv ? as : -as;
      acc2 += gn > 0;
      S.gain[e] = gn;
      aux = gn > 0;
    }
    const unsigned ma = __ballot_sync(0xffffffffu, act);
    const unsigned mx = __ballot_sync(0xffffffffu, aux);
    const unsigned mf = __ballot_sync(0xffffffffu, fr);
    if (lane == 0 && ma) {
      sA[vl * Bw + wk] = (sA[vl * Bw + wk] & ~ma) | (mx & ma);
      if (mis) sF[vl * Bw + wk] = (sF[vl * Bw + wk] & ~ma) | (mf & ma);
    }
  }
  if (acc0) atomicAdd(&s_cnt[4 * b + 0], (unsigned long long)acc0);
  if (acc1) atomicAdd(&s_cnt[4 * b + 1], (unsigned long long)acc1);
  if (acc2) atomicAdd(&s_cnt[4 * b + 2], (unsigned long long)acc2);
  if (acc3) atomicAdd(&s_cnt[4 * b + 3], (unsigned long long)acc3);
  __syncthreads();

  for (int i = threadIdx.x; i < nw; i += blockDim.x) {
    const int64_t gi = (int64_t)off * Bw + i;
    S.Zwork[gi] = sW[i];
    S.Zaux[gi] = sA[i];
    S.Zfree[gi] = sF[i];
  }
  for (int i = threadIdx.x; i < 4 * B; i += blockDim.x) {
    const unsigned long long val = s_cnt[i];
    if (val) {
      Counters* c = S.cnt + ((int64_t)g * B + i / 4) * S.R;  // replica 0
      const int k = i & 3;
      unsigned long long* p = k == 0 ? &c->value : k == 1 ? &c->a : k == 2 ? &c->b : &c->commits;
      atomicAdd(p, val);
    }
  }
}

size_t disc_graph_smem_bytes(int B, int max_ng) {
  const size_t nw = (size_t)max_ng * ((B + 31) / 32);
  return 4 * nw * 4 + (size_t)((B + 1) & ~1) * 4 + 4 * (size_t)B * 8 + ((size_t)max_ng + 1) * 4;
}

cudaError_t launch_disc_graph(const SolverDev& S, size_t smem, cudaStream_t stream) {
  cudaFuncSetAttribute(k_disc_graph, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_disc_graph<<<S.g.num_graphs, kDgThreads, smem, stream>>>(S);
  return cudaGetLastError();
}

}  // namespace mqo
