// mqo_tick.cu -- the per-trajectory machine of Alg. 1 / Alg. 2 on the GPU.
//
// One tick = (pool mode: the graphs' pool decisions, mqo_pool.cu ->)
// control (one thread, or one warp, per trajectory) -> apply (accept copies,
// resets, initialisations) -> fused descent step -> discrete round passes
// A, B and the count pass C (or the fused per-graph kernel,
// mqo_disc_graph.cu) -> tick end.  The control kernel decides, from the
// exact counters of the previous tick, what each trajectory does now; the
// node-parallel kernels then act on (node, trajectory) pairs.  Member
// graphs with nothing to do in a pass are skipped through per-graph tick
// stamps written by the control kernel.
//
// Pair kernels map thread -> (node v, trajectory b), trajectory fastest,
// one CTA per item (<= 256 nodes of one member graph), or a slice of an item
// per CTA when there are few items (item_slice).  The lanes that
// share one bit word of a node (G = min(B,32) lanes) form a group; MIS set
// logic is done on whole words: the group splits v's neighbour list, ORs
// (or once/twice-accumulates) the neighbours' words and reduces by shuffles.
#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

// ---------------------------------------------------------------- control
struct CtrlArgs {
  SolverDev S;
  int mode;
  const uint8_t* mask;
};

__device__ __forceinline__ void reset_keys(const Params& p, int64_t tau, int32_t o, int32_t r, int32_t n_g,
                                           TrajState& st) {
  const U64x4 k = philox4x64_10(TAG_RESET, (uint64_t)o, (uint64_t)r, 0ULL, p.seed, (uint64_t)tau);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    st.rkeys[2 * i] = (uint32_t)(k.v[i] & 0xffffffffULL);
    st.rkeys[2 * i + 1] = (uint32_t)(k.v[i] >> 32);
  }
  st.rk = (int64_t)floor(p.rho * (double)n_g);
}

// The control step of trajectory tau; c = its counters of the previous tick
// (all replicas summed; not used by a forced reset).
__device__ __forceinline__ void ctrl_one(const CtrlArgs& A, int64_t tau, const Counters& c) {
  const SolverDev& S = A.S;
  const int64_t t = *S.tick;
  const int g = (int)(tau / S.B);
  const int32_t n_g = S.g.node_off[g + 1] - S.g.node_off[g];
  const Params& p = S.p;
  const bool mis = p.problem == PROB_MIS;
  TrajState st = S.st[tau];
  int act = 0;
  int round = RD_NONE;

  auto accept = [&](int bit, int64_t value, bool from_ls) {
    if (value > st.best) {
      credit_gain(st, value, from_ls);
      st.best = value;
      act |= bit;
      st.accepts += 1;
    }
  };

  if (A.mode == CTRL_RESET) {
    // forced reset (mqo_reset): round r+1 from the best set, new descent;
    // the counters of the last tick stay in place
    if (A.mask == nullptr || A.mask[tau]) {
      st.r += 1;
      st.s = 0;
      st.phase = PH_DESCENT;
      reset_keys(p, tau, st.o, st.r, n_g, st);
      act = ACT_RESET;
    }
    st.act = act;
    st.round = RD_NONE;
    S.st[tau] = st;
    S.act[tau] = act;
    S.rnd[tau] = RD_NONE;
    if (act) {
      S.gflag[g] = (int32_t)(t + 1);
      S.any[0] = (int32_t)(t + 1);
    }
    return;
  }

  // fold the previous tick's exact counters (summed and cleared by the
  // caller); in pool mode a trajectory that waited last tick keeps its
  // evaluation
  const bool pool = p.pool_k > 0 && A.mode == CTRL_MACHINE;
  if (!pool || (st.act & ACT_STEP) || st.round != RD_NONE) {
    const int64_t cv = (int64_t)c.value;
    st.ev_value = mis ? cv : cv / 2;
    st.ev_a = (int64_t)c.a;
    st.ev_b = (int64_t)c.b;
    st.last_commits = (int64_t)c.commits;
  }

  if (A.mode == CTRL_LS_BEGIN) {
    st.ls_done = 0;
    act = ACT_WORK_BEST;
    round = RD_COUNT;
    st.last_round = RD_COUNT;
  } else if (A.mode == CTRL_LS) {
    if (!st.ls_done) {
      bool done;
      if (mis) {
        if (st.ev_b > 0) { round = RD_COMPLETE; done = false; }
        else if (!(st.last_round == RD_SWAP && st.last_commits == 0)) { round = RD_SWAP; done = false; }
        else done = true;
      } else {
        if (st.ev_b > 0) { round = RD_FLIP1; done = false; }
        else if (!(st.last_round == RD_FLIP2 && st.last_commits == 0)) { round = RD_FLIP2; done = false; }
        else done = true;
      }
      if (done) {
        accept(ACT_ACC_WORK, st.ev_value, true);
        st.ls_done = 1;
        round = RD_NONE;
      }
      st.last_round = round;
    }
  } else if (pool) {
    // ----- pmQO (Alg. 3/4): the per-trajectory part of the graph's
    // decision of this tick (k_pool_ctrl) -----
    const PoolState ps = S.pool[g];
    const int b = (int)(tau - (int64_t)g * S.B);
    if (ps.best_src >= 0) {  // the graph's best set was replaced (steps 5, 12, 13)
      credit_gain(st, ps.best, ps.best_src >= S.K);
      st.best = ps.best;
      st.accepts += 1;
    }
    auto hold = [&](int bits, int64_t value) {
      act |= bits;
      st.held = value;
      st.phase = PH_WAIT;
    };
    if (st.phase == PH_WAIT) {
      if (ps.dec == DEC_NEXT) {  // steps 6-10 from pool member pbase[tau]
        st.r += 1;
        st.s = 0;
        st.phase = PH_DESCENT;
        reset_keys(p, tau, st.o, st.r, n_g, st);
        act |= ACT_RESET | ACT_POOL;
      } else if (ps.dec == DEC_LS) {  // step 13
        st.held = (int64_t)(-9223372036854775807LL - 1);
        if (mis ? b == 0 : b < ps.count) {
          st.phase = PH_LS;
          act |= mis ? ACT_WORK_BEST : (ACT_WORK_BEST | ACT_POOL);
          round = RD_COUNT;
        }
      } else if (ps.dec == DEC_OUTER) {  // step 2
        st.held = (int64_t)(-9223372036854775807LL - 1);
        st.o += 1;
        st.r = 0;
        st.s = 0;
        st.phase = PH_DESCENT;
        act |= ACT_INIT;
      }
    } else if (st.phase == PH_DESCENT) {
      if (st.s > 0) {
        const bool pass = mis ? (st.ev_a == 0 && st.ev_b == 0) : (st.ev_a == 0);
        if (pass) {
          st.descents += 1;
          hold(ACT_WORK_ZX, st.ev_value);
        } else if (st.s >= p.cap) {
          st.descents += 1;
          if (mis && p.repair) {
            st.phase = PH_REPAIR;
            act |= ACT_WORK_ZX;
            round = RD_COUNT;
          } else {
            // an unrepaired capped MIS point is not a candidate
            hold(ACT_WORK_ZX, mis ? (int64_t)(-9223372036854775807LL - 1) : st.ev_value);
          }
        }
      }
    } else if (st.phase == PH_REPAIR) {
      if (st.ev_a > 0) round = RD_DROP;
      else if (st.ev_b > 0) round = RD_COMPLETE;
      else hold(0, st.ev_value);
    } else if (st.phase == PH_LS) {
      bool done;
      if (mis) {
        if (st.ev_b > 0) { round = RD_COMPLETE; done = false; }
        else if (!(st.last_round == RD_SWAP && st.last_commits == 0)) { round = RD_SWAP; done = false; }
        else done = true;
      } else {
        if (st.ev_b > 0) { round = RD_FLIP1; done = false; }
        else if (!(st.last_round == RD_FLIP2 && st.last_commits == 0)) { round = RD_FLIP2; done = false; }
        else done = true;
      }
      if (done) {
        hold(0, st.ev_value);
        round = RD_NONE;
      }
    }
    if (st.phase == PH_DESCENT) {
      act |= ACT_STEP;
      st.s += 1;
      st.steps += 1;
      st.last_round = RD_NONE;
      round = RD_NONE;
    } else if (round != RD_NONE) {
      st.last_round = round;
    }
    st.ticks += 1;
  } else {
    // ----- the machine (same decisions as the oracle's control step) -----
    auto start_outer = [&]() {
      st.o += 1;
      st.r = 0;
      st.s = 0;
      st.phase = PH_DESCENT;
      act |= ACT_INIT;
    };
    auto after_accept = [&]() -> int {
      if (st.r < p.t_gs) {
        st.r += 1;
        st.s = 0;
        st.phase = PH_DESCENT;
        reset_keys(p, tau, st.o, st.r, n_g, st);
        act |= ACT_RESET;
        return RD_NONE;
      }
      if (p.local_search) {
        st.phase = PH_LS;
        act |= ACT_WORK_BEST;
        return RD_COUNT;
      }
      start_outer();
      return RD_NONE;
    };
    if (st.phase == PH_DESCENT) {
      if (st.s > 0) {
        const bool pass = mis ? (st.ev_a == 0 && st.ev_b == 0) : (st.ev_a == 0);
        if (pass) {
          st.descents += 1;
          accept(ACT_ACC_ZX, st.ev_value, false);
          round = after_accept();
        } else if (st.s >= p.cap) {
          st.descents += 1;
          if (mis) {
            if (p.repair) {
              st.phase = PH_REPAIR;
              act |= ACT_WORK_ZX;
              round = RD_COUNT;
            } else {
              round = after_accept();
            }
          } else {
            accept(ACT_ACC_ZX, st.ev_value, false);
            round = after_accept();
          }
        }
      }
    } else if (st.phase == PH_REPAIR) {
      if (st.ev_a > 0) round = RD_DROP;
      else if (st.ev_b > 0) round = RD_COMPLETE;
      else {
        accept(ACT_ACC_WORK, st.ev_value, false);
        round = after_accept();
      }
    } else if (st.phase == PH_LS) {
      bool done;
      if (mis) {
        if (st.ev_b > 0) { round = RD_COMPLETE; done = false; }
        else if (!(st.last_round == RD_SWAP && st.last_commits == 0)) { round = RD_SWAP; done = false; }
        else done = true;
      } else {
        if (st.ev_b > 0) { round = RD_FLIP1; done = false; }
        else if (!(st.last_round == RD_FLIP2 && st.last_commits == 0)) { round = RD_FLIP2; done = false; }
        else done = true;
      }
      if (done) {
        accept(ACT_ACC_WORK, st.ev_value, true);
        start_outer();
        round = RD_NONE;
      }
    }
    if (st.phase == PH_DESCENT) {
      act |= ACT_STEP;
      st.s += 1;
      st.steps += 1;
      st.last_round = RD_NONE;
      round = RD_NONE;
    } else {
      st.last_round = round;
    }
    st.ticks += 1;
  }
  st.act = act;
  st.round = round;
  S.st[tau] = st;
  S.act[tau] = act;
  S.rnd[tau] = round;
  S.bestv[tau] = st.best;
  const int32_t stamp = (int32_t)(t + 1);
  const int G = S.g.num_graphs;
  if (act & ACT_APPLY_MASK) {
    S.gflag[g] = stamp;
    S.any[0] = stamp;
  }
  if (round != RD_NONE) {
    S.gflag[G + g] = stamp;
    S.any[1] = stamp;
  }
  if (act & ACT_STEP) {
    S.gflag[2 * G + g] = stamp;
    S.any[2] = stamp;
  }
}

// one thread per trajectory: few counter replicas
__global__ void k_ctrl(CtrlArgs A) {
  const SolverDev& S = A.S;
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  const int64_t tau = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tau >= T) return;
  Counters c{0ull, 0ull, 0ull, 0ull};
  if (A.mode != CTRL_RESET) {  // a forced reset leaves the counters in place
    c = sum_replicas(S.cnt, tau, S.R);
    for (int r = 0; r < S.R; ++r) S.cnt[tau * S.R + r] = Counters{0ull, 0ull, 0ull, 0ull};
  }
  ctrl_one(A, tau, c);
}

// one warp per trajectory: the lanes sum and clear the R replicas together
__global__ void k_ctrl_w(CtrlArgs A) {
  const SolverDev& S = A.S;
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  const int64_t tau = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (tau >= T) return;
  Counters c{0ull, 0ull, 0ull, 0ull};
  if (A.mode != CTRL_RESET) {
    for (int r = lane; r < S.R; r += 32) {
      const Counters x = S.cnt[tau * S.R + r];
      c.value += x.value;
      c.a += x.a;
      c.b += x.b;
      c.commits += x.commits;
      S.cnt[tau * S.R + r] = Counters{0ull, 0ull, 0ull, 0ull};
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c.value += __shfl_xor_sync(0xffffffffu, c.value, o);
      c.a += __shfl_xor_sync(0xffffffffu, c.a, o);
      c.b += __shfl_xor_sync(0xffffffffu, c.b, o);
      c.commits += __shfl_xor_sync(0xffffffffu, c.commits, o);
    }
  }
  if (lane == 0) ctrl_one(A, tau, c);
}

cudaError_t launch_ctrl(const SolverDev& S, int mode, const uint8_t* mask, cudaStream_t stream) {
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  CtrlArgs a{S, mode, mask};
  if (S.R >= 8) k_ctrl_w<<<(unsigned)((T * 32 + 255) / 256), 256, 0, stream>>>(a);
  else k_ctrl<<<(unsigned)((T + 127) / 128), 128, 0, stream>>>(a);
  return cudaGetLastError();
}

__global__ void k_tick_end(int64_t* tick) { *tick += 1; }

cudaError_t launch_tick_end(const SolverDev& S, cudaStream_t stream) {
  k_tick_end<<<1, 1, 0, stream>>>(S.tick);
  return cudaGetLastError();
}

// ------------------------------------------------------- pair-kernel frame
struct PairCtx {
  int g;
  int64_t v;
  int b;
  int64_t tau;
  bool in;
  int gl;          // lane within the word group
  int G;           // group size min(B, 32)
  unsigned gmask;  // lanes of the group
  int wk;          // word index of the group inside the node
};

// Walk the (node, trajectory) pairs of one item; warp w covers pair
// indices [v0*B + 32k, ...) so that each group holds one whole bit word.
// `body(ctx)` is called by all 32 lanes together.
template <typename Body>
__device__ __forceinline__ void item_pairs(const SolverDev& S, const Item& item, Body body) {
  const int B = S.B;
  const int lane = threadIdx.x & 31;
  const int G = B < 32 ? B : 32;
  const int gbase = lane & ~(G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gbase);
  const int64_t lo = (int64_t)item.v0 * B, hi = (int64_t)item.v1 * B;
  for (int64_t base = lo + (threadIdx.x & ~31); base < hi; base += blockDim.x) {
    const int64_t idx = base + lane;
    PairCtx c;
    c.in = idx < hi;
    c.v = c.in ? idx / B : (int64_t)item.v0;
    c.b = (int)(idx % B);
    c.g = item.g;
    c.tau = (int64_t)item.g * B + c.b;
    c.gl = lane - gbase;
    c.G = G;
    c.gmask = gmask;
    c.wk = c.b >> 5;
    body(c);
  }
}

// OR over the neighbours u of v (only u < v if `less`) of word wk, computed
// by the lanes of a group together.
__device__ __forceinline__ uint32_t group_nb_or(const SolverDev& S, const uint32_t* words, const PairCtx& c,
                                                bool less) {
  const int32_t* rp = S.g.row_ptr;
  const int32_t* col = S.g.col;
  uint32_t r = 0u;
  for (int32_t j = rp[c.v] + c.gl; j < rp[c.v + 1]; j += c.G) {
    const int32_t u = col[j];
    if (less && u >= c.v) break;  // rows are sorted ascending
    r |= words[(int64_t)u * S.Bw + c.wk];
  }
  for (int o = 1; o < c.G; o <<= 1) r |= __shfl_xor_sync(c.gmask, r, o);
  return r;
}

// ---------------------------------------------------------------- apply
// Each CTA (one item) first lists the trajectories of its member graph that
// have an apply action this tick, then visits only those (node, trajectory)
// pairs, node fastest.  Bit updates are atomic (several listed trajectories
// may touch the same node's word).
__device__ __forceinline__ void set_bit_atomic(uint32_t* words, int64_t v, int Bw, int b, bool val) {
  uint32_t* wp = words + v * Bw + (b >> 5);
  const uint32_t bit = 1u << (b & 31);
  if (val) atomicOr(wp, bit);
  else atomicAnd(wp, ~bit);
}

// Each CTA (a slice of one item) first lists, in increasing order, the
// trajectories of its member graph that have an apply action this tick and
// caches their actions, reset keys and bases in shared memory; it then visits
// only those (node, trajectory) pairs, trajectory fastest, so that the x and V
// writes of one node's listed trajectories are adjacent.  Bit updates are
// atomic (several listed trajectories share a node's word).
__global__ void __launch_bounds__(kPairThreads) k_apply(SolverDev S) {
  __shared__ int s_list[128];
  __shared__ int s_act[128];
  __shared__ uint32_t s_keys[128][6];
  __shared__ int64_t s_rk[128];
  __shared__ int32_t s_o[128];
  __shared__ int32_t s_pb[128];
  __shared__ int s_wcnt[4];
  const int64_t t = *S.tick;
  if (S.any[0] != (int32_t)(t + 1)) return;
  int it;
  Item item;
  if (!item_slice(S, it, item)) return;
  if (S.gflag[item.g] != (int32_t)(t + 1)) return;
  const int B = S.B, Bw = S.Bw;
  const int g = item.g;
  // ordered compaction of the acting trajectories (B <= 128: warps 0..3)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int myact = 0;
  if (threadIdx.x < B) myact = S.act[(int64_t)g * B + threadIdx.x];
  const bool on = threadIdx.x < B && (myact & ACT_APPLY_MASK);
  const unsigned bal = __ballot_sync(0xffffffffu, on);
  if (warp < 4 && lane == 0) s_wcnt[warp] = __popc(bal);
  __syncthreads();
  if (on) {
    int pos = __popc(bal & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) pos += s_wcnt[w];
    const int64_t tau = (int64_t)g * B + threadIdx.x;
    s_list[pos] = threadIdx.x;
    s_act[pos] = myact;
    if (myact & ACT_RESET) {
      const TrajState& st = S.st[tau];
#pragma unroll
      for (int i = 0; i < 6; ++i) s_keys[pos][i] = st.rkeys[i];
      s_rk[pos] = st.rk;
    }
    if (myact & ACT_INIT) s_o[pos] = S.st[tau].o;
    s_pb[pos] = (myact & ACT_POOL) ? S.pbase[tau] : -1;
  }
  __syncthreads();
  const int nact = s_wcnt[0] + s_wcnt[1] + s_wcnt[2] + s_wcnt[3];
  const int nodes = item.v1 - item.v0;
  const bool mis = S.p.problem == PROB_MIS;
  const float thr = mis ? 0.5f : 0.0f;
  void* Xc = (t & 1) ? S.X1 : S.X0;
  uint32_t* Zc = (t & 1) ? S.ZX1 : S.ZX0;
  const uint32_t* Zp = (t & 1) ? S.ZX0 : S.ZX1;  // rounding of the x the last step evaluated
  const int32_t off = S.g.node_off[g];
  const uint32_t n_g = (uint32_t)(S.g.node_off[g + 1] - off);
  for (int idx = threadIdx.x; idx < nact * nodes; idx += blockDim.x) {
    const int j = idx % nact;
    const int b = s_list[j];
    const int64_t v = item.v0 + idx / nact;
    const int64_t tau = (int64_t)g * B + b;
    const int act = s_act[j];
    bool zb = get_bit(S.Zbest, v, Bw, b);
    if (act & (ACT_ACC_ZX | ACT_ACC_WORK)) {
      const bool src = (act & ACT_ACC_ZX) ? get_bit(Zp, v, Bw, b) : get_bit(S.Zwork, v, Bw, b);
      if (src != zb) set_bit_atomic(S.Zbest, v, Bw, b, src);
      zb = src;
    }
    // pool mode: the base of a reset / local search is pool member pbase[tau]
    bool base = zb;
    if (act & ACT_POOL) {
      const int32_t k = s_pb[j];
      base = k >= 0 && ((S.Pool[v * S.Kw + (k >> 5)] >> (k & 31)) & 1u);
    }
    if (act & (ACT_WORK_ZX | ACT_WORK_BEST)) {
      const bool wv = (act & ACT_WORK_ZX) ? get_bit(Zp, v, Bw, b) : base;
      set_bit_atomic(S.Zwork, v, Bw, b, wv);
    }
    if (act & (ACT_RESET | ACT_INIT)) {
      const uint32_t vl = (uint32_t)(v - off);
      float x;
      if (act & ACT_RESET) {
        x = base ? 1.0f : (mis ? 0.0f : -1.0f);
        // v in R sets x_v = 0: only needed where x_v is not 0 already (for
        // MIS the nodes of the base set, a few percent of the graph)
        if (x != 0.0f && (int64_t)feistel_sigma(n_g, s_keys[j], vl) < s_rk[j]) x = 0.0f;
      } else {
        const Params& p = S.p;
        const U64x4 r = philox4x64_10(TAG_INIT, (uint64_t)s_o[j], (uint64_t)vl, 0ULL, p.seed, (uint64_t)tau);
        const float lo = mis ? 0.0f : -1.0f, hi = 1.0f;
        if (p.init_kind == 0) {
          const float u = unit24(r.v[0]);
          x = lo + (hi - lo) * u;
        } else {
          const int32_t d = S.g.row_ptr[v + 1] - S.g.row_ptr[v];
          const int32_t dm = S.g.dmax[g];
          const float q = dm > 0 ? (float)d / (float)dm : 0.0f;
          float base = 1.0f - q;
          if (!mis) base = 2.0f * base - 1.0f;
          float s = unit24(r.v[0]) + unit24(r.v[1]);
          s = s + unit24(r.v[2]);
          s = s + unit24(r.v[3]);
          s = s - 2.0f;
          float eps = s * 1.7320508075688772f;
          eps = p.sigma * eps;
          x = clamp_box(base + eps, lo, hi);
        }
      }
      const int64_t e = v * B + b;
      if (S.p.x_dtype == DT_F32) {
        static_cast<float*>(Xc)[e] = x;
      } else if (S.p.x_dtype == DT_BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        static_cast<__nv_bfloat16*>(Xc)[e] = h;
        x = __bfloat162float(h);
      } else {
        const __half h = __float2half_rn(x);
        static_cast<__half*>(Xc)[e] = h;
        x = __half2float(h);
      }
      if (S.p.v_dtype == DT_F32) static_cast<float*>(S.V)[e] = 0.0f;
      else if (S.p.v_dtype == DT_BF16) static_cast<__nv_bfloat16*>(S.V)[e] = __float2bfloat16_rn(0.0f);
      else static_cast<__half*>(S.V)[e] = __float2half_rn(0.0f);
      set_bit_atomic(Zc, v, Bw, b, x > thr);
    }
  }
}

cudaError_t launch_apply(const SolverDev& S, cudaStream_t stream) {
  k_apply<<<S.g.num_items * S.split, kPairThreads, 0, stream>>>(S);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- discrete rounds
__device__ __forceinline__ void flush_pair_counters(const SolverDev& S, unsigned long long* s_cnt, int g, int it,
                                                    Counters* dst) {
  __syncthreads();
  const int B = S.B;
  const int rep = it % S.R;
  for (int i = threadIdx.x; i < 4 * B; i += blockDim.x) {
    const unsigned long long val = s_cnt[i];
    if (val) {
      Counters* c = dst + ((int64_t)g * B + i / 4) * S.R + rep;
      const int k = i & 3;
      unsigned long long* p = k == 0 ? &c->value : k == 1 ? &c->a : k == 2 ? &c->b : &c->commits;
      atomicAdd(p, val);
    }
  }
}

// pass 0 = A (decide / propose), 1 = B (commit), 2 = C (count)
__global__ void __launch_bounds__(kPairThreads) k_disc(SolverDev S, int pass) {
  __shared__ unsigned long long s_cnt[4 * 128];
  const int64_t t = *S.tick;
  if (S.any[1] != (int32_t)(t + 1)) return;
  int it;
  Item item;
  if (!item_slice(S, it, item)) return;
  const int G = S.g.num_graphs;
  if (S.gflag[G + item.g] != (int32_t)(t + 1)) return;
  const int B = S.B, Bw = S.Bw;
  const bool mis = S.p.problem == PROB_MIS;
  const int32_t* rp = S.g.row_ptr;
  const int32_t* col = S.g.col;
  const int8_t* wts = S.g.w;
  for (int i = threadIdx.x; i < 4 * B; i += blockDim.x) s_cnt[i] = 0ull;
  __syncthreads();
  long long acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
  int my_b = (int)(threadIdx.x % B);
  item_pairs(S, item, [&](const PairCtx& c) {
    const int64_t v = c.v;
    const int b = c.b;
    const int round = c.in ? S.rnd[c.tau] : RD_NONE;
    const int64_t e = v * B + b;
    const int32_t rs = rp[v], re = rp[v + 1];
    const uint32_t bit = 1u << (b & 31);
    if (pass == 0) {
      // ---------------- pass A
      const bool zv = get_bit(S.Zwork, v, Bw, b);
      const bool need_drop = __any_sync(c.gmask, round == RD_DROP);
      const bool need_comp = __any_sync(c.gmask, round == RD_COMPLETE);
      const bool need_flip = __any_sync(c.gmask, round == RD_FLIP1);
      bool dropv = false, addv = false, flipv = false;
      if (need_drop) {
        const uint32_t o = group_nb_or(S, S.Zwork, c, true);
        dropv = round == RD_DROP && zv && (o & bit);
      }
      if (need_comp) {
        const uint32_t o = group_nb_or(S, S.Zfree, c, true);
        addv = round == RD_COMPLETE && get_bit(S.Zfree, v, Bw, b) && !(o & bit);
      }
      if (need_flip) {
        const uint32_t o = group_nb_or(S, S.Zaux, c, true);
        flipv = round == RD_FLIP1 && get_bit(S.Zaux, v, Bw, b) && !(o & bit);
      }
      update_word(S.Zdrop, v, Bw, b, B, dropv, round == RD_DROP);
      // complete sets bits, flip1 toggles: both are own-word updates
      update_word(S.Zwork, v, Bw, b, B, addv ? true : !zv, addv || flipv);
      acc3 += dropv + addv + flipv;
      if (round == RD_SWAP) {
        int32_t fa = -1, fb = -1;
        if (zv) {
          for (int32_t i = rs; i < re && fa < 0; ++i) {
            const int32_t a = col[i];
            if (!get_bit(S.Zaux, a, Bw, b)) continue;
            for (int32_t j = i + 1; j < re; ++j) {
              const int32_t cc = col[j];
              if (!get_bit(S.Zaux, cc, Bw, b)) continue;
              if (!sorted_contains(col, rp[a], rp[a + 1], cc)) { fa = a; fb = cc; break; }
            }
          }
        }
        S.pa[e] = fa;
        S.pb[e] = fb;
        if (fa >= 0) {
          S.owner[(int64_t)fa * B + b] = (int32_t)v;
          S.owner[(int64_t)fb * B + b] = (int32_t)v;
        }
      }
      if (round == RD_FLIP2) {
        int32_t fb = -1;
        const int32_t ga = S.gain[e];
        for (int32_t j = rs; j < re; ++j) {
          const int32_t u = col[j];
          if (u <= v) continue;
          if (get_bit(S.Zwork, u, Bw, b) == zv) continue;
          const int w = wts ? (int)wts[j] : 1;
          if (ga + S.gain[(int64_t)u * B + b] + 2 * w > 0) { fb = u; break; }
        }
        S.pb[e] = fb;
        if (fb >= 0) {
          atomicMin(&S.owner[e], (int32_t)v);
          atomicMin(&S.owner[(int64_t)fb * B + b], (int32_t)v);
        }
      }
    } else if (pass == 1) {
      // ---------------- pass B
      const bool dv = round == RD_DROP && get_bit(S.Zdrop, v, Bw, b);
      update_word_atomic(S.Zwork, v, Bw, b, B, false, dv);
      if (round == RD_SWAP) {
        const int32_t fa = S.pa[e];
        if (fa >= 0) {
          const int32_t fb = S.pb[e];
          bool ok = true;
          const int32_t ends[2] = {fa, fb};
          for (int k = 0; k < 2 && ok; ++k) {
            const int32_t x = ends[k];
            for (int32_t j = rp[x]; j < rp[x + 1]; ++j) {
              const int32_t o = S.owner[(int64_t)col[j] * B + b];
              if (o < (int32_t)v) { ok = false; break; }
            }
          }
          if (ok) {
            atomicAnd(&S.Zwork[v * Bw + (b >> 5)], ~bit);
            atomicOr(&S.Zwork[(int64_t)fa * Bw + (b >> 5)], bit);
            atomicOr(&S.Zwork[(int64_t)fb * Bw + (b >> 5)], bit);
            acc3 += 1;
          }
        }
      }
      if (round == RD_FLIP2) {
        const int32_t fb = S.pb[e];
        if (fb >= 0) {
          bool ok = S.owner[e] == (int32_t)v && S.owner[(int64_t)fb * B + b] == (int32_t)v;
          const int32_t ends[2] = {(int32_t)v, fb};
          for (int k = 0; k < 2 && ok; ++k) {
            const int32_t x = ends[k];
            for (int32_t j = rp[x]; j < rp[x + 1]; ++j) {
              const int32_t y = col[j];
              if (y == (int32_t)v || y == fb) continue;
              if (S.owner[(int64_t)y * B + b] < (int32_t)v) { ok = false; break; }
            }
          }
          if (ok) {
            atomicXor(&S.Zwork[v * Bw + (b >> 5)], bit);
            atomicXor(&S.Zwork[(int64_t)fb * Bw + (b >> 5)], bit);
            acc3 += 1;
          }
        }
      }
    } else {
      // ---------------- pass C: counts of the (new) work set
      const bool act = round != RD_NONE;
      const bool zv = get_bit(S.Zwork, v, Bw, b);
      bool aux = false, fr = false;
      if (act) S.owner[e] = 0x7fffffff;
      if (mis) {
        if (__any_sync(c.gmask, act)) {
          // once / twice: neighbours with the bit set at least once / twice
          uint32_t once = 0u, twice = 0u;
          for (int32_t j = rs + c.gl; j < re; j += c.G) {
            const uint32_t w = S.Zwork[(int64_t)col[j] * Bw + c.wk];
            twice |= once & w;
            once |= w;
          }
          for (int o = 1; o < c.G; o <<= 1) {
            const uint32_t o2 = __shfl_xor_sync(c.gmask, once, o);
            const uint32_t t2 = __shfl_xor_sync(c.gmask, twice, o);
            twice = twice | t2 | (once & o2);
            once |= o2;
          }
          if (act) {
            const bool one = (once & bit) != 0, two = (twice & bit) != 0;
            acc0 += zv;
            acc1 += zv && one;
            fr = !zv && !one;
            acc2 += fr;
            aux = !zv && one && !two;  // tight: exactly one neighbour in the set
          }
        }
      } else if (act) {
        int P = 0, W = 0;
        for (int32_t j = rs; j < re; ++j) {
          const int w = wts ? (int)wts[j] : 1;
          W += w;
          if (get_bit(S.Zwork, col[j], Bw, b)) P += w;
        }
        const int as = 2 * P - W;
        acc0 += zv ? (W - P) : P;
        const bool fixed = zv ? (as <= -1) : (as >= 0);  // f_B rule (Thm 3.6), any objective
        acc1 += !fixed;
        const int gn = zv ? as : -as;
        acc2 += gn > 0;
        S.gain[e] = gn;
        aux = gn > 0;
      }
      update_word(S.Zaux, v, Bw, b, B, aux, act);
      update_word(S.Zfree, v, Bw, b, B, fr, act && mis);
    }
  });
  if (acc0) atomicAdd(&s_cnt[4 * my_b + 0], (unsigned long long)acc0);
  if (acc1) atomicAdd(&s_cnt[4 * my_b + 1], (unsigned long long)acc1);
  if (acc2) atomicAdd(&s_cnt[4 * my_b + 2], (unsigned long long)acc2);
  if (acc3) atomicAdd(&s_cnt[4 * my_b + 3], (unsigned long long)acc3);
  flush_pair_counters(S, s_cnt, item.g, it, S.cnt);
}

cudaError_t launch_disc(const SolverDev& S, int pass, cudaStream_t stream) {
  k_disc<<<S.g.num_items * S.split, kPairThreads, 0, stream>>>(S, pass);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- readouts
__global__ void __launch_bounds__(kPairThreads) k_round_bits(SolverDev S, uint32_t* z) {
  const int64_t t = *S.tick;
  const void* Xc = (t & 1) ? S.X1 : S.X0;
  const bool mis = S.p.problem == PROB_MIS;
  const float thr = mis ? 0.5f : 0.0f;
  const Item item = S.g.items[blockIdx.x];
  item_pairs(S, item, [&](const PairCtx& c) {
    float x = 0.0f;
    if (c.in) {
      const int64_t e = c.v * S.B + c.b;
      if (S.p.x_dtype == DT_F32) x = static_cast<const float*>(Xc)[e];
      else if (S.p.x_dtype == DT_BF16) x = __bfloat162float(static_cast<const __nv_bfloat16*>(Xc)[e]);
      else x = __half2float(static_cast<const __half*>(Xc)[e]);
    }
    update_word(z, c.v, S.Bw, c.b, S.B, x > thr, c.in);
  });
}

cudaError_t launch_round_bits(const SolverDev& S, uint32_t* z, cudaStream_t stream) {
  k_round_bits<<<S.g.num_items, kPairThreads, 0, stream>>>(S, z);
  return cudaGetLastError();
}

// exact evaluation of given bits: MIS (size, conflicting edges x2, uncovered);
// MaxCut (2*cut, non-fixed, positive gain)
__global__ void __launch_bounds__(kPairThreads) k_eval(SolverDev S, const uint32_t* z, Counters* out) {
  __shared__ unsigned long long s_cnt[4 * 128];
  const int B = S.B, Bw = S.Bw;
  const bool mis = S.p.problem == PROB_MIS;
  const int32_t* rp = S.g.row_ptr;
  const int32_t* col = S.g.col;
  const int8_t* wts = S.g.w;
  const int it = blockIdx.x;
  const Item item = S.g.items[it];
  for (int i = threadIdx.x; i < 4 * B; i += blockDim.x) s_cnt[i] = 0ull;
  __syncthreads();
  long long a0 = 0, a1 = 0, a2 = 0;
  const int my_b = (int)(threadIdx.x % B);
  item_pairs(S, item, [&](const PairCtx& c) {
    if (!c.in) return;
    const int64_t v = c.v;
    const int b = c.b;
    const bool zv = get_bit(z, v, Bw, b);
    if (mis) {
      int cnt = 0;
      for (int32_t j = rp[v]; j < rp[v + 1]; ++j) cnt += get_bit(z, col[j], Bw, b);
      a0 += zv;
      a1 += zv ? cnt : 0;
      a2 += !zv && cnt == 0;
    } else {
      int P = 0, W = 0;
      for (int32_t j = rp[v]; j < rp[v + 1]; ++j) {
        const int w = wts ? (int)wts[j] : 1;
        W += w;
        if (get_bit(z, col[j], Bw, b)) P += w;
      }
      const int as = 2 * P - W;
      a0 += zv ? (W - P) : P;
      a1 += !(zv ? (as <= -1) : (as >= 0));
      a2 += (zv ? as : -as) > 0;
    }
  });
  if (a0) atomicAdd(&s_cnt[4 * my_b + 0], (unsigned long long)a0);
  if (a1) atomicAdd(&s_cnt[4 * my_b + 1], (unsigned long long)a1);
  if (a2) atomicAdd(&s_cnt[4 * my_b + 2], (unsigned long long)a2);
  flush_pair_counters(S, s_cnt, item.g, it, out);
}

cudaError_t launch_eval(const SolverDev& S, const uint32_t* z, Counters* out, cudaStream_t stream) {
  k_eval<<<S.g.num_items, kPairThreads, 0, stream>>>(S, z, out);
  return cudaGetLastError();
}

// counters (R replicas) -> user arrays. kind 0: step/machine counters
// (MaxCut value is 2*cut); kind 1: evaluation counters (MIS a = 2*edges,
// MaxCut value = 2*cut)
__global__ void k_counters_out(const Counters* c, int64_t T, int R, int mis, int kind, int64_t* value, int64_t* a,
                               int64_t* b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T) return;
  const Counters x = sum_replicas(c, i, R);
  int64_t v = (int64_t)x.value, aa = (int64_t)x.a;
  if (!mis) v /= 2;
  if (mis && kind == 1) aa /= 2;
  if (value) value[i] = v;
  if (a) a[i] = aa;
  if (b) b[i] = (int64_t)x.b;
}

cudaError_t launch_counters_out(const SolverDev& S, const Counters* c, int64_t* value, int64_t* a, int64_t* b,
                                int kind, cudaStream_t stream) {
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  k_counters_out<<<(unsigned)((T + 255) / 256), 256, 0, stream>>>(c, T, S.R, S.p.problem == PROB_MIS, kind, value,
                                                                  a, b);
  return cudaGetLastError();
}

// relaxed objective per trajectory in double: (Ax)_v in float32 (CSR order),
// then the node's terms in double (MIS h; MaxCut f_B, f_L = 1/4 x'(D-A)x,
// f_P = x'(D-A+lambda I)x or f_A = -x'Ax), accumulated per thread and
// reduced per item in shared memory
__global__ void __launch_bounds__(kPairThreads) k_objective(SolverDev S, double* out) {
  __shared__ double s_obj[128];
  const int64_t t = *S.tick;
  const void* Xc = (t & 1) ? S.X1 : S.X0;
  const int B = S.B;
  const bool mis = S.p.problem == PROB_MIS;
  auto ld = [&](int64_t e) -> float {
    if (S.p.x_dtype == DT_F32) return static_cast<const float*>(Xc)[e];
    if (S.p.x_dtype == DT_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(Xc)[e]);
    return __half2float(static_cast<const __half*>(Xc)[e]);
  };
  for (int i = threadIdx.x; i < B; i += blockDim.x) s_obj[i] = 0.0;
  __syncthreads();
  const Item item = S.g.items[blockIdx.x];
  double part = 0.0;
  item_pairs(S, item, [&](const PairCtx& c) {
    if (!c.in) return;
    float acc = 0.0f;
    int d = 0;
    for (int32_t j = S.g.row_ptr[c.v]; j < S.g.row_ptr[c.v + 1]; ++j) {
      const float xu = ld((int64_t)S.g.col[j] * B + c.b);
      const int w = S.g.w == nullptr ? 1 : (int)S.g.w[j];
      d += w;
      if (w >= 0) acc = acc + xu;
      else acc = acc - xu;
    }
    const double xv = (double)ld(c.v * B + c.b);
    const double xax = xv * (double)acc, lam = (double)S.p.lambda_;
    if (mis) {
      part += xv - 0.5 * (double)S.p.gamma * xax;
    } else {
      const double xdx = (double)d * xv * xv;
      switch (S.p.objective) {
        case OBJ_FL: part += 0.25 * (xdx - xax); break;
        case OBJ_FP: part += (xdx - xax) + lam * xv * xv; break;
        case OBJ_FA: part += -xax; break;
        default: part += -lam * xv - xax; break;
      }
    }
  });
  if (part != 0.0) atomicAdd(&s_obj[threadIdx.x % B], part);
  __syncthreads();
  for (int i = threadIdx.x; i < B; i += blockDim.x)
    if (s_obj[i] != 0.0) atomicAdd(&out[(int64_t)item.g * B + i], s_obj[i]);
}

cudaError_t launch_objective(const SolverDev& S, double* out, cudaStream_t stream) {
  k_objective<<<S.g.num_items, kPairThreads, 0, stream>>>(S, out);
  return cudaGetLastError();
}

// after a standalone local search: restore the machine state, keep best
__global__ void k_ls_merge(TrajState* st, const TrajState* saved, int64_t* bestv, int64_t T) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T) return;
  TrajState s = saved[i];
  s.best = st[i].best;
  s.accepts = st[i].accepts;
  s.first_value = st[i].first_value;
  s.gain_descent = st[i].gain_descent;
  s.gain_ls = st[i].gain_ls;
  st[i] = s;
  bestv[i] = s.best;
}

cudaError_t launch_ls_merge(const SolverDev& S, const TrajState* saved, cudaStream_t stream) {
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  k_ls_merge<<<(unsigned)((T + 255) / 256), 256, 0, stream>>>(S.st, saved, S.bestv, T);
  return cudaGetLastError();
}

// fresh machine state for every trajectory: first descent of outer
// iteration 0, no best set; the apply pass then writes the initial x
__global__ void k_state_init(SolverDev S) {
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  const int64_t tau = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = *S.tick;
  if (tau < T) {
    TrajState st;
    st.phase = PH_DESCENT;
    st.s = 0;
    st.r = 0;
    st.o = 0;
    st.best = (int64_t)(-9223372036854775807LL - 1);
    st.ticks = 0;
    st.last_round = RD_NONE;
    st.round = RD_NONE;
    st.last_commits = 0;
    st.ev_value = st.ev_a = st.ev_b = 0;
    st.accepts = st.descents = 0;
    st.act = ACT_INIT;
    st.ls_done = 0;
    for (int i = 0; i < 6; ++i) st.rkeys[i] = 0u;
    st.rk = 0;
    st.held = (int64_t)(-9223372036854775807LL - 1);
    st.first_value = st.held;
    st.gain_descent = st.gain_ls = 0;
    st.steps = 0;
    S.st[tau] = st;
    if (S.K > 0 && tau < S.g.num_graphs) {
      PoolState ps;
      ps.epoch = EP_DESCENT;
      ps.count = 0;
      ps.best = st.best;
      ps.merges = 0;
      ps.dec = DEC_NONE;
      ps.best_src = -1;
      ps.merged = 0;
      ps.stamp = 0;
      S.pool[tau] = ps;
    }
    S.act[tau] = ACT_INIT;
    S.rnd[tau] = RD_NONE;
    S.bestv[tau] = st.best;
    for (int r = 0; r < S.R; ++r) S.cnt[tau * S.R + r] = Counters{0ull, 0ull, 0ull, 0ull};
    const int g = (int)(tau / S.B);
    S.gflag[g] = (int32_t)(t + 1);
  }
  if (tau == 0) S.any[0] = (int32_t)(t + 1);
}

cudaError_t launch_state_init(const SolverDev& S, cudaStream_t stream) {
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  k_state_init<<<(unsigned)((T + 127) / 128), 128, 0, stream>>>(S);
  return cudaGetLastError();
}

// out = number of trajectories still running a standalone local search
__global__ void k_any_pending(SolverDev S, int32_t* out) {
  const int64_t T = (int64_t)S.g.num_graphs * S.B;
  int c = 0;
  for (int64_t i = threadIdx.x; i < T; i += blockDim.x) c += S.st[i].ls_done == 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += s[i];
    *out = tot;
  }
}

cudaError_t launch_any_pending(const SolverDev& S, int32_t* out, cudaStream_t stream) {
  k_any_pending<<<1, 1024, 0, stream>>>(S, out);
  return cudaGetLastError();
}

}  // namespace mqo
