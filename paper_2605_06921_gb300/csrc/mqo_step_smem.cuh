// mqo_step_smem.cuh -- the fused descent step for member graphs whose block
// of x fits in shared memory (k_step_s), instantiated by mqo_step.cu (column
// indices from the CSR arrays) and mqo_step_ell.cu (the sliced-ELL offset
// stream).  The step itself (gradient, momentum, projection, rounding, exact
// evaluation) is described in mqo_step.cuh.
#pragma once

#include "mqo_step.cuh"

namespace mqo {

// ---------------------------------------------------------------- shared memory
// Each lane owns VEC consecutive trajectories (8 or 16 bytes of x), a row
// group of LPR = B/VEC lanes one node, and the RPW = 32/LPR row groups of a
// warp walk their rows' neighbour lists in lockstep, so one shared-memory
// load instruction serves RPW rows.  An item's rows are taken in
// decreasing-degree order, so the rows of a warp have nearly equal lengths;
// rows shorter than the warp's longest are padded with a dummy neighbour,
// local index ng, whose shared-memory row of x and bit words are zero:
// adding +0.0 leaves a float32 sum that is not -0.0 unchanged, and sums of
// values that are never -0.0 are never -0.0, so the padded sums equal the
// CSR-order sums exactly and the inner loop needs no predicates.  DUP
// (64-byte rows): the block of x is stored with a 128-byte pitch and each row
// twice, at bytes [0,64) and [64,128); row groups of odd index read the
// second copy, so the two row groups of a half-warp always use opposite
// halves of the 32 banks.
//
// Where the neighbours' ids come from:
//  * CSR (ELL = false): LPR neighbours (one chunk) at a time, one coalesced
//    index load per row group, each id broadcast to the row group by a
//    shuffle;
//  * sliced ELL (ELL = true): the item's rows in groups of RPW consecutive
//    rows of the processing order, one group per warp pass; the group's
//    lists padded with the dummy neighbour to 4·nvec entries and stored as
//    nvec chunks of RPW 16-byte vectors, vector r of chunk c holding entries
//    4c .. 4c+3 of the group's row r as byte offsets of the neighbours' rows
//    in the staged block (local id × pitch).  One 16-byte load per row group
//    brings four neighbours, and the RPW loads of a warp read one contiguous
//    RPW·16-byte piece: no shuffles and no index arithmetic per neighbour.
//    ell_pos[p] = {first vector of the group of processing position p, nvec}.
//    The next group's vectors are prefetched into L2 while the current
//    group is summed.

// add_bf16_row plus a running maximum of the row's bfloat16 bit patterns read
// as signed 16-bit integers, one 32-bit word (two trajectories) per mx[]
// entry.  For bfloat16 values in [0, 1] that order is the order of the
// values, and -0 (0x8000) reads as the most negative: after a row, half k of
// mx[w] > 0x3F00 (= 0.5) iff some neighbour of trajectory 2w + k has x > 0.5.
template <int VEC>
__device__ __forceinline__ void add_bf16_row_max(float* acc, uint32_t* mx, const unsigned char* p);
template <>
__device__ __forceinline__ void add_bf16_row_max<4>(float* acc, uint32_t* mx, const unsigned char* p) {
  const uint2 r = *reinterpret_cast<const uint2*>(p);
  add_bf16x2_word(acc[0], acc[1], r.x);
  add_bf16x2_word(acc[2], acc[3], r.y);
  mx[0] = __vmaxs2(mx[0], r.x);
  mx[1] = __vmaxs2(mx[1], r.y);
}
template <>
__device__ __forceinline__ void add_bf16_row_max<8>(float* acc, uint32_t* mx, const unsigned char* p) {
  const uint4 r = *reinterpret_cast<const uint4*>(p);
  add_bf16x2_word(acc[0], acc[1], r.x);
  add_bf16x2_word(acc[2], acc[3], r.y);
  add_bf16x2_word(acc[4], acc[5], r.z);
  add_bf16x2_word(acc[6], acc[7], r.w);
  mx[0] = __vmaxs2(mx[0], r.x);
  mx[1] = __vmaxs2(mx[1], r.y);
  mx[2] = __vmaxs2(mx[2], r.z);
  mx[3] = __vmaxs2(mx[3], r.w);
}

// MIS with bfloat16 x and 4 or 8 trajectories per lane: the checker's
// neighbour test comes from a running signed max of the gathered bfloat16
// words (add_bf16_row_max) instead of the neighbours' rounding words
template <typename TX, int VEC, bool MIS>
constexpr bool kMaxCheck = MIS && std::is_same<TX, __nv_bfloat16>::value && (VEC == 4 || VEC == 8);

// 16-byte global-to-shared copy that bypasses the registers (cp.async,
// cached in L2 only); complete after stage_wait_all
static __device__ __forceinline__ void stage_copy16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
static __device__ __forceinline__ void stage_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// L2 prefetch of `bytes` (a multiple of 16) from a 16-byte aligned address
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// CTAs of kStepThreads threads (two per SM), kStepThreadsWideEll for 16-byte
// lanes with the ELL stream, whose ring of four vectors and eight
// accumulators per lane need more than 64 registers: eight warps then take
// exactly four groups of an item of 256 rows each (measured: 256 threads
// 0.161 ms, 384 threads 0.164 ms, 512 threads at one CTA per SM 0.203 ms)
constexpr int kStepThreads = 512;
constexpr int kStepThreadsWideEll = 256;
template <int VEC, bool ELL>
constexpr int kStepNT = (ELL && VEC == 8) ? kStepThreadsWideEll : kStepThreads;

template <typename TX, typename TV, int VEC, int LPR, bool MIS, bool DUP, bool ELL>
__global__ void __launch_bounds__(kStepNT<VEC, ELL>, 2)
    k_step_s(StepArgs a, const int4* __restrict__ ell, const int2* __restrict__ ell_pos) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RPW = 32 / LPR;
  constexpr bool kMax = kMaxCheck<TX, VEC, MIS>;
  // the ELL stream carries no weights and no rounding words: unweighted
  // MaxCut, or MIS with the checker from the gathered words
  static_assert(!ELL || !MIS || kMax, "sliced ELL: MIS needs the max checker");
  const int it = blockIdx.x;
  const Item item = a.g.items[it];
  const int g = item.g;
  const int64_t t = *a.tick;
  if (a.gflag_step && a.gflag_step[g] != (int32_t)(t + 1)) return;
  constexpr int B = VEC * LPR;  // a row group of LPR lanes holds the whole batch
  constexpr int BW = (B + 31) / 32;
  const int32_t off = a.g.node_off[g];
  const int32_t ng = a.g.node_off[g + 1] - off;
  const int rowb = B * (int)sizeof(TX);  // bytes of one node's x
  const int pitch = DUP ? 128 : rowb;
  const size_t xbytes = ((size_t)(ng + 1) * pitch + 15) & ~(size_t)15;
  uint32_t* sZ = reinterpret_cast<uint32_t*>(smem + xbytes);
  const size_t zbytes = MIS ? (((size_t)(ng + 1) * BW * 4 + 15) & ~(size_t)15) : 0;
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(smem + xbytes + zbytes);
  // the item's rows in processing order: {node, row start, row end, -} from
  // the CSR, {node, group's first vector, group's nvec, degree} with ELL
  int4* s_rows = reinterpret_cast<int4*>(smem + xbytes + zbytes + ((3 * (size_t)B * 8 + 15) & ~(size_t)15));
  const int nrows = item.v1 - item.v0;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  if constexpr (ELL) {
    // this warp's first group towards L2 while the block of x is staged
    if (lane == 0 && warp * RPW < nrows) {
      const int2 ep = ell_pos[item.v0 + warp * RPW];
      if (ep.y > 0) prefetch_l2(ell + ep.x, (uint32_t)ep.y * RPW * 16u);
    }
  }

  const TX* __restrict__ Xc = static_cast<const TX*>((t & 1) ? a.X1 : a.X0);
  TX* __restrict__ Xn = static_cast<TX*>((t & 1) ? a.X0 : a.X1);
  const uint32_t* __restrict__ Zc = (t & 1) ? a.ZX1 : a.ZX0;
  uint32_t* __restrict__ Zn = (t & 1) ? a.ZX0 : a.ZX1;
  TV* __restrict__ V = static_cast<TV*>(a.V);

  // stage the member graph's x block (16-byte asynchronous copies, all of a
  // thread's in flight at once), the zero dummy row, and the rounding words
  {
    const int4* src = reinterpret_cast<const int4*>(Xc + (int64_t)off * B);
    const int per = rowb / 16;  // 16-byte pieces per node
    const int n16 = ng * per;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
      const int node = i / per, piece = i - node * per;
      unsigned char* d = smem + (size_t)node * pitch + piece * 16;
      stage_copy16(d, src + i);
      if (DUP) stage_copy16(d + 64, src + i);
    }
    for (int i = threadIdx.x; i < pitch / 16; i += blockDim.x)
      *reinterpret_cast<int4*>(smem + (size_t)ng * pitch + i * 16) = make_int4(0, 0, 0, 0);
    if (MIS && !kMax) {
      const uint32_t* zs = Zc + (int64_t)off * BW;
      for (int i = threadIdx.x; i < ng * BW; i += blockDim.x) sZ[i] = zs[i];
      for (int i = threadIdx.x; i < BW; i += blockDim.x) sZ[ng * BW + i] = 0u;
    }
    for (int i = threadIdx.x; i < 3 * B; i += blockDim.x) s_cnt[i] = 0ull;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const int v = a.g.order[item.v0 + i];
      if constexpr (ELL) {
        const int2 ep = ell_pos[item.v0 + i];
        s_rows[i] = make_int4(v, ep.x, ep.y, a.g.row_ptr[v + 1] - a.g.row_ptr[v]);
      } else {
        s_rows[i] = make_int4(v, a.g.row_ptr[v], a.g.row_ptr[v + 1], 0);
      }
    }
    stage_wait_all();
  }
  __syncthreads();

  const int sub = lane / LPR;
  const int l = lane - sub * LPR;
  const int b0 = l * VEC;
  const float thr = MIS ? 0.5f : 0.0f;
  const float lo = MIS ? 0.0f : -1.0f;
  const bool weighted = !ELL && !MIS && a.g.w != nullptr;
  const int32_t* __restrict__ col = a.g.col;
  // 16-bit member-local indices where the graph has them: half the index bytes
  const uint16_t* __restrict__ col16 = a.g.col16;
  const bool c16 = col16 != nullptr;
  const int8_t* __restrict__ wts = a.g.w;
  constexpr int K = (LPR < 32 / VEC) ? LPR : 32 / VEC;  // lanes sharing one output word
  const unsigned rmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (sub * LPR));
  const unsigned char* sXl = smem + (DUP ? (sub & 1) * 64 : 0) + l * (VEC * (int)sizeof(TX));

  uint32_t stepm = 0u;  // bit e: trajectory b0 + e steps
#pragma unroll
  for (int e = 0; e < VEC; ++e)
    stepm |= (uint32_t)(a.act ? (a.act[(int64_t)g * B + b0 + e] & ACT_STEP) != 0 : true) << e;
  // counts of nodes stay below 2^10 per lane (an item has at most 256 rows),
  // so they are packed into one word per trajectory: MIS all three, MaxCut
  // the last two (its first counter sums cut edges)
  int c0[VEC], c1[VEC], c2[VEC];
  uint32_t cp[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) c0[e] = c1[e] = c2[e] = 0, cp[e] = 0u;

  // column indices (CSR) come in groups of four chunks; each group's loads
  // are issued before the previous group is consumed (software pipeline), and
  // a row's first group during the previous row's epilogue.  With ELL the
  // group's first two vectors are loaded during the previous epilogue.
  int nxu[4], nxw[4];
  int4 e0, e1;
  auto first_group = [&](int i) {
    if constexpr (ELL) {
      // i: the group's first position (warp-uniform)
      const int dummy = ng * pitch;
      e0 = e1 = make_int4(dummy, dummy, dummy, dummy);
      if (i < nrows) {
        const int4 r = s_rows[i];
        const int4* p = ell + r.y + sub;
        if (r.z > 0) e0 = __ldcs(p);
        if (r.z > 1) e1 = __ldcs(p + RPW);
      }
    } else {
      const bool h = i < nrows;
      const int4 r = s_rows[h ? i : 0];
      const int rs_ = h ? r.y : 0, re_ = h ? r.z : 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = rs_ + c * LPR + l;
        const bool jin = j < re_;
        nxu[c] = jin ? (c16 ? (int)__ldcs(col16 + j) : __ldcs(col + j) - off) : ng;
        nxw[c] = jin ? (weighted ? (int)wts[j] : 1) : 0;
      }
    }
  };
  first_group(ELL ? warp * RPW : warp * RPW + sub);
  for (int vb = warp * RPW; vb < nrows;) {
    // the warp's next group of rows: every nwarps-th group (claiming groups
    // from a shared counter instead measured 5 % slower)
    const int vn = vb + nwarps * RPW;
    const bool has = vb + sub < nrows;
    const int4 row = s_rows[has ? vb + sub : (ELL ? vb : 0)];
    const int v = row.x;
    const int vl = has ? v - off : ng;
    const int64_t base = (int64_t)(has ? v : item.v0) * B + b0;
    const Pack<TX, VEC> xv = *reinterpret_cast<const Pack<TX, VEC>*>(sXl + (size_t)vl * pitch);
    Pack<TV, VEC> vv{};
    if (has) vv = ld_pack_stream<TV, VEC>(V + base);
    float acc[VEC];
    int pos[VEC];
    uint32_t orw[4] = {0u, 0u, 0u, 0u};  // OR of the neighbours' words (BW <= 4)
    uint32_t mx[VEC / 2 > 0 ? VEC / 2 : 1];  // running max of the neighbours' bfloat16 patterns
#pragma unroll
    for (int w = 0; w < (VEC / 2 > 0 ? VEC / 2 : 1); ++w) mx[w] = 0u;
#pragma unroll
    for (int e = 0; e < VEC; ++e) { acc[e] = 0.0f; pos[e] = 0; }
    // one unweighted neighbour whose row of x starts o bytes into the block
    auto add_plain = [&](int o) {
      if constexpr (kMax) {
        // one mixed-precision add per trajectory (the bfloat16 operand is
        // widened exactly inside the add, which rounds once, so the sums are
        // those of the widened values added one by one) and the checker's
        // "some neighbour in the set" from the same words
        add_bf16_row_max<VEC>(acc, mx, sXl + o);
      } else if constexpr (MIS && std::is_same<TX, __nv_bfloat16>::value) {
        add_bf16_row<VEC>(acc, sXl + o);
      } else {
        float f[VEC];
        load_unpack<TX, VEC>(sXl + o, f);
        // two trajectories per packed add (IEEE round-to-nearest per
        // element: the same sums as one scalar add each)
#pragma unroll
        for (int e = 0; e < VEC; e += 2) add_f32x2(acc[e], acc[e + 1], f[e], f[e + 1]);
        if (!MIS) {
#pragma unroll
          for (int e = 0; e < VEC; ++e) pos[e] += (f[e] > thr);
        }
      }
    };
    int wsum;
    if constexpr (ELL) {
      wsum = has ? row.w : 0;
      const int4 grp = s_rows[vb];  // the group's vectors (same for its rows)
      const int nvec = grp.z;
      if (lane == 0 && vn < nrows) {
        const int4 gn = s_rows[vn];
        if (gn.z > 0) prefetch_l2(ell + gn.y, (uint32_t)gn.z * RPW * 16u);
      }
      const int4* ep = ell + grp.y + sub;
      // a ring of four vectors (0 and 1 loaded during the previous group's
      // epilogue): each is summed, then refilled four vectors ahead
      const int dummy = ng * pitch;
      int4 e2 = make_int4(dummy, dummy, dummy, dummy), e3 = e2;
      if (nvec > 2) e2 = __ldcs(ep + 2 * RPW);
      if (nvec > 3) e3 = __ldcs(ep + 3 * RPW);
      auto add4 = [&](const int4& q) {
        add_plain(q.x);
        add_plain(q.y);
        add_plain(q.z);
        add_plain(q.w);
      };
      int c = 0;
      for (; c + 4 <= nvec; c += 4) {
        add4(e0);
        if (c + 4 < nvec) e0 = __ldcs(ep + (c + 4) * RPW);
        add4(e1);
        if (c + 5 < nvec) e1 = __ldcs(ep + (c + 5) * RPW);
        add4(e2);
        if (c + 6 < nvec) e2 = __ldcs(ep + (c + 6) * RPW);
        add4(e3);
        if (c + 7 < nvec) e3 = __ldcs(ep + (c + 7) * RPW);
      }
      if (c < nvec) add4(e0);
      if (c + 1 < nvec) add4(e1);
      if (c + 2 < nvec) add4(e2);
      first_group(vn);
    } else {
      const int rs = has ? row.y : 0, re = has ? row.z : 0;
      const int nch_w = __reduce_max_sync(0xffffffffu, (re - rs + LPR - 1) / LPR);
      wsum = weighted ? 0 : re - rs;
      for (int ch0 = 0; ch0 < nch_w; ch0 += 4) {
        int myo[4], myw[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (MIS && !kMax)
            for (int w = 0; w < BW; ++w) orw[w] |= sZ[nxu[c] * BW + w];
          myo[c] = nxu[c] * pitch;  // byte offset of the neighbour's row
          myw[c] = nxw[c];
        }
        if (ch0 + 4 < nch_w) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = rs + (ch0 + 4 + c) * LPR + l;
            const bool jin = j < re;
            nxu[c] = jin ? (c16 ? (int)__ldcs(col16 + j) : __ldcs(col + j) - off) : ng;
            nxw[c] = jin ? (weighted ? (int)wts[j] : 1) : 0;
          }
        }
        // one chunk: the LPR neighbours whose offsets (and weights) the
        // row group's lanes hold
        auto chunk = [&](int mo, int mw) {
#pragma unroll
          for (int k = 0; k < LPR; ++k) {
            const int o = __shfl_sync(0xffffffffu, mo, k, LPR);
            if (!weighted) {
              add_plain(o);
              continue;
            }
            float f[VEC];
            load_unpack<TX, VEC>(sXl + o, f);
            const int w = __shfl_sync(0xffffffffu, mw, k, LPR);
            wsum += w;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
              acc[e] = w >= 0 ? acc[e] + f[e] : acc[e] - f[e];
              pos[e] += (f[e] > thr) ? w : 0;
            }
          }
        };
        if (ch0 + 4 <= nch_w) {
          // a full group of four chunks: no per-chunk test
          chunk(myo[0], myw[0]);
          chunk(myo[1], myw[1]);
          chunk(myo[2], myw[2]);
          chunk(myo[3], myw[3]);
        } else {
          // the row's last one to three chunks
          chunk(myo[0], myw[0]);
          if (ch0 + 1 < nch_w) chunk(myo[1], myw[1]);
          if (ch0 + 2 < nch_w) chunk(myo[2], myw[2]);
        }
      }
      first_group(vn + sub);
    }
    if constexpr (kMax) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int16_t h = (int16_t)(uint16_t)(mx[e >> 1] >> (16 * (e & 1)));
        pos[e] = h > (int16_t)0x3F00;  // bfloat16 0.5
      }
    } else if (MIS) {
      for (int w = 0; w < BW; ++w)
        for (int o = 1; o < LPR; o <<= 1) orw[w] |= __shfl_xor_sync(0xffffffffu, orw[w], o);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int bb = b0 + e;
        uint32_t word = orw[0];
        for (int w = 1; w < BW; ++w)
          if ((bb >> 5) == w) word = orw[w];
        pos[e] = (word >> (bb & 31)) & 1u;
      }
    }
    Pack<TX, VEC> xo;
    Pack<TV, VEC> vo;
    unsigned zbits = 0u;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      bool zn;
      int d0 = 0, d1 = 0, d2 = 0;
      step_element<TX, TV>(a, MIS, thr, lo, xv.e[e], vv.e[e], acc[e], pos[e], wsum, (stepm >> e) & 1u, xo.e[e],
                           vo.e[e], zn, d0, d1, d2);
      if (has) {
        if constexpr (MIS) {
          cp[e] += (uint32_t)d0 | ((uint32_t)d1 << 10) | ((uint32_t)d2 << 20);
        } else {
          c0[e] += d0;
          cp[e] += ((uint32_t)d1 << 10) | ((uint32_t)d2 << 20);
        }
      }
      zbits |= (unsigned)zn << e;
    }
    if (has) {
      st_pack<TX, VEC>(Xn + base, xo);
      st_pack<TV, VEC>(V + base, vo);
    }
    unsigned word = zbits << (b0 & 31);
#pragma unroll
    for (int o = 1; o < K; o <<= 1) word |= __shfl_xor_sync(rmask, word, o);
    if (has && (l % K) == 0) Zn[(int64_t)v * BW + (b0 >> 5)] = word;
    vb = vn;
  }
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    if constexpr (MIS) c0[e] = (int)(cp[e] & 1023u);
    c1[e] = (int)((cp[e] >> 10) & 1023u);
    c2[e] = (int)(cp[e] >> 20);
  }
  flush_step_counters<VEC>(a, s_cnt, g, it, b0, LPR, c0, c1, c2, stepm);
}

template <typename TX, typename TV, int VEC, int LPR, bool MIS, bool DUP, bool ELL>
static cudaError_t launch_s(size_t smem, const StepArgs& a, const int4* ell, const int2* ell_pos, int grid,
                            cudaStream_t s) {
  if (a.B != VEC * LPR) return cudaErrorInvalidValue;
  auto kern = k_step_s<TX, TV, VEC, LPR, MIS, DUP, ELL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, kStepNT<VEC, ELL>, smem, s>>>(a, ell, ell_pos);
  return cudaGetLastError();
}

// lanes hold 8 bytes of x, or 16 when B/32 elements need more:
// 2-byte x: B=32 -> (VEC 4, LPR 8, DUP), B=64 -> (4, 16), B=128 -> (4, 32);
// 4-byte x: B=32 -> (2, 16), B=64 -> (2, 32), B=128 -> (4, 32).
// Wide lanes (16 bytes, half the lanes per row, twice the rows per warp):
// 2-byte x: B=32 -> (8, 4, DUP), B=64 -> (8, 8), B=128 -> (8, 16);
// 4-byte x: B=32 -> (4, 8), B=64 -> (4, 16)
template <typename TX, typename TV, bool ELL>
static cudaError_t launch_smem(int B, bool wide, size_t smem, bool mis, const StepArgs& a, const int4* ell,
                               const int2* ell_pos, int grid, cudaStream_t s) {
  if constexpr (sizeof(TX) == 2) {
    // MIS with the sliced ELL stream: bfloat16 x only (the max checker)
    constexpr bool mis_ok = !ELL || std::is_same<TX, __nv_bfloat16>::value;
    if (wide) {
      if (mis) {
        if constexpr (mis_ok) {
          if (B == 32) return launch_s<TX, TV, 8, 4, true, true, ELL>(smem, a, ell, ell_pos, grid, s);
          if (B == 64) return launch_s<TX, TV, 8, 8, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
          if (B == 128) return launch_s<TX, TV, 8, 16, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
        }
      } else {
        if (B == 32) return launch_s<TX, TV, 8, 4, false, true, ELL>(smem, a, ell, ell_pos, grid, s);
        if (B == 64) return launch_s<TX, TV, 8, 8, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
        if (B == 128) return launch_s<TX, TV, 8, 16, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
      }
    } else if (mis) {
      if constexpr (mis_ok) {
        if (B == 32) return launch_s<TX, TV, 4, 8, true, true, ELL>(smem, a, ell, ell_pos, grid, s);
        if (B == 64) return launch_s<TX, TV, 4, 16, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
        if (B == 128) return launch_s<TX, TV, 4, 32, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
      }
    } else {
      if (B == 32) return launch_s<TX, TV, 4, 8, false, true, ELL>(smem, a, ell, ell_pos, grid, s);
      if (B == 64) return launch_s<TX, TV, 4, 16, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
    }
  } else if constexpr (!ELL) {
    if (wide) {
      if (mis) {
        if (B == 32) return launch_s<TX, TV, 4, 8, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
        if (B == 64) return launch_s<TX, TV, 4, 16, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
      } else {
        if (B == 32) return launch_s<TX, TV, 4, 8, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
        if (B == 64) return launch_s<TX, TV, 4, 16, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
      }
    } else if (mis) {
      if (B == 32) return launch_s<TX, TV, 2, 16, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
      if (B == 64) return launch_s<TX, TV, 2, 32, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, true, false, ELL>(smem, a, ell, ell_pos, grid, s);
    } else {
      if (B == 32) return launch_s<TX, TV, 2, 16, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
      if (B == 64) return launch_s<TX, TV, 2, 32, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, false, false, ELL>(smem, a, ell, ell_pos, grid, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace mqo
