// mqo_step.cu -- the fused descent step (one tick of gradient work).
//
// For every node v and trajectory b of a stepping trajectory:
//   (A x)_vb  = sum over the CSR row of v, in row order, of w_vu x_ub (float32)
//   grad      = 1 - gamma (A x)_vb              (h, Eq. MIS QUBO)
//             | -lambda - 2 (A x)_vb            (f_B, Eq. adj_lin_two_props)
//             | or the gradient of f_L, f_P, f_A (Sec. 3), selected by
//               `objective`; f_L and f_P also use the weighted degree d_v
//   V'        = mu V + alpha grad               (momentum ascent, Sec. 5)
//   x'        = Pi_box(x + V')                  (projection of Sec. 3)
// and, from the same neighbour gather, the exact evaluation of the rounded
// incoming point z = [x > 0.5] (MIS) or [x > 0] (MaxCut): set size,
// conflicting and uncovered nodes (checker, Eq. MIS checking), or cut,
// nodes violating the f_B fixed-point condition and positive-gain nodes.
// The rounding of x' is written next to x' (ZX), so the next step and the
// acceptance of this step's point read it without recomputing.
//
// Thread mapping: a row group of LPR = B/VEC lanes handles one node; lane l
// owns trajectories l*VEC .. l*VEC+VEC-1 and accumulates them sequentially
// over the row, so every (v,b) sum is in CSR order.  Column indices are
// loaded LPR at a time with one coalesced load and broadcast by shuffles.
// One CTA per item (a range of at most 256 nodes of one member graph).
//
// k_step_g: generic; neighbour rows of x are gathered from global memory.
// k_step_s: member graphs small enough for shared memory: the CTA first
//   copies its graph's block of x (and, for MIS, of the rounding bits) to
//   shared memory; every neighbour gather then hits shared memory, and the
//   MIS checker ORs whole 32-trajectory words of neighbour bits.  Several
//   rows per warp share each shuffle and shared-memory instruction.
#include <type_traits>

#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

struct StepArgs {
  GraphDev g;
  int32_t B, Bw, R, problem, objective;
  int32_t split;  // generic kernel: CTAs per item, each taking a contiguous slice of its rows
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
// neighbours with z = 1 (wsum = weighted degree).
template <typename TX, typename TV>
__device__ __forceinline__ void step_element(const StepArgs& a, bool mis, float thr, float lo, TX xin, TV vin,
                                             float acc, int nb, int wsum, bool stepping, TX& xout, TV& vout,
                                             bool& znew, int& c0, int& c1, int& c2) {
  const float x = to_f(xin);
  const float vold = to_f(vin);
  const bool z = x > thr;
  if (mis) {
    const bool any = nb != 0;
    c0 += z;
    c1 += z && any;
    c2 += !z && !any;
  } else {
    const int as = 2 * nb - wsum;
    c0 += z ? (wsum - nb) : nb;
    const bool fixed = cut_fixed(a.objective, a.lambda_, z, as, wsum);
    c1 += !fixed;
    const int gn = z ? as : -as;
    c2 += gn > 0;
  }
  float grad;
  if (mis) {
    const float tt = a.gamma * acc;
    grad = 1.0f - tt;
  } else {
    grad = cut_grad(a.objective, a.lambda_, x, acc, wsum);
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

// ---------------------------------------------------------------- generic
// The CTA first stages its item's row pointers and (up to kColCap) column
// indices / weights in shared memory with coalesced loads, so that a row's
// neighbour ids cost no dependent global load.  A row group of LPR = B/VEC
// lanes owns two rows at a time: it issues the loads of both rows' x and V
// and of up to kGather neighbour rows of x for each before consuming any,
// then runs both epilogues, so every lane keeps two rows' memory traffic in
// flight.  MIS and WEIGHTED are compile-time: the unweighted MaxCut and MIS
// variants carry no per-neighbour weight logic.
constexpr int kColCap = 4096;  // staged column indices per item
constexpr int kGather = 4;     // neighbour rows of x in flight per row and row group
// rows a row group keeps in flight: two for narrow lanes, one for lanes of 4
// or more trajectories (their packs and sums would not fit the registers of
// two CTAs per SM)
template <int VEC>
__host__ __device__ constexpr int rows_in_flight() { return VEC >= 4 ? 1 : 2; }

template <typename TX, typename TV, int VEC, bool MIS, bool WEIGHTED>
__global__ void __launch_bounds__(512, (VEC >= 8 ? 1 : 2)) k_step_g(StepArgs a) {
  __shared__ unsigned long long s_cnt[3 * 128];
  __shared__ int32_t s_rp[kItemMaxNodes + 1];
  __shared__ int32_t s_col[kColCap];
  __shared__ int8_t s_w[WEIGHTED ? kColCap : 1];
  const int it = blockIdx.x / a.split;
  Item item = a.g.items[it];
  const int g = item.g;
  const int64_t t = *a.tick;
  if (a.gflag_step && a.gflag_step[g] != (int32_t)(t + 1)) return;
  {  // this CTA's slice of the item's rows
    const int part = blockIdx.x - it * a.split;
    const int per = (item.v1 - item.v0 + a.split - 1) / a.split;
    const int r0 = item.v0 + part * per;
    item.v1 = min(item.v1, r0 + per);
    item.v0 = r0;
    if (item.v0 >= item.v1) return;
  }
  const int B = a.B;
  const int32_t* __restrict__ rp = a.g.row_ptr;
  const int32_t* __restrict__ col = a.g.col;
  const int8_t* __restrict__ wts = a.g.w;
  const int nrows = item.v1 - item.v0;
  for (int i = threadIdx.x; i < 3 * B; i += blockDim.x) s_cnt[i] = 0ull;
  for (int i = threadIdx.x; i <= nrows; i += blockDim.x) s_rp[i] = rp[item.v0 + i];
  __syncthreads();
  const int32_t j0 = s_rp[0];
  const int32_t ncol = min(s_rp[nrows] - j0, kColCap);
  for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
    s_col[i] = __ldcs(col + j0 + i);
    if constexpr (WEIGHTED) s_w[i] = wts[j0 + i];
  }
  __syncthreads();

  const int lpr = B / VEC;
  const int rpw = 32 / lpr;
  const int lane = threadIdx.x & 31;
  const int sub = lane / lpr;
  const int l = lane - sub * lpr;
  const int b0 = l * VEC;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const float thr = MIS ? 0.5f : 0.0f;
  const float lo = MIS ? 0.0f : -1.0f;
  const TX* __restrict__ Xc = static_cast<const TX*>((t & 1) ? a.X1 : a.X0);
  TX* __restrict__ Xn = static_cast<TX*>((t & 1) ? a.X0 : a.X1);
  uint32_t* __restrict__ Zn = (t & 1) ? a.ZX0 : a.ZX1;
  TV* __restrict__ V = static_cast<TV*>(a.V);
  const int K = (lpr < 32 / VEC) ? lpr : 32 / VEC;  // lanes sharing one output bit word
  const unsigned rmask = lpr == 32 ? 0xffffffffu : (((1u << lpr) - 1u) << (sub * lpr));

  uint32_t stepm = 0u;  // bit e: trajectory b0 + e steps
#pragma unroll
  for (int e = 0; e < VEC; ++e)
    stepm |= (uint32_t)(a.act ? (a.act[(int64_t)g * B + b0 + e] & ACT_STEP) != 0 : true) << e;
  int c0[VEC], c1[VEC], c2[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) c0[e] = c1[e] = c2[e] = 0;

  constexpr int ROWS = rows_in_flight<VEC>();
  auto entry = [&](int32_t j, int32_t& u, int& w) {
    const int32_t r = j - j0;
    u = r < ncol ? s_col[r] : col[j];
    if constexpr (WEIGHTED) w = (int)(r < ncol ? s_w[r] : wts[j]);
    else w = 1;
  };

  // row group rows: vr (and vr + rpw when ROWS = 2), then ROWS*rpw*nwarps further
  for (int vr = warp * rpw * ROWS + sub; vr < nrows; vr += nwarps * rpw * ROWS) {
    const int vr2 = vr + rpw;
    const bool two = ROWS == 2 && vr2 < nrows;
    int v[ROWS], rs[ROWS], dg[ROWS];
    v[0] = item.v0 + vr;
    rs[0] = s_rp[vr];
    dg[0] = s_rp[vr + 1] - rs[0];
    if constexpr (ROWS == 2) {
      v[1] = item.v0 + (two ? vr2 : vr);
      rs[1] = two ? s_rp[vr2] : 0;
      dg[1] = two ? s_rp[vr2 + 1] - s_rp[vr2] : 0;
    }
    Pack<TX, VEC> xv[ROWS];
    Pack<TV, VEC> vv[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int64_t base = (int64_t)v[r] * B + b0;
      xv[r] = ld_pack<TX, VEC>(Xc + base);
      vv[r] = ld_pack_stream<TV, VEC>(V + base);
    }
    float acc[ROWS][VEC];
    int pos[ROWS][VEC];
    int wsum[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      wsum[r] = WEIGHTED ? 0 : dg[r];
#pragma unroll
      for (int e = 0; e < VEC; ++e) { acc[r][e] = 0.0f; pos[r][e] = 0; }
    }
    int dmax = dg[0];
    if constexpr (ROWS == 2) dmax = dg[0] > dg[1] ? dg[0] : dg[1];
    for (int k = 0; k < dmax; k += kGather) {
      int w[ROWS][kGather];
      Pack<TX, VEC> p[ROWS][kGather];
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int q = 0; q < kGather; ++q) {
          int32_t u = v[r];  // past the row: a harmless load of the row's own x
          w[r][q] = 0;
          if (k + q < dg[r]) entry(rs[r] + k + q, u, w[r][q]);
          p[r][q] = ld_pack<TX, VEC>(Xc + (int64_t)u * B + b0);
        }
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int q = 0; q < kGather; ++q) {
          if (k + q >= dg[r]) break;
          if constexpr (WEIGHTED) wsum[r] += w[r][q];
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float f = to_f(p[r][q].e[e]);
            if constexpr (WEIGHTED) {
              acc[r][e] = w[r][q] >= 0 ? acc[r][e] + f : acc[r][e] - f;
              pos[r][e] += (f > thr) ? w[r][q] : 0;
            } else {
              acc[r][e] = acc[r][e] + f;
              pos[r][e] += (f > thr);
            }
          }
        }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      if (r == 1 && !two) break;
      Pack<TX, VEC> xo;
      Pack<TV, VEC> vo;
      unsigned zbits = 0u;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        bool zn;
        step_element<TX, TV>(a, MIS, thr, lo, xv[r].e[e], vv[r].e[e], acc[r][e], pos[r][e], wsum[r],
                             (stepm >> e) & 1u, xo.e[e], vo.e[e], zn, c0[e], c1[e], c2[e]);
        zbits |= (unsigned)zn << e;
      }
      const int64_t base = (int64_t)v[r] * B + b0;
      st_pack<TX, VEC>(Xn + base, xo);
      st_pack<TV, VEC>(V + base, vo);
      unsigned word = zbits << (b0 & 31);
      for (int off = 1; off < K; off <<= 1) word |= __shfl_xor_sync(rmask, word, off);
      if ((l % K) == 0) Zn[(int64_t)v[r] * a.Bw + (b0 >> 5)] = word;
    }
  }
  flush_step_counters<VEC>(a, s_cnt, g, it, b0, lpr, c0, c1, c2, stepm);
}

// ---------------------------------------------------------------- shared memory
// Each lane owns VEC consecutive trajectories (8 or 16 bytes of x), a row
// group of LPR = B/VEC lanes one node, and the RPW = 32/LPR row groups of a
// warp walk their rows' neighbour lists in lockstep, LPR neighbours (one
// chunk) at a time, so one shuffle and one shared-memory load instruction
// serve RPW rows.  An item's rows are taken in decreasing-degree order, so
// the rows of a warp have nearly equal lengths; rows shorter than the
// warp's longest are padded with a
// dummy neighbour, local index ng, whose shared-memory row of x and bit
// words are zero: adding +0.0 leaves a float32 sum that is not -0.0
// unchanged, and sums of values that are never -0.0 are never -0.0, so the
// padded sums equal the CSR-order sums exactly and the inner loop needs no
// predicates.  DUP (64-byte rows): the block of x is stored with a 128-byte
// pitch and each row twice, at bytes [0,64) and [64,128); row groups of odd
// index read the second copy, so the two row groups of a half-warp always
// use opposite halves of the 32 banks.
template <typename TX, typename TV, int VEC, int LPR, bool MIS, bool DUP>
__global__ void __launch_bounds__(512, 2) k_step_s(StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RPW = 32 / LPR;
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
  // the item's rows in processing order: {node, row start, row end}
  int4* s_rows = reinterpret_cast<int4*>(smem + xbytes + zbytes + ((3 * (size_t)B * 8 + 15) & ~(size_t)15));
  const int nrows = item.v1 - item.v0;

  const TX* __restrict__ Xc = static_cast<const TX*>((t & 1) ? a.X1 : a.X0);
  TX* __restrict__ Xn = static_cast<TX*>((t & 1) ? a.X0 : a.X1);
  const uint32_t* __restrict__ Zc = (t & 1) ? a.ZX1 : a.ZX0;
  uint32_t* __restrict__ Zn = (t & 1) ? a.ZX0 : a.ZX1;
  TV* __restrict__ V = static_cast<TV*>(a.V);

  // stage the member graph's x block (16-byte copies), the zero dummy row,
  // and the rounding words
  {
    const int4* src = reinterpret_cast<const int4*>(Xc + (int64_t)off * B);
    const int per = rowb / 16;  // 16-byte pieces per node
    const int n16 = ng * per;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) {
      const int4 vv = src[i];
      const int node = i / per, piece = i - node * per;
      unsigned char* d = smem + (size_t)node * pitch + piece * 16;
      *reinterpret_cast<int4*>(d) = vv;
      if (DUP) *reinterpret_cast<int4*>(d + 64) = vv;
    }
    for (int i = threadIdx.x; i < pitch / 16; i += blockDim.x)
      *reinterpret_cast<int4*>(smem + (size_t)ng * pitch + i * 16) = make_int4(0, 0, 0, 0);
    if (MIS) {
      const uint32_t* zs = Zc + (int64_t)off * BW;
      for (int i = threadIdx.x; i < ng * BW; i += blockDim.x) sZ[i] = zs[i];
      for (int i = threadIdx.x; i < BW; i += blockDim.x) sZ[ng * BW + i] = 0u;
    }
    for (int i = threadIdx.x; i < 3 * B; i += blockDim.x) s_cnt[i] = 0ull;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const int v = a.g.order[item.v0 + i];
      s_rows[i] = make_int4(v, a.g.row_ptr[v], a.g.row_ptr[v + 1], 0);
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR;
  const int l = lane - sub * LPR;
  const int b0 = l * VEC;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const float thr = MIS ? 0.5f : 0.0f;
  const float lo = MIS ? 0.0f : -1.0f;
  const bool weighted = !MIS && a.g.w != nullptr;
  const int32_t* __restrict__ col = a.g.col;
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

  // column indices come in groups of four chunks; each group's loads are
  // issued before the previous group is consumed (software pipeline), and a
  // row's first group during the previous row's epilogue
  int nxu[4], nxw[4];
  auto first_group = [&](int i) {
    const bool h = i < nrows;
    const int4 r = s_rows[h ? i : 0];
    const int rs_ = h ? r.y : 0, re_ = h ? r.z : 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = rs_ + c * LPR + l;
      const bool jin = j < re_;
      nxu[c] = jin ? __ldcs(col + j) - off : ng;
      nxw[c] = jin ? (weighted ? (int)wts[j] : 1) : 0;
    }
  };
  first_group(warp * RPW + sub);
  for (int vb = warp * RPW; vb < nrows; vb += nwarps * RPW) {
    const bool has = vb + sub < nrows;
    const int4 row = s_rows[has ? vb + sub : 0];
    const int v = row.x;
    const int vl = has ? v - off : ng;
    const int64_t base = (int64_t)(has ? v : item.v0) * B + b0;
    const Pack<TX, VEC> xv = *reinterpret_cast<const Pack<TX, VEC>*>(sXl + (size_t)vl * pitch);
    Pack<TV, VEC> vv{};
    if (has) vv = ld_pack_stream<TV, VEC>(V + base);
    float acc[VEC];
    int pos[VEC];
    uint32_t orw[4] = {0u, 0u, 0u, 0u};  // OR of the neighbours' words (BW <= 4)
#pragma unroll
    for (int e = 0; e < VEC; ++e) { acc[e] = 0.0f; pos[e] = 0; }
    const int rs = has ? row.y : 0, re = has ? row.z : 0;
    const int nch_w = __reduce_max_sync(0xffffffffu, (re - rs + LPR - 1) / LPR);
    int wsum = weighted ? 0 : re - rs;
    for (int ch0 = 0; ch0 < nch_w; ch0 += 4) {
      int myo[4], myw[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (MIS)
          for (int w = 0; w < BW; ++w) orw[w] |= sZ[nxu[c] * BW + w];
        myo[c] = nxu[c] * pitch;  // byte offset of the neighbour's row
        myw[c] = nxw[c];
      }
      if (ch0 + 4 < nch_w) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = rs + (ch0 + 4 + c) * LPR + l;
          const bool jin = j < re;
          nxu[c] = jin ? __ldcs(col + j) - off : ng;
          nxw[c] = jin ? (weighted ? (int)wts[j] : 1) : 0;
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (ch0 + c >= nch_w) break;
#pragma unroll
        for (int k = 0; k < LPR; ++k) {
          const int o = __shfl_sync(0xffffffffu, myo[c], k, LPR);
          if constexpr (MIS && std::is_same<TX, __nv_bfloat16>::value) {
            // one mixed-precision add per trajectory: the bfloat16 operand is
            // widened exactly inside the add, which rounds once (RN), so the
            // sums are those of the widened values added one by one
            add_bf16_row<VEC>(acc, sXl + o);
            continue;
          }
          float f[VEC];
          load_unpack<TX, VEC>(sXl + o, f);
          if (weighted) {
            const int w = __shfl_sync(0xffffffffu, myw[c], k, LPR);
            wsum += w;
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
              acc[e] = w >= 0 ? acc[e] + f[e] : acc[e] - f[e];
              pos[e] += (f[e] > thr) ? w : 0;
            }
          } else {
            // two trajectories per packed add (IEEE round-to-nearest per
            // element: the same sums as one scalar add each)
#pragma unroll
            for (int e = 0; e < VEC; e += 2) add_f32x2(acc[e], acc[e + 1], f[e], f[e + 1]);
            if (!MIS) {
#pragma unroll
              for (int e = 0; e < VEC; ++e) pos[e] += (f[e] > thr);
            }
          }
        }
      }
    }
    first_group(vb + nwarps * RPW + sub);
    if (MIS) {
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
                           vo.e[e],
                           zn, d0, d1, d2);
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
  }
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    if constexpr (MIS) c0[e] = (int)(cp[e] & 1023u);
    c1[e] = (int)((cp[e] >> 10) & 1023u);
    c2[e] = (int)(cp[e] >> 20);
  }
  flush_step_counters<VEC>(a, s_cnt, g, it, b0, LPR, c0, c1, c2, stepm);
}

size_t step_smem_bytes(int B, int x_dtype, int problem, int max_ng) {
  const size_t sx = x_dtype == DT_F32 ? 4 : 2;
  const size_t rowb = (size_t)B * sx;
  const size_t pitch = rowb == 64 ? 128 : rowb;
  const size_t xb = ((size_t)(max_ng + 1) * pitch + 15) & ~(size_t)15;
  const size_t zb = problem == PROB_MIS ? (((size_t)(max_ng + 1) * ((B + 31) / 32) * 4 + 15) & ~(size_t)15) : 0;
  return xb + zb + ((3 * (size_t)B * 8 + 15) & ~(size_t)15) + (size_t)kItemMaxNodes * 16;
}

template <typename TX, typename TV, int VEC, int LPR, bool MIS, bool DUP>
static cudaError_t launch_s(size_t smem, const StepArgs& a, int grid, cudaStream_t s) {
  if (a.B != VEC * LPR) return cudaErrorInvalidValue;
  cudaFuncSetAttribute(k_step_s<TX, TV, VEC, LPR, MIS, DUP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_step_s<TX, TV, VEC, LPR, MIS, DUP><<<grid, 512, smem, s>>>(a);
  return cudaGetLastError();
}

// lanes hold 8 bytes of x, or 16 when B/32 elements need more:
// 2-byte x: B=32 -> (VEC 4, LPR 8, DUP), B=64 -> (4, 16), B=128 -> (4, 32);
// 4-byte x: B=32 -> (2, 16), B=64 -> (2, 32), B=128 -> (4, 32).
// Wide lanes (16 bytes, half the lanes per row, twice the rows per warp):
// 2-byte x: B=32 -> (8, 4, DUP), B=64 -> (8, 8), B=128 -> (8, 16);
// 4-byte x: B=32 -> (4, 8), B=64 -> (4, 16)
template <typename TX, typename TV>
static cudaError_t launch_smem(int B, bool wide, size_t smem, bool mis, const StepArgs& a, int grid, cudaStream_t s) {
  if constexpr (sizeof(TX) == 2) {
    if (wide) {
      if (mis) {
        if (B == 32) return launch_s<TX, TV, 8, 4, true, true>(smem, a, grid, s);
        if (B == 64) return launch_s<TX, TV, 8, 8, true, false>(smem, a, grid, s);
        if (B == 128) return launch_s<TX, TV, 8, 16, true, false>(smem, a, grid, s);
      } else {
        if (B == 32) return launch_s<TX, TV, 8, 4, false, true>(smem, a, grid, s);
        if (B == 64) return launch_s<TX, TV, 8, 8, false, false>(smem, a, grid, s);
        if (B == 128) return launch_s<TX, TV, 8, 16, false, false>(smem, a, grid, s);
      }
    } else if (mis) {
      if (B == 32) return launch_s<TX, TV, 4, 8, true, true>(smem, a, grid, s);
      if (B == 64) return launch_s<TX, TV, 4, 16, true, false>(smem, a, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, true, false>(smem, a, grid, s);
    } else {
      if (B == 32) return launch_s<TX, TV, 4, 8, false, true>(smem, a, grid, s);
      if (B == 64) return launch_s<TX, TV, 4, 16, false, false>(smem, a, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, false, false>(smem, a, grid, s);
    }
  } else {
    if (wide) {
      if (mis) {
        if (B == 32) return launch_s<TX, TV, 4, 8, true, false>(smem, a, grid, s);
        if (B == 64) return launch_s<TX, TV, 4, 16, true, false>(smem, a, grid, s);
      } else {
        if (B == 32) return launch_s<TX, TV, 4, 8, false, false>(smem, a, grid, s);
        if (B == 64) return launch_s<TX, TV, 4, 16, false, false>(smem, a, grid, s);
      }
    } else if (mis) {
      if (B == 32) return launch_s<TX, TV, 2, 16, true, false>(smem, a, grid, s);
      if (B == 64) return launch_s<TX, TV, 2, 32, true, false>(smem, a, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, true, false>(smem, a, grid, s);
    } else {
      if (B == 32) return launch_s<TX, TV, 2, 16, false, false>(smem, a, grid, s);
      if (B == 64) return launch_s<TX, TV, 2, 32, false, false>(smem, a, grid, s);
      if (B == 128) return launch_s<TX, TV, 4, 32, false, false>(smem, a, grid, s);
    }
  }
  return cudaErrorInvalidValue;
}

// Default trajectories per lane of the global-memory step kernel (before
// any autotuning): at least 8 bytes of x per lane where the batch allows it,
// and at most 32 lanes per row.
int default_step_vec(int B, int x_dtype) {
  const int sx = x_dtype == DT_F32 ? 4 : 2;
  int vec = 8 / sx;
  if (vec < B / 32) vec = B / 32;
  if (vec > B) vec = B;
  if (vec > 4) vec = 4;
  return vec;
}

bool step_wide_possible(int B, int x_dtype) { return x_dtype != DT_F32 ? (B == 32 || B == 64 || B == 128) : (B == 32 || B == 64); }

template <typename TX, typename TV, int VEC>
static cudaError_t launch_vec(const StepArgs& a, int grid, cudaStream_t s) {
  if (a.problem == PROB_MIS) k_step_g<TX, TV, VEC, true, false><<<grid, 512, 0, s>>>(a);
  else if (a.g.w) k_step_g<TX, TV, VEC, false, true><<<grid, 512, 0, s>>>(a);
  else k_step_g<TX, TV, VEC, false, false><<<grid, 512, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename TX, typename TV>
static cudaError_t launch_tv(int vec, bool smem_path, bool wide, size_t smem, bool mis, const StepArgs& a,
                             int grid, cudaStream_t s) {
  if (smem_path) return launch_smem<TX, TV>(a.B, wide, smem, mis, a, grid, s);
  switch (vec) {
    case 1: return launch_vec<TX, TV, 1>(a, grid, s);
    case 2: return launch_vec<TX, TV, 2>(a, grid, s);
    case 4: return launch_vec<TX, TV, 4>(a, grid, s);
    case 8:
      if constexpr (sizeof(TX) == 2 && sizeof(TV) == 2) return launch_vec<TX, TV, 8>(a, grid, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(const SolverDev& S, Counters* cnt, const int32_t* act, const int32_t* gflag_step,
                        size_t smem, cudaStream_t stream) {
  StepArgs a;
  a.g = S.g;
  a.B = S.B;
  a.Bw = S.Bw;
  a.R = S.R;
  a.problem = S.p.problem;
  a.objective = S.p.objective;
  a.alpha = S.p.alpha;
  a.momentum = S.p.momentum;
  a.gamma = S.p.gamma;
  a.lambda_ = S.p.lambda_;
  a.X0 = S.X0;
  a.X1 = S.X1;
  a.V = S.V;
  a.ZX0 = S.ZX0;
  a.ZX1 = S.ZX1;
  a.cnt = cnt;
  a.split = 1;
  a.act = act;
  a.gflag_step = gflag_step;
  a.tick = S.tick;
  const int vec = S.step_vec > 0 ? S.step_vec : default_step_vec(S.B, S.p.x_dtype);
  const bool sp = smem > 0;
  const bool wide = S.step_wide != 0;
  const bool mis = S.p.problem == PROB_MIS;
  int grid = S.g.num_items;
  if (!sp) {  // few items (a handful of member graphs): several CTAs per item
    a.split = S.split;
    grid = S.g.num_items * a.split;
  }
  const int xd = S.p.x_dtype, vd = S.p.v_dtype;
  if (xd == DT_F32) return launch_tv<float, float>(vec, sp, wide, smem, mis, a, grid, stream);
  if (xd == DT_BF16 && vd == DT_BF16) return launch_tv<__nv_bfloat16, __nv_bfloat16>(vec, sp, wide, smem, mis, a, grid, stream);
  if (xd == DT_BF16 && vd == DT_F32) return launch_tv<__nv_bfloat16, float>(vec, sp, wide, smem, mis, a, grid, stream);
  if (xd == DT_F16 && vd == DT_F16) return launch_tv<__half, __half>(vec, sp, wide, smem, mis, a, grid, stream);
  if (xd == DT_F16 && vd == DT_F32) return launch_tv<__half, float>(vec, sp, wide, smem, mis, a, grid, stream);
  return cudaErrorInvalidValue;
}

}  // namespace mqo
