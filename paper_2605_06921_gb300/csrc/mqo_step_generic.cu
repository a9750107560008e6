// mqo_step_generic.cu -- the fused descent step for any graph: neighbour rows
// of x gathered from global memory (L2), the item's CSR staged in shared
// memory.  The step itself (gradient, momentum, projection, rounding, exact
// evaluation) is the one of mqo_step.cuh.
#include "mqo_step.cuh"

namespace mqo {

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

template <typename TX, typename TV, int VEC, bool MIS, bool WEIGHTED, int OBJ>
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
        step_element<TX, TV, OBJ>(a, MIS, thr, lo, xv[r].e[e], vv[r].e[e], acc[r][e], pos[r][e], wsum[r],
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

template <typename TX, typename TV, int VEC>
static cudaError_t launch_vec(const StepArgs& a, int grid, cudaStream_t s) {
  const bool fb = a.objective == OBJ_FB;
  if (a.problem == PROB_MIS) k_step_g<TX, TV, VEC, true, false, -1><<<grid, 512, 0, s>>>(a);
  else if (a.g.w && fb) k_step_g<TX, TV, VEC, false, true, OBJ_FB><<<grid, 512, 0, s>>>(a);
  else if (a.g.w) k_step_g<TX, TV, VEC, false, true, -1><<<grid, 512, 0, s>>>(a);
  else if (fb) k_step_g<TX, TV, VEC, false, false, OBJ_FB><<<grid, 512, 0, s>>>(a);
  else k_step_g<TX, TV, VEC, false, false, -1><<<grid, 512, 0, s>>>(a);
  return cudaGetLastError();
}

// The global-memory step kernel for the solver's storage types.
cudaError_t launch_step_generic(const StepArgs& a, int vec, int x_dtype, int v_dtype, int grid, cudaStream_t s) {
  auto go = [&](auto tx, auto tv) -> cudaError_t {
    using TX = decltype(tx);
    using TV = decltype(tv);
    switch (vec) {
      case 1: return launch_vec<TX, TV, 1>(a, grid, s);
      case 2: return launch_vec<TX, TV, 2>(a, grid, s);
      case 4: return launch_vec<TX, TV, 4>(a, grid, s);
      case 8:
        if constexpr (sizeof(TX) == 2 && sizeof(TV) == 2) return launch_vec<TX, TV, 8>(a, grid, s);
        return cudaErrorInvalidValue;
      default: return cudaErrorInvalidValue;
    }
  };
  if (x_dtype == DT_F32) return go(float{}, float{});
  if (x_dtype == DT_BF16 && v_dtype == DT_BF16) return go(__nv_bfloat16{}, __nv_bfloat16{});
  if (x_dtype == DT_BF16 && v_dtype == DT_F32) return go(__nv_bfloat16{}, float{});
  if (x_dtype == DT_F16 && v_dtype == DT_F16) return go(__half{}, __half{});
  if (x_dtype == DT_F16 && v_dtype == DT_F32) return go(__half{}, float{});
  return cudaErrorInvalidValue;
}

}  // namespace mqo
