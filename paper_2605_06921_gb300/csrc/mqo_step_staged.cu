// mqo_step_staged.cu -- the fused descent step for any graph, with every
// neighbour row of x a slice needs copied into shared memory before any sum
// starts.  The step itself (gradient, momentum, projection, rounding, exact
// evaluation) is the one of mqo_step.cuh.
//
// Large graphs (x far larger than L2) make the step a stream of random
// 32- to 256-byte row gathers.  Issued one row group at a time, a few per
// row, they leave the memory system mostly idle (latency-bound); here a CTA
// owns a slice of at most `slice_rows` consecutive rows of one work item
// whose neighbour rows take at most `slice_cols` rows of x, and
//   1. copies the slice's row pointers and column indices (and weights),
//   2. issues cp.async copies (16 bytes each, L2 only) of its own rows of x
//      and V and of the x row of every CSR entry of the slice, in CSR order,
//      all at once: one slice keeps tens of kilobytes of gathers in flight,
//      and several resident CTAs overlap one slice's gathers with another's
//      arithmetic;
//   3. waits, then the row groups of a warp sum their rows' neighbours in
//      CSR order from shared memory, in lockstep over the warp's longest row
//      (same float32 sums as the other step kernels), and run the step tail.
// Requirements (checked on the host): a row of x and a row of V are
// multiples of 16 bytes, and every row's neighbours fit in one slice.
#include "mqo_step.cuh"

namespace mqo {

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// VEC elements of T at p (aligned) as floats
template <typename T, int VEC>
__device__ __forceinline__ void unpack_row(const unsigned char* p, float* f) {
  if constexpr (std::is_same<T, float>::value && VEC == 8) {
    load_unpack<float, 4>(p, f);
    load_unpack<float, 4>(p + 16, f + 4);
  } else {
    load_unpack<T, VEC>(p, f);
  }
}

// (a, b) += the two 16-bit elements of word w, one mixed-precision add each
// (sm_100 family: the 16-bit operand is widened exactly inside the add, which
// rounds once, so the sums equal widening first and adding in float32)
template <typename TX>
__device__ __forceinline__ void add_x16x2_word(float& a, float& b, uint32_t w);
template <>
__device__ __forceinline__ void add_x16x2_word<__nv_bfloat16>(float& a, float& b, uint32_t w) {
  add_bf16x2_word(a, b, w);
}
template <>
__device__ __forceinline__ void add_x16x2_word<__half>(float& a, float& b, uint32_t w) {
  asm("{\n\t.reg .b16 lo, hi;\n\t"
      "mov.b32 {lo, hi}, %2;\n\t"
      "add.rn.f32.f16 %0, lo, %0;\n\t"
      "add.rn.f32.f16 %1, hi, %1;\n\t}"
      : "+f"(a), "+f"(b)
      : "r"(w));
}
// the 16-bit pattern of 0.5: for values in [0, 1] the patterns read as
// signed 16-bit integers order like the values (-0 reads as negative), so
// "some neighbour has x > 0.5" is "the running max of the patterns > it"
template <typename TX>
constexpr int16_t kHalfPattern = std::is_same<TX, __half>::value ? (int16_t)0x3800 : (int16_t)0x3F00;

template <typename TX, typename TV, int VEC, bool MIS, bool WEIGHTED, int OBJ>
__global__ void __launch_bounds__(kStagedThreads, VEC >= 8 ? 2 : 4) k_step_q(StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Slice sl = a.slices[blockIdx.x];
  const int g = sl.g;
  const int64_t t = *a.tick;
  if (a.gflag_step && a.gflag_step[g] != (int32_t)(t + 1)) return;
  const int B = a.B;
  const int rowx = B * (int)sizeof(TX), rowv = B * (int)sizeof(TV);
  const int nrows = sl.v1 - sl.v0;
  const StagedLayout L = staged_layout(B, (int)sizeof(TX), (int)sizeof(TV), a.slice_cols, a.slice_rows, WEIGHTED);
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(smem + L.cnt);
  int32_t* s_rp = reinterpret_cast<int32_t*>(smem + L.rp);
  int32_t* s_col = reinterpret_cast<int32_t*>(smem + L.col);
  int8_t* s_w = reinterpret_cast<int8_t*>(smem + L.w);
  unsigned char* s_xo = smem + L.xo;
  unsigned char* s_vo = smem + L.vo;
  unsigned char* s_nb = smem + L.nb;

  const TX* __restrict__ Xc = static_cast<const TX*>((t & 1) ? a.X1 : a.X0);
  TX* __restrict__ Xn = static_cast<TX*>((t & 1) ? a.X0 : a.X1);
  uint32_t* __restrict__ Zn = (t & 1) ? a.ZX0 : a.ZX1;
  TV* __restrict__ V = static_cast<TV*>(a.V);
  const int32_t* __restrict__ rp = a.g.row_ptr;
  const int32_t* __restrict__ col = a.g.col;
  const int8_t* __restrict__ wts = a.g.w;
  const int nt = blockDim.x;
  const int tid = threadIdx.x;

  // 1. counters, row pointers (relative to the slice), column indices;
  //    the own rows of x and V go out as cp.async copies right away
  const int32_t j0 = rp[sl.v0];
  const int32_t ncol = rp[sl.v1] - j0;
  for (int i = tid; i < 3 * B; i += nt) s_cnt[i] = 0ull;
  for (int i = tid; i <= nrows; i += nt) s_rp[i] = rp[sl.v0 + i] - j0;
  for (int i = tid; i < ncol; i += nt) {
    s_col[i] = __ldcs(col + j0 + i);
    if constexpr (WEIGHTED) s_w[i] = __ldcs(wts + j0 + i);
  }
  {
    const unsigned char* xs = reinterpret_cast<const unsigned char*>(Xc + (int64_t)sl.v0 * B);
    const unsigned char* vs = reinterpret_cast<const unsigned char*>(V + (int64_t)sl.v0 * B);
    const int nx = nrows * rowx / 16, nv = nrows * rowv / 16;
    for (int i = tid; i < nx; i += nt) cp_async16(s_xo + 16 * i, xs + 16 * i);
    for (int i = tid; i < nv; i += nt) cp_async16(s_vo + 16 * i, vs + 16 * i);
  }
  __syncthreads();
  // 2. the x row of every entry, in CSR order: entry j's row at s_nb + j*rowx
  {
    const int sh = __ffs(rowx >> 4) - 1;  // rowx / 16 is a power of two
    const int per = 1 << sh;
    const int total = ncol << sh;
    const unsigned char* xb = reinterpret_cast<const unsigned char*>(Xc);
    for (int e = tid; e < total; e += nt) {
      const int j = e >> sh;
      const int c = e & (per - 1);
      cp_async16(s_nb + 16 * e, xb + (int64_t)s_col[j] * rowx + 16 * c);
    }
  }
  // the lane's trajectories and which of them step this tick
  const int lpr = B / VEC;
  const int rpw = 32 / lpr;
  const int lane = tid & 31;
  const int sub = lane / lpr;
  const int l = lane - sub * lpr;
  const int b0 = l * VEC;
  const int warp = tid >> 5;
  const int nwarps = nt >> 5;
  uint32_t stepm = 0u;
#pragma unroll
  for (int e = 0; e < VEC; ++e)
    stepm |= (uint32_t)(a.act ? (a.act[(int64_t)g * B + b0 + e] & ACT_STEP) != 0 : true) << e;
  int c0[VEC], c1[VEC], c2[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) c0[e] = c1[e] = c2[e] = 0;
  const float thr = MIS ? 0.5f : 0.0f;
  const float lo = MIS ? 0.0f : -1.0f;
  const int K = (lpr < 32 / VEC) ? lpr : 32 / VEC;  // lanes sharing one output bit word
  const unsigned rmask = lpr == 32 ? 0xffffffffu : (((1u << lpr) - 1u) << (sub * lpr));
  // a zero row of x for the padded steps of lockstep rows (rows of x are at
  // most B = 256 values of 4 bytes)
  __shared__ __align__(16) unsigned char s_zero[1024];
  for (int i = tid; i < 1024 / 16; i += nt) reinterpret_cast<int4*>(s_zero)[i] = make_int4(0, 0, 0, 0);
  cp_async_wait_all();
  __syncthreads();

  // 3. the rows of a warp in lockstep (row group sub takes row vr0 + sub),
  //    each summing its neighbours in CSR order for as many steps as the
  //    warp's longest row; a row's steps past its end read the zero row:
  //    adding +0.0 leaves a float32 sum that is not -0.0 unchanged (and the
  //    sums are never -0.0), so the sums equal the CSR-order sums and the
  //    loop has no per-row branches.  MIS with 16-bit x: one mixed-precision
  //    add per element, and the checker's "some neighbour in the set" from a
  //    running signed max of the gathered 16-bit words.
  constexpr bool kMax16 = MIS && sizeof(TX) == 2 && (VEC == 2 || VEC == 4 || VEC == 8);
  constexpr int NW = VEC / 2 > 0 ? VEC / 2 : 1;  // 32-bit words of a lane's elements
  const unsigned char* zp = s_zero + b0 * (int)sizeof(TX);
  for (int vr0 = warp * rpw; vr0 < nrows; vr0 += nwarps * rpw) {
    const int vr = vr0 + sub;
    const bool has = vr < nrows;
    const int vrc = has ? vr : 0;
    const int rs = has ? s_rp[vr] : 0, re = has ? s_rp[vr + 1] : 0;
    const int len = re - rs;
    const int nmax = __reduce_max_sync(0xffffffffu, len);
    const Pack<TX, VEC> xv = *reinterpret_cast<const Pack<TX, VEC>*>(s_xo + vrc * rowx + b0 * (int)sizeof(TX));
    const Pack<TV, VEC> vv = *reinterpret_cast<const Pack<TV, VEC>*>(s_vo + vrc * rowv + b0 * (int)sizeof(TV));
    float acc[VEC];
    int pos[VEC];
    uint32_t mx[NW];
#pragma unroll
    for (int e = 0; e < VEC; ++e) { acc[e] = 0.0f; pos[e] = 0; }
#pragma unroll
    for (int w = 0; w < NW; ++w) mx[w] = 0u;
    int wsum = WEIGHTED ? 0 : len;
    const unsigned char* p = s_nb + rs * rowx + b0 * (int)sizeof(TX);
#pragma unroll 4
    for (int k = 0; k < nmax; ++k) {
      const bool in = k < len;
      const unsigned char* q = in ? p + k * rowx : zp;
      if constexpr (kMax16) {
        uint32_t wd[NW];
        if constexpr (VEC == 8) {
          const uint4 r = *reinterpret_cast<const uint4*>(q);
          wd[0] = r.x, wd[1] = r.y, wd[2] = r.z, wd[3] = r.w;
        } else if constexpr (VEC == 4) {
          const uint2 r = *reinterpret_cast<const uint2*>(q);
          wd[0] = r.x, wd[1] = r.y;
        } else {
          wd[0] = *reinterpret_cast<const uint32_t*>(q);
        }
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          add_x16x2_word<TX>(acc[2 * w], acc[2 * w + 1], wd[w]);
          mx[w] = __vmaxs2(mx[w], wd[w]);
        }
      } else {
        float f[VEC];
        unpack_row<TX, VEC>(q, f);
        if constexpr (WEIGHTED) {
          const int w = in ? (int)s_w[rs + k] : 0;
          wsum += w;
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            acc[e] = w >= 0 ? acc[e] + f[e] : acc[e] - f[e];
            pos[e] += (f[e] > thr) ? w : 0;
          }
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            acc[e] = acc[e] + f[e];
            pos[e] += (f[e] > thr);
          }
        }
      }
    }
    if constexpr (kMax16) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const int16_t h = (int16_t)(uint16_t)(mx[e >> 1] >> (16 * (e & 1)));
        pos[e] = h > kHalfPattern<TX>;
      }
    }
    if (!has) continue;  // the whole row group (its lanes share vr)
    Pack<TX, VEC> xo;
    Pack<TV, VEC> vo;
    unsigned zbits = 0u;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      bool zn;
      step_element<TX, TV, OBJ>(a, MIS, thr, lo, xv.e[e], vv.e[e], acc[e], pos[e], wsum, (stepm >> e) & 1u, xo.e[e],
                           vo.e[e], zn, c0[e], c1[e], c2[e]);
      zbits |= (unsigned)zn << e;
    }
    const int64_t v = sl.v0 + vr;
    const int64_t base = v * B + b0;
    st_pack<TX, VEC>(Xn + base, xo);
    st_pack<TV, VEC>(V + base, vo);
    unsigned word = zbits << (b0 & 31);
    for (int o = 1; o < K; o <<= 1) word |= __shfl_xor_sync(rmask, word, o);
    if ((l % K) == 0) Zn[v * a.Bw + (b0 >> 5)] = word;
  }
  flush_step_counters<VEC>(a, s_cnt, g, sl.it, b0, lpr, c0, c1, c2, stepm);
}

template <typename TX, typename TV, int VEC>
static cudaError_t launch_q_vec(const StepArgs& a, size_t smem, cudaStream_t s) {
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.num_slices, kStagedThreads, smem, s>>>(a);
    return cudaGetLastError();
  };
  const bool fb = a.objective == OBJ_FB;
  if (a.problem == PROB_MIS) return run(k_step_q<TX, TV, VEC, true, false, -1>);
  if (a.g.w) return fb ? run(k_step_q<TX, TV, VEC, false, true, OBJ_FB>) : run(k_step_q<TX, TV, VEC, false, true, -1>);
  return fb ? run(k_step_q<TX, TV, VEC, false, false, OBJ_FB>) : run(k_step_q<TX, TV, VEC, false, false, -1>);
}

bool staged_vec_ok(int B, int x_dtype, int vec) {
  if (vec != 2 && vec != 4 && vec != 8) return false;
  (void)x_dtype;
  return B % vec == 0 && B / vec <= 32 && 32 % (B / vec) == 0;
}

int default_staged_vec(int B, int x_dtype) {
  // 8 bytes of x per lane, at most 32 lanes per row
  int vec = x_dtype == DT_F32 ? 2 : 4;
  while (vec < 8 && B / vec > 32) vec *= 2;
  return vec;
}

cudaError_t launch_step_staged(const StepArgs& a, int vec, int x_dtype, int v_dtype, size_t smem, cudaStream_t s) {
  if (a.num_slices == 0) return cudaSuccess;
  auto go = [&](auto tx, auto tv) -> cudaError_t {
    using TX = decltype(tx);
    using TV = decltype(tv);
    switch (vec) {
      case 2: return launch_q_vec<TX, TV, 2>(a, smem, s);
      case 4: return launch_q_vec<TX, TV, 4>(a, smem, s);
      case 8: return launch_q_vec<TX, TV, 8>(a, smem, s);
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
