// mqo_step.cu -- the fused descent step (one tick of gradient work).
//
// For every node v and trajectory b of a stepping trajectory:
//   (A x)_vb  = sum over the CSR row of v, in row order, of w_vu x_ub (float32)
//   grad      = 1 - gamma (A x)_vb              (h, Eq. MIS QUBO)
//             | -lambda - 2 (A x)_vb            (f_B, Eq. adj_lin_two_props)
//   V'        = mu V + alpha grad               (momentum ascent, Sec. 5)
//   x'        = Pi_box(x + V')                  (projection of Sec. 3)
// and, from the same neighbour gather, the exact evaluation of the rounded
// incoming point z = [x > 0.5] (MIS) or [x > 0] (MaxCut): set size,
// conflicting and uncovered nodes (checker, Eq. MIS checking), or cut,
// nodes violating the f_B fixed-point condition and positive-gain nodes.
//
// Thread mapping: a row group of LPR = B/VEC lanes handles one node; lane l
// owns trajectories l*VEC .. l*VEC+VEC-1 and accumulates them sequentially
// over the row, so every (v,b) sum is in CSR order.  Rows are streamed in
// items (node ranges inside one member graph); per-item integer counters
// are reduced in shared memory and flushed with one atomic per trajectory.
#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

struct StepArgs {
  GraphDev g;
  int32_t B, Bw, problem;
  float alpha, momentum, gamma, lambda_;
  const void* X0;      // x buffers: tick t reads X[t&1], writes X[(t+1)&1]
  void* X1;
  void* V;             // momentum (read/write)
  uint32_t* zout;      // z of the current x, node-major bits
  Counters* cnt;       // per-trajectory counters
  const TrajState* st; // nullptr: every trajectory steps
  const int32_t* gflag_step;
  const int64_t* tick;
};

template <typename TX, typename TV, int VEC>
__global__ void __launch_bounds__(256) k_step(StepArgs a) {
  extern __shared__ unsigned long long smem_u64[];
  const int B = a.B;
  unsigned long long* s_cnt = smem_u64;              // [B][3]
  int* s_step = reinterpret_cast<int*>(s_cnt + 3 * B);  // [B]

  const int lpr = B / VEC;
  const int rpw = 32 / lpr;
  const int lane = threadIdx.x & 31;
  const int sub = lane / lpr;
  const int l = lane - sub * lpr;
  const int b0 = l * VEC;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int64_t t = *a.tick;
  const bool mis = a.problem == PROB_MIS;
  const float thr = mis ? 0.5f : 0.0f;
  const float lo = mis ? 0.0f : -1.0f;
  const bool weighted = a.g.w != nullptr;
  const TX* __restrict__ Xc = static_cast<const TX*>((t & 1) ? a.X1 : a.X0);
  TX* __restrict__ Xn = static_cast<TX*>((t & 1) ? const_cast<void*>(a.X0) : a.X1);
  TV* __restrict__ V = static_cast<TV*>(a.V);
  const int32_t* __restrict__ rp = a.g.row_ptr;
  const int32_t* __restrict__ col = a.g.col;
  const int8_t* __restrict__ wts = a.g.w;
  // lanes sharing one output bit word
  const int K = (lpr < 32 / VEC) ? lpr : 32 / VEC;
  const unsigned rmask = lpr == 32 ? 0xffffffffu : (((1u << lpr) - 1u) << (sub * lpr));

  for (int it = blockIdx.x; it < a.g.num_items; it += gridDim.x) {
    const Item item = a.g.items[it];
    const int g = item.g;
    if (a.gflag_step && a.gflag_step[g] != (int32_t)(t + 1)) continue;
    for (int i = threadIdx.x; i < 3 * B; i += blockDim.x) s_cnt[i] = 0ull;
    for (int i = threadIdx.x; i < B; i += blockDim.x)
      s_step[i] = a.st ? (a.st[(int64_t)g * B + i].act & ACT_STEP) : 1;
    __syncthreads();

    bool stepping[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) stepping[e] = s_step[b0 + e] != 0;
    int c0[VEC], c1[VEC], c2[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) c0[e] = c1[e] = c2[e] = 0;

    for (int v = item.v0 + warp * rpw + sub; v < item.v1; v += nwarps * rpw) {
      const int64_t base = (int64_t)v * B + b0;
      const Pack<TX, VEC> xv = ld_pack<TX, VEC>(Xc + base);
      const Pack<TV, VEC> vv = ld_pack_stream<TV, VEC>(V + base);
      float acc[VEC];
      int pos[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) { acc[e] = 0.0f; pos[e] = 0; }
      const int rs = rp[v], re = rp[v + 1];
      int wsum = re - rs;
      if (!weighted) {
        int j = rs;
        for (; j + 4 <= re; j += 4) {
          const int u0 = __ldcs(col + j), u1 = __ldcs(col + j + 1), u2 = __ldcs(col + j + 2),
                    u3 = __ldcs(col + j + 3);
          const Pack<TX, VEC> p0 = ld_pack<TX, VEC>(Xc + (int64_t)u0 * B + b0);
          const Pack<TX, VEC> p1 = ld_pack<TX, VEC>(Xc + (int64_t)u1 * B + b0);
          const Pack<TX, VEC> p2 = ld_pack<TX, VEC>(Xc + (int64_t)u2 * B + b0);
          const Pack<TX, VEC> p3 = ld_pack<TX, VEC>(Xc + (int64_t)u3 * B + b0);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float f0 = to_f(p0.e[e]), f1 = to_f(p1.e[e]), f2 = to_f(p2.e[e]), f3 = to_f(p3.e[e]);
            acc[e] = acc[e] + f0;
            acc[e] = acc[e] + f1;
            acc[e] = acc[e] + f2;
            acc[e] = acc[e] + f3;
            pos[e] += (f0 > thr) + (f1 > thr) + (f2 > thr) + (f3 > thr);
          }
        }
        for (; j < re; ++j) {
          const int u = __ldcs(col + j);
          const Pack<TX, VEC> p = ld_pack<TX, VEC>(Xc + (int64_t)u * B + b0);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float f = to_f(p.e[e]);
            acc[e] = acc[e] + f;
            pos[e] += (f > thr);
          }
        }
      } else {
        wsum = 0;
        for (int j = rs; j < re; ++j) {
          const int u = __ldcs(col + j);
          const int w = wts[j];
          wsum += w;
          const Pack<TX, VEC> p = ld_pack<TX, VEC>(Xc + (int64_t)u * B + b0);
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const float f = to_f(p.e[e]);
            if (w >= 0) acc[e] = acc[e] + f;
            else acc[e] = acc[e] - f;
            pos[e] += (f > thr) ? w : 0;
          }
        }
      }

      Pack<TX, VEC> xo;
      Pack<TV, VEC> vo;
      unsigned zbits = 0u;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float x = to_f(xv.e[e]);
        const float vold = to_f(vv.e[e]);
        const bool z = x > thr;
        zbits |= (unsigned)z << e;
        if (mis) {
          const bool any = pos[e] > 0;
          c0[e] += z;
          c1[e] += z && any;
          c2[e] += !z && !any;
        } else {
          const int as = 2 * pos[e] - wsum;
          c0[e] += z ? (wsum - pos[e]) : pos[e];
          const bool fixed = z ? (as <= -1) : (as >= 0);
          c1[e] += !fixed;
          const int gn = z ? as : -as;
          c2[e] += gn > 0;
        }
        float grad;
        if (mis) {
          const float tt = a.gamma * acc[e];
          grad = 1.0f - tt;
        } else {
          const float tt = 2.0f * acc[e];
          grad = -a.lambda_ - tt;
        }
        const float m1 = a.momentum * vold;
        const float m2 = a.alpha * grad;
        const float vn = m1 + m2;
        const float xn = clamp_box(x + vn, lo, 1.0f);
        xo.e[e] = stepping[e] ? from_f<TX>(xn) : xv.e[e];
        vo.e[e] = stepping[e] ? from_f<TV>(vn) : vv.e[e];
      }
      st_pack<TX, VEC>(Xn + base, xo);
      st_pack<TV, VEC>(V + base, vo);
      // gather the bits of the lanes sharing this output word
      unsigned word = zbits << (b0 & 31);
      for (int off = 1; off < K; off <<= 1) word |= __shfl_xor_sync(rmask, word, off);
      if ((l % K) == 0) a.zout[(int64_t)v * a.Bw + (b0 >> 5)] = word;
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      if (c0[e]) atomicAdd(&s_cnt[3 * (b0 + e) + 0], (unsigned long long)(long long)c0[e]);
      if (c1[e]) atomicAdd(&s_cnt[3 * (b0 + e) + 1], (unsigned long long)(long long)c1[e]);
      if (c2[e]) atomicAdd(&s_cnt[3 * (b0 + e) + 2], (unsigned long long)(long long)c2[e]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * B; i += blockDim.x) {
      const int bb = i / 3, k = i - 3 * bb;
      const unsigned long long val = s_cnt[i];
      if (val && s_step[bb]) {
        Counters* c = a.cnt + (int64_t)g * B + bb;
        unsigned long long* dst = k == 0 ? &c->value : (k == 1 ? &c->a : &c->b);
        atomicAdd(dst, val);
      }
    }
    __syncthreads();
  }
}

template <typename TX, typename TV>
static cudaError_t launch_tv(int vec, const StepArgs& a, int grid, cudaStream_t s) {
  const size_t sm = (size_t)a.B * (3 * sizeof(unsigned long long) + sizeof(int));
  switch (vec) {
    case 1: k_step<TX, TV, 1><<<grid, 256, sm, s>>>(a); break;
    case 2: k_step<TX, TV, 2><<<grid, 256, sm, s>>>(a); break;
    case 4: k_step<TX, TV, 4><<<grid, 256, sm, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_step(const SolverDev& S, uint32_t* zout, Counters* cnt, const TrajState* st,
                        const int32_t* gflag_step, int grid, cudaStream_t stream) {
  StepArgs a;
  a.g = S.g;
  a.B = S.B;
  a.Bw = S.Bw;
  a.problem = S.p.problem;
  a.alpha = S.p.alpha;
  a.momentum = S.p.momentum;
  a.gamma = S.p.gamma;
  a.lambda_ = S.p.lambda_;
  a.X0 = S.X0;
  a.X1 = S.X1;
  a.V = S.V;
  a.zout = zout;
  a.cnt = cnt;
  a.st = st;
  a.gflag_step = gflag_step;
  a.tick = S.tick;
  const int vec = S.B >= 32 ? S.B / 32 : 1;
  const int xd = S.p.x_dtype, vd = S.p.v_dtype;
  if (xd == DT_F32) return launch_tv<float, float>(vec, a, grid, stream);
  if (xd == DT_BF16 && vd == DT_BF16) return launch_tv<__nv_bfloat16, __nv_bfloat16>(vec, a, grid, stream);
  if (xd == DT_BF16 && vd == DT_F32) return launch_tv<__nv_bfloat16, float>(vec, a, grid, stream);
  if (xd == DT_F16 && vd == DT_F16) return launch_tv<__half, __half>(vec, a, grid, stream);
  if (xd == DT_F16 && vd == DT_F32) return launch_tv<__half, float>(vec, a, grid, stream);
  return cudaErrorInvalidValue;
}

}  // namespace mqo
