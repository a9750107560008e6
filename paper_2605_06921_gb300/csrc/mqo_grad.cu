// mqo_grad.cu -- f_B forward / backward on a float32 block, and the
// projected momentum / Adam updates that drive it (autograd path).
//
// f_B(x) = -lambda 1^T x - x^T A x (Eq. 7), per column b of
// X (n x B, node-major); grad f_B = -lambda 1 - 2 A x (proof of Thm 3.6).
//
// Power-law graphs have rows of very different length.  Rows of degree up
// to kSplit are accumulated whole by one row group (CSR order); longer rows
// are cut into chunks of kSplit entries whose partial sums go to scratch,
// and a second kernel adds a row's chunk partials in chunk order.  The
// objective is accumulated per lane in float32 over a few rows, then in
// double, then reduced per block and across blocks with double atomics.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

template <int VEC>
struct FbOut {
  __device__ __forceinline__ static void emit(int64_t row, const float* acc, const float* X, int B, int b0,
                                              float lambda_, const float* gout, float* G, bool want_obj,
                                              float* objf) {
    if (G) {
      float o[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float tt = 2.0f * acc[e];
        float gr = -lambda_ - tt;
        if (gout) gr = gout[b0 + e] * gr;
        o[e] = gr;
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) G[row * B + b0 + e] = o[e];
    }
    if (want_obj) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float x = X[row * B + b0 + e];
        const float t1 = lambda_ * x;
        const float t2 = x * acc[e];
        objf[e] = objf[e] - t1;
        objf[e] = objf[e] - t2;
      }
    }
  }
};

struct FbArgs {
  GraphDev g;
  HeavyPlan hp;
  const float* X;
  int B;
  float lambda_;
  const float* gout;
  float* G;
  double* obj;
  float* scratch;
};

template <int VEC>
__device__ __forceinline__ void flush_obj(float* objf, double* objd, int& pending) {
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    objd[e] += (double)objf[e];
    objf[e] = 0.0f;
  }
  pending = 0;
}

template <int VEC>
__global__ void __launch_bounds__(256) k_fb_units(FbArgs a) {
  __shared__ double s_obj[256];
  const int B = a.B;
  const int lpr = B / VEC;
  const int rpw = 32 / lpr;
  const int lane = threadIdx.x & 31;
  const int sub = lane / lpr;
  const int l = lane - sub * lpr;
  const int b0 = l * VEC;
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32 * rpw + sub;
  const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / 32 * rpw;
  const int64_t nunits = (int64_t)a.hp.num_light + a.hp.num_chunks;
  const bool want_obj = a.obj != nullptr;
  for (int i = threadIdx.x; i < B; i += blockDim.x) s_obj[i] = 0.0;
  __syncthreads();
  float objf[VEC];
  double objd[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) { objf[e] = 0.0f; objd[e] = 0.0; }
  int pending = 0;
  for (int64_t u = group; u < nunits; u += ngroups) {
    int64_t row;
    int32_t j0, j1;
    const bool whole = u < a.hp.num_light;
    if (whole) {
      row = a.hp.light_rows[u];
      j0 = a.g.row_ptr[row];
      j1 = a.g.row_ptr[row + 1];
    } else {
      const int64_t c = u - a.hp.num_light;
      row = a.hp.heavy_row[c];
      j0 = a.hp.heavy_j0[c];
      j1 = a.hp.heavy_j1[c];
    }
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0.0f;
    int j = j0;
    for (; j + 4 <= j1; j += 4) {
      const int c0 = __ldcs(a.g.col + j), c1 = __ldcs(a.g.col + j + 1), c2 = __ldcs(a.g.col + j + 2),
                c3 = __ldcs(a.g.col + j + 3);
      const Pack<float, VEC> p0 = ld_pack<float, VEC>(a.X + (int64_t)c0 * B + b0);
      const Pack<float, VEC> p1 = ld_pack<float, VEC>(a.X + (int64_t)c1 * B + b0);
      const Pack<float, VEC> p2 = ld_pack<float, VEC>(a.X + (int64_t)c2 * B + b0);
      const Pack<float, VEC> p3 = ld_pack<float, VEC>(a.X + (int64_t)c3 * B + b0);
      const int8_t w0 = a.g.w ? a.g.w[j] : 1, w1 = a.g.w ? a.g.w[j + 1] : 1, w2 = a.g.w ? a.g.w[j + 2] : 1,
                   w3 = a.g.w ? a.g.w[j + 3] : 1;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        acc[e] = w0 >= 0 ? acc[e] + p0.e[e] : acc[e] - p0.e[e];
        acc[e] = w1 >= 0 ? acc[e] + p1.e[e] : acc[e] - p1.e[e];
        acc[e] = w2 >= 0 ? acc[e] + p2.e[e] : acc[e] - p2.e[e];
        acc[e] = w3 >= 0 ? acc[e] + p3.e[e] : acc[e] - p3.e[e];
      }
    }
    for (; j < j1; ++j) {
      const int c = __ldcs(a.g.col + j);
      const int8_t w = a.g.w ? a.g.w[j] : 1;
      const Pack<float, VEC> p = ld_pack<float, VEC>(a.X + (int64_t)c * B + b0);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = w >= 0 ? acc[e] + p.e[e] : acc[e] - p.e[e];
    }
    if (whole) {
      FbOut<VEC>::emit(row, acc, a.X, B, b0, a.lambda_, a.gout, a.G, want_obj, objf);
      if (++pending == 16) flush_obj<VEC>(objf, objd, pending);
    } else {
      const int64_t c = u - a.hp.num_light;
#pragma unroll
      for (int e = 0; e < VEC; ++e) a.scratch[c * B + b0 + e] = acc[e];
    }
  }
  if (want_obj) {
    flush_obj<VEC>(objf, objd, pending);
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (objd[e] != 0.0) atomicAdd(&s_obj[b0 + e], objd[e]);
    __syncthreads();
    for (int i = threadIdx.x; i < B; i += blockDim.x)
      if (s_obj[i] != 0.0) atomicAdd(&a.obj[i], s_obj[i]);
  }
}

template <int VEC>
__global__ void __launch_bounds__(256) k_fb_heavy(FbArgs a) {
  __shared__ double s_obj[256];
  const int B = a.B;
  const int lpr = B / VEC;
  const int rpw = 32 / lpr;
  const int lane = threadIdx.x & 31;
  const int sub = lane / lpr;
  const int l = lane - sub * lpr;
  const int b0 = l * VEC;
  const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32 * rpw + sub;
  const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / 32 * rpw;
  const bool want_obj = a.obj != nullptr;
  for (int i = threadIdx.x; i < B; i += blockDim.x) s_obj[i] = 0.0;
  __syncthreads();
  float objf[VEC];
  double objd[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) { objf[e] = 0.0f; objd[e] = 0.0; }
  int pending = 0;
  for (int64_t h = group; h < a.hp.num_heavy; h += ngroups) {
    const int64_t row = a.hp.heavy_rows[h];
    const int32_t c0 = a.hp.heavy_first[h], c1 = a.hp.heavy_first[h + 1];
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0.0f;
    for (int32_t c = c0; c < c1; ++c) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = acc[e] + a.scratch[(int64_t)c * B + b0 + e];
    }
    FbOut<VEC>::emit(row, acc, a.X, B, b0, a.lambda_, a.gout, a.G, want_obj, objf);
    if (++pending == 16) flush_obj<VEC>(objf, objd, pending);
  }
  if (want_obj) {
    flush_obj<VEC>(objf, objd, pending);
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (objd[e] != 0.0) atomicAdd(&s_obj[b0 + e], objd[e]);
    __syncthreads();
    for (int i = threadIdx.x; i < B; i += blockDim.x)
      if (s_obj[i] != 0.0) atomicAdd(&a.obj[i], s_obj[i]);
  }
}

// ---------------------------------------------------------------- pipelined rows
// B >= 32: one warp is one row group (lane l owns columns l*VEC ..); batches
// of at most PIPE CSR entries (PIPE * B * 4 bytes = 4 KB) are copied into the
// warp's two shared-memory buffers with cp.async, one batch ahead.
constexpr int kFbPipeBytes = 4096;  // gathered bytes per batch and warp
constexpr int kFbPipeThreads = 256;

// MQO_FB_KERNEL=units selects the plain unit kernel for every batch size
// (read at every launch, so that a test can compare the two)
bool fb_pipe_enabled() {
  const char* e = getenv("MQO_FB_KERNEL");
  return !(e && strcmp(e, "units") == 0);
}

__device__ __forceinline__ void fb_cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}

// ---------------------------------------------------------------- segment stream
// B >= 32, light rows: warp w walks segments w, w + W, ... (consecutive
// light rows, their entries contiguous in CSR) as one stream of batches of
// at most PIPE entries; a batch never spans two segments.  Three positions
// move along the stream: the column indices (and weights) of batch i+2 are
// loaded into lane registers, the neighbour rows of batch i+1 are copied
// into shared memory with cp.async (from indices loaded one batch earlier),
// and batch i is summed.  Row ends come from a window of 32 row pointers
// held across the lanes; every row is summed in CSR order and emitted as in
// k_fb_units (gradient, objective), so the results equal k_fb_units's.
struct FbBatch {
  int64_t seg;  // segment index (>= num_segs: past the end)
  int4 d;       // {first row, end row, first entry, end entry} of the segment
  int32_t jb;   // first entry of the batch
};

template <int VEC, bool WEIGHTED>
__global__ void __launch_bounds__(kFbPipeThreads) k_fb_seg(FbArgs a) {
  extern __shared__ __align__(16) unsigned char smem_fb[];
  __shared__ double s_obj[256];
  constexpr int B = 32 * VEC;
  constexpr int ROWB = B * 4;
  constexpr int PIPE = kFbPipeBytes / ROWB < 32 ? kFbPipeBytes / ROWB : 32;
  constexpr int PER = ROWB / 16;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int b0 = lane * VEC;
  unsigned char* buf = smem_fb + (size_t)warp * 2 * PIPE * ROWB;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nseg = a.hp.num_segs;
  const bool want_obj = a.obj != nullptr;
  for (int i = threadIdx.x; i < B; i += blockDim.x) s_obj[i] = 0.0;
  __syncthreads();
  float objf[VEC];
  double objd[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) { objf[e] = 0.0f; objd[e] = 0.0; }
  int pending = 0;

  auto first = [&](int64_t sg) {
    FbBatch x;
    x.seg = sg;
    x.d = sg < nseg ? a.hp.segs[sg] : make_int4(0, 0, 0, 0);
    x.jb = x.d.z;
    return x;
  };
  auto next = [&](const FbBatch& x) {
    if (x.jb + PIPE < x.d.w) {
      FbBatch y = x;
      y.jb = x.jb + PIPE;
      return y;
    }
    return first(x.seg + W);
  };
  auto count = [&](const FbBatch& x) { return x.seg < nseg ? min(PIPE, x.d.w - x.jb) : 0; };
  // lane e < count: the column index and weight of entry jb + e
  auto load_idx = [&](const FbBatch& x, int32_t& c, int& w) {
    c = 0;
    w = 1;
    if (lane < count(x)) {
      c = __ldcs(a.g.col + x.jb + lane);
      if constexpr (WEIGHTED) w = a.g.w[x.jb + lane];
    }
  };
  // a batch is PIPE * PER = 256 pieces of 16 bytes: in step i lane l copies
  // piece 32i + l (consecutive lanes, consecutive pieces of a row: whole
  // rows per instruction), entry k / PER's piece k % PER, to byte 16k of the
  // buffer; eight steps, unrolled
  static_assert(PIPE * PER == 256, "256 pieces per batch");
  auto issue = [&](const FbBatch& x, int32_t c, int slot) {
    unsigned char* dst = buf + (size_t)slot * PIPE * ROWB + 16 * lane;
    const int cnt = count(x);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = 32 * i + lane;
      const int e = k / PER;
      const int32_t ue = __shfl_sync(0xffffffffu, c, e);
      if (e < cnt)
        fb_cp_async16(dst + 512 * i,
                      reinterpret_cast<const unsigned char*>(a.X + (int64_t)ue * B) + 16 * (k % PER));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // row state of the batch being summed
  int32_t row = 0, rbase = 0, rend_lane = 0, row_end = 0, seg_end_row = 0;
  float acc[VEC];
  float xo[VEC];  // own row of x (objective)
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc[e] = 0.0f, xo[e] = 0.0f;
  auto window = [&](int32_t r) {  // lane i: end entry of row r + i
    rbase = r;
    rend_lane = r + lane < seg_end_row ? a.g.row_ptr[r + lane + 1] : 0x7fffffff;
  };
  auto start_row = [&](int32_t r) {
    row = r;
    if (r - rbase >= 32) window(r);
    row_end = __shfl_sync(0xffffffffu, rend_lane, r - rbase);
    if (want_obj && r < seg_end_row) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) xo[e] = a.X[(int64_t)r * B + b0 + e];
    }
  };
  auto emit = [&]() {
    if (a.G) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float tt = 2.0f * acc[e];
        float gr = -a.lambda_ - tt;
        if (a.gout) gr = a.gout[b0 + e] * gr;
        __stcs(a.G + (int64_t)row * B + b0 + e, gr);
      }
    }
    if (want_obj) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float t1 = a.lambda_ * xo[e];
        const float t2 = xo[e] * acc[e];
        objf[e] = objf[e] - t1;
        objf[e] = objf[e] - t2;
      }
      if (++pending == 16) flush_obj<VEC>(objf, objd, pending);
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0.0f;
  };

  FbBatch cur = first((int64_t)blockIdx.x * (blockDim.x >> 5) + warp);
  FbBatch nx1 = next(cur);
  FbBatch nx2 = next(nx1);
  int32_t c_cur, c1, c2;
  int w_cur, w1, w2;
  load_idx(cur, c_cur, w_cur);
  load_idx(nx1, c1, w1);
  issue(cur, c_cur, 0);
  load_idx(nx2, c2, w2);
  int slot = 0;
  while (cur.seg < nseg) {
    // rows of batch i+1 out (indices loaded one batch ago), indices of
    // batch i+2 in; then wait for batch i
    issue(nx1, c1, slot ^ 1);
    FbBatch nx3 = next(nx2);
    int32_t c3;
    int w3;
    load_idx(nx3, c3, w3);
    if (cur.jb == cur.d.z) {  // the first batch of a segment
      seg_end_row = cur.d.y;
      window(cur.d.x);
      start_row(cur.d.x);
    }
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncwarp();
    const int cnt = count(cur);
    const unsigned char* src = buf + (size_t)slot * PIPE * ROWB + b0 * 4;
    for (int e = 0; e < cnt;) {
      const int32_t j = cur.jb + e;
      while (j >= row_end) {  // rows that end before entry j (empty rows too)
        emit();
        start_row(row + 1);
      }
      // the entries of this row in the batch, without a row-end test each
      const int stop = e + min(cnt - e, row_end - j);
      for (; e < stop; ++e) {
        const int w = WEIGHTED ? __shfl_sync(0xffffffffu, w_cur, e) : 1;
        float f[VEC];
        if constexpr (VEC == 1) {
          f[0] = *reinterpret_cast<const float*>(src + e * ROWB);
        } else if constexpr (VEC == 2) {
          const float2 p = *reinterpret_cast<const float2*>(src + e * ROWB);
          f[0] = p.x;
          f[1] = p.y;
        } else {
  #pragma unroll
          for (int q = 0; q < VEC; q += 4) {
            const float4 p = *reinterpret_cast<const float4*>(src + e * ROWB + q * 4);
            f[q] = p.x;
            f[q + 1] = p.y;
            f[q + 2] = p.z;
            f[q + 3] = p.w;
          }
        }
  #pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = (!WEIGHTED || w >= 0) ? acc[q] + f[q] : acc[q] - f[q];
      }
    }
    __syncwarp();
    if (cur.jb + PIPE >= cur.d.w) {  // the segment's last batch: its remaining rows
      while (row < seg_end_row) {
        emit();
        start_row(row + 1);
      }
    }
    cur = nx1;
    nx1 = nx2;
    nx2 = nx3;
    c1 = c2;
    w_cur = w1;
    w1 = w2;
    c2 = c3;
    w2 = w3;
    slot ^= 1;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (want_obj) {
    flush_obj<VEC>(objf, objd, pending);
#pragma unroll
    for (int e = 0; e < VEC; ++e)
      if (objd[e] != 0.0) atomicAdd(&s_obj[b0 + e], objd[e]);
    __syncthreads();
    for (int i = threadIdx.x; i < B; i += blockDim.x)
      if (s_obj[i] != 0.0) atomicAdd(&a.obj[i], s_obj[i]);
  }
}

template <int VEC>
static cudaError_t launch_fb_vec(const FbArgs& a, int grid, cudaStream_t s) {
  if (a.B == 32 * VEC && fb_pipe_enabled()) {
    // light rows: the segment stream; heavy rows: their 512-entry chunks by
    // the unit kernel, then the chunk sums
    if (a.hp.num_segs > 0) {
      constexpr int ROWB = 32 * VEC * 4;
      constexpr int PIPE = kFbPipeBytes / ROWB < 32 ? kFbPipeBytes / ROWB : 32;
      const size_t smem = (size_t)(kFbPipeThreads / 32) * 2 * PIPE * ROWB;
      auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // one wave: the resident CTAs of every SM (each warp strides over the segments)
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFbPipeThreads, smem);
        if (e != cudaSuccess) return e;
        const int pgrid = std::max(1, std::min(grid, per_sm * (grid / 8)));
        kern<<<pgrid, kFbPipeThreads, smem, s>>>(a);
        return cudaGetLastError();
      };
      const cudaError_t e = a.g.w ? run(k_fb_seg<VEC, true>) : run(k_fb_seg<VEC, false>);
      if (e != cudaSuccess) return e;
    }
    if (a.hp.num_chunks > 0) {
      FbArgs c = a;
      c.hp.num_light = 0;  // units = the chunks of heavy rows only
      k_fb_units<VEC><<<grid, 256, 0, s>>>(c);
    }
  } else if ((int64_t)a.hp.num_light + a.hp.num_chunks > 0) {
    k_fb_units<VEC><<<grid, 256, 0, s>>>(a);
  }
  if (a.hp.num_heavy > 0) k_fb_heavy<VEC><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fb(const GraphDev& g, const HeavyPlan& hp, const float* X, int B, float lambda_,
                      const float* gout, float* G, double* obj, float* scratch, int grid, cudaStream_t stream) {
  FbArgs a{g, hp, X, B, lambda_, gout, G, obj, scratch};
  const int vec = B >= 32 ? B / 32 : 1;
  switch (vec) {
    case 1: return launch_fb_vec<1>(a, grid, stream);
    case 2: return launch_fb_vec<2>(a, grid, stream);
    case 4: return launch_fb_vec<4>(a, grid, stream);
    case 8: return launch_fb_vec<8>(a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- optimisers
__global__ void k_momentum(float* x, float* v, const float* grad, int64_t n, float lr, float mu, float lo, float hi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = mu * v[i];
    const float vn = a + grad[i];
    v[i] = vn;
    const float step = lr * vn;
    x[i] = clamp_box(x[i] + step, lo, hi);
  }
}

__global__ void k_adam(float* x, float* m, float* u, const float* grad, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2, float lo, float hi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mn = b1 * m[i] + (1.0f - b1) * g;
    const float un = b2 * u[i] + (1.0f - b2) * (g * g);
    m[i] = mn;
    u[i] = un;
    const float mh = mn * c1;
    const float uh = un * c2;
    const float step = lr * mh / (sqrtf(uh) + eps);
    x[i] = clamp_box(x[i] + step, lo, hi);
  }
}

cudaError_t launch_momentum(float* x, float* v, const float* grad, int64_t n, float lr, float mu, float lo,
                            float hi, cudaStream_t stream) {
  const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  if (n > 0) k_momentum<<<grid, 256, 0, stream>>>(x, v, grad, n, lr, mu, lo, hi);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* x, float* m, float* u, const float* grad, int64_t n, float lr, float b1, float b2,
                        float eps, int64_t t, float lo, float hi, cudaStream_t stream) {
  const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  const float c1 = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
  const float c2 = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
  if (n > 0) k_adam<<<grid, 256, 0, stream>>>(x, m, u, grad, n, lr, b1, b2, eps, c1, c2, lo, hi);
  return cudaGetLastError();
}

}  // namespace mqo
