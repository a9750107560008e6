// mqo_static.cu -- gradient of f_B with no allocation: scratch lives in a
// fixed-size static device array owned by the library.
//
// For callers that cannot allocate device memory during the call:
// applications whose device memory is held entirely by their own pool or
// allocator (e.g. a framework's caching allocator that has reserved the
// device), and loops that must not pay for cudaMalloc / cudaFree, which can
// synchronise the device.  The regular mqo_spmm_grad keeps a per-graph
// scratch buffer and its chunk plan, both allocated on first use.
//
// This variant computes the same gradient G = gout * (-lambda - 2 A X):
//   pass 1: every row of degree <= kSplitS is accumulated whole (CSR order)
//           and written; every longer row reserves ceil(d/kSplitS) partial
//           slots in the static array with two atomic counters;
//   pass 2: each reserved chunk of kSplitS entries is summed into its slot;
//   pass 3: each long row adds its partials in chunk order and writes G.
// Slot numbers depend on scheduling, but every row's partials are added in
// chunk order, so the result is the same on every call.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mqo.h"
#include "mqo_host.h"

namespace mqo {
namespace {

constexpr int kSplitS = 512;                   // entries per chunk of a long row
constexpr size_t kStaticWords = (size_t)1 << 20;  // 4 MiB of scratch (1M 32-bit words)
constexpr size_t kHeader = 64;                 // words: two counters, padded
constexpr int kMaxDevices = 64;

// The scratch: [0] long-row counter, [1] chunk-slot counter, then for each
// long row a (row, first slot) pair, then the float partials.  Every GPU
// that loads the library holds these 4 MiB until the process exits.
__device__ __align__(256) uint32_t g_fb_static[kStaticWords];

std::mutex g_mu;
uint32_t* g_ptr[kMaxDevices];  // device address of g_fb_static per device

struct StaticArgs {
  const int32_t* rp;
  const int32_t* col;
  const int8_t* w;
  int32_t n;
  const float* X;
  int B;
  float lambda_;
  const float* gout;
  float* G;
  uint32_t* scratch;
  int32_t max_rows;    // capacity of the (row, first slot) list
  int64_t max_floats;  // capacity of the partials
};

__device__ __forceinline__ void emit_row(const StaticArgs& a, int64_t row, int b, float acc) {
  const float tt = 2.0f * acc;
  float gr = -a.lambda_ - tt;
  if (a.gout) gr = a.gout[b] * gr;
  a.G[row * a.B + b] = gr;
}

// one thread per (row, trajectory); the B threads of a row sum in CSR order
__global__ void k_static_pass1(StaticArgs a) {
  const int64_t total = (int64_t)a.n * a.B;
  uint32_t* cnt = a.scratch;
  int32_t* list = reinterpret_cast<int32_t*>(a.scratch + kHeader);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / a.B;
    const int b = (int)(i % a.B);
    const int32_t j0 = a.rp[row], j1 = a.rp[row + 1];
    if (j1 - j0 > kSplitS) {
      if (b == 0) {
        const uint32_t chunks = (uint32_t)((j1 - j0 + kSplitS - 1) / kSplitS);
        const uint32_t k = atomicAdd(&cnt[0], 1u);
        const uint32_t first = atomicAdd(&cnt[1], chunks);
        if ((int64_t)k < a.max_rows) {
          list[2 * k] = (int32_t)row;
          list[2 * k + 1] = (int32_t)first;
        }
      }
      continue;
    }
    float acc = 0.0f;
    for (int32_t j = j0; j < j1; ++j) {
      const float xu = a.X[(int64_t)a.col[j] * a.B + b];
      acc = (a.w == nullptr || a.w[j] >= 0) ? acc + xu : acc - xu;
    }
    emit_row(a, row, b, acc);
  }
}

// one block per listed long row; thread (chunk, trajectory)
__global__ void k_static_pass2(StaticArgs a) {
  const uint32_t* cnt = a.scratch;
  const int32_t* list = reinterpret_cast<const int32_t*>(a.scratch + kHeader);
  float* part = reinterpret_cast<float*>(a.scratch + kHeader + 2 * (size_t)a.max_rows);
  const uint32_t rows = min(cnt[0], (uint32_t)a.max_rows);
  for (uint32_t k = blockIdx.x; k < rows; k += gridDim.x) {
    const int32_t row = list[2 * k], first = list[2 * k + 1];
    const int32_t j0 = a.rp[row], j1 = a.rp[row + 1];
    const int32_t chunks = (j1 - j0 + kSplitS - 1) / kSplitS;
    for (int32_t i = threadIdx.x; i < chunks * a.B; i += blockDim.x) {
      const int32_t c = i / a.B;
      const int b = i % a.B;
      const int32_t s0 = j0 + c * kSplitS, s1 = min(j1, s0 + kSplitS);
      float acc = 0.0f;
      for (int32_t j = s0; j < s1; ++j) {
        const float xu = a.X[(int64_t)a.col[j] * a.B + b];
        acc = (a.w == nullptr || a.w[j] >= 0) ? acc + xu : acc - xu;
      }
      part[((int64_t)first + c) * a.B + b] = acc;
    }
  }
}

__global__ void k_static_pass3(StaticArgs a) {
  const uint32_t* cnt = a.scratch;
  const int32_t* list = reinterpret_cast<const int32_t*>(a.scratch + kHeader);
  const float* part = reinterpret_cast<const float*>(a.scratch + kHeader + 2 * (size_t)a.max_rows);
  const uint32_t rows = min(cnt[0], (uint32_t)a.max_rows);
  for (uint32_t k = blockIdx.x; k < rows; k += gridDim.x) {
    const int32_t row = list[2 * k], first = list[2 * k + 1];
    const int32_t chunks = (a.rp[row + 1] - a.rp[row] + kSplitS - 1) / kSplitS;
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
      float acc = 0.0f;
      for (int32_t c = 0; c < chunks; ++c) acc = acc + part[((int64_t)first + c) * a.B + b];
      emit_row(a, row, b, acc);
    }
  }
}

}  // namespace
}  // namespace mqo

using namespace mqo;

extern "C" mqo_status mqo_spmm_grad_static(mqo_graph g, const float* X, const float* gout, float* G, int32_t B,
                                           float lambda_, void* cuda_stream) {
  if (!g || !X || !G) return set_last_error(MQO_EINVAL, "mqo_spmm_grad_static: null argument");
  if (B < 1 || B > 256 || (B & (B - 1)))
    return set_last_error(MQO_EINVAL, "mqo_spmm_grad_static: B must be a power of two in [1,256]");
  GraphCsrView csr;
  graph_csr_view(g, &csr);
  // capacity: two counters, one (row, slot) pair per long row, B floats per chunk
  const size_t need = kHeader + 2 * (size_t)csr.long_rows + (size_t)csr.long_chunks * (size_t)B;
  if (need > kStaticWords) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "mqo_spmm_grad_static: graph needs %zu scratch words (%d long rows, %lld chunks x B=%d), "
             "the static scratch holds %zu",
             need, csr.long_rows, (long long)csr.long_chunks, B, kStaticWords);
    return set_last_error(MQO_EINVAL, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(MQO_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(MQO_EINVAL, "mqo_spmm_grad_static: device id too large");
  uint32_t* scratch = nullptr;
  {
    // first call on this device: look up the device address of the array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_fb_static);
      if (e != cudaSuccess) return set_last_error(MQO_ECUDA, cudaGetErrorString(e));
      g_ptr[dev] = static_cast<uint32_t*>(p);
    }
    scratch = g_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the two counters must start at zero; everything else is written before it is read
  e = cudaMemsetAsync(scratch, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return set_last_error(MQO_ECUDA, cudaGetErrorString(e));
  StaticArgs a{csr.row_ptr, csr.col, csr.w, csr.n, X, B, lambda_, gout, G, scratch, csr.long_rows,
               (int64_t)csr.long_chunks * B};
  const int64_t total = (int64_t)csr.n * B;
  const int grid1 = (int)std::min<int64_t>((total + 255) / 256, (int64_t)csr.sms * 32);
  k_static_pass1<<<grid1, 256, 0, s>>>(a);
  if (csr.long_rows > 0) {
    const int grid2 = std::min(csr.long_rows, csr.sms * 8);
    k_static_pass2<<<grid2, 256, 0, s>>>(a);
    k_static_pass3<<<grid2, 256, 0, s>>>(a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(MQO_ECUDA, cudaGetErrorString(e));
  return MQO_OK;
}
