// mqo_validate.cu -- the entry checks of a symmetric CSR graph on the device,
// one warp per row: every column index in range and not the row itself,
// rows strictly ascending, weights in {-1,+1}, no edge joining two member
// graphs, and for every entry (v,u) a reverse entry (u,v) with the same
// weight (a binary search in row u).  The smallest bad row is reported; the
// host words the error from that row.
#include "mqo_dev.cuh"
#include "mqo_host.h"

namespace mqo {

__device__ __forceinline__ int32_t member_of(const int32_t* node_off, int32_t G, int32_t v) {
  int32_t lo = 0, hi = G;  // largest g with node_off[g] <= v
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (node_off[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_validate_csr(const int32_t* rp, const int32_t* col, const int8_t* w,
                                                      const int32_t* node_off, int32_t G, int32_t n,
                                                      int32_t* bad_row) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int32_t rs = rp[v], re = rp[v + 1];
    const int32_t gv = G > 1 ? member_of(node_off, G, (int32_t)v) : 0;
    bool bad = false;
    for (int32_t j = rs + lane; j < re; j += 32) {
      const int32_t u = col[j];
      if (u < 0 || u >= n || u == (int32_t)v) { bad = true; continue; }
      if (j > rs && col[j - 1] >= u) { bad = true; continue; }
      if (w && w[j] != 1 && w[j] != -1) { bad = true; continue; }
      if (G > 1 && member_of(node_off, G, u) != gv) { bad = true; continue; }
      int32_t lo = rp[u], hi = rp[u + 1];  // reverse entry (u, v)
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (col[mid] < (int32_t)v) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= rp[u + 1] || col[lo] != (int32_t)v || (w && w[lo] != w[j])) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMin(bad_row, (int32_t)v);
  }
}

// 16-bit member-local column indices: one CTA per work item (a node range
// of one member graph), entry j of a row of member graph g gets
// col[j] - node_off[g]
__global__ void __launch_bounds__(256) k_col16(const int32_t* rp, const int32_t* col, const int32_t* node_off,
                                               const Item* items, uint16_t* col16) {
  const Item it = items[blockIdx.x];
  const int32_t off = node_off[it.g];
  for (int32_t j = rp[it.v0] + threadIdx.x; j < rp[it.v1]; j += blockDim.x) col16[j] = (uint16_t)(col[j] - off);
}

cudaError_t launch_col16(const GraphDev& g, uint16_t* col16, cudaStream_t stream) {
  if (g.num_items > 0) k_col16<<<g.num_items, 256, 0, stream>>>(g.row_ptr, g.col, g.node_off, g.items, col16);
  return cudaGetLastError();
}

cudaError_t launch_validate_csr(const int32_t* rp, const int32_t* col, const int8_t* w, const int32_t* node_off,
                                int32_t G, int32_t n, int32_t* bad_row, int sms, cudaStream_t stream) {
  const int64_t want = ((int64_t)n * 32 + 255) / 256;
  const int grid = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  k_validate_csr<<<grid > 0 ? grid : 1, 256, 0, stream>>>(rp, col, w, node_off, G, n, bad_row);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e;
}

}  // namespace mqo
