// mqo_probe.cu -- measured shared-memory load bandwidth of the device: the
// denominator of the shared-memory step kernel's roofline (mqo_measure_smem_gbs
// in mqo_api.cu times it).
//
// Every SM runs two CTAs of 1024 threads (64 KB of shared memory each);
// after filling its buffer a CTA streams 16-byte loads in which each warp
// reads 512 consecutive bytes (four conflict-free wavefronts of 128 bytes),
// four loads per iteration at fixed 16 KB offsets, folding them into a
// register by XOR so that no load can be removed.  Bytes per launch =
// CTAs x 1024 threads x 4 x iters x 16; one untimed launch, then one timed
// with CUDA events.  No thread waits on another beyond the block barrier
// after the fill, and every loop has a fixed trip count.
#include <cuda_runtime.h>

#include <cstdint>

#include "mqo_host.h"

namespace mqo {

constexpr int kProbeThreads = 1024;
constexpr int kProbeWords = 4096;  // uint4 words: 64 KB

__global__ void __launch_bounds__(kProbeThreads, 2) k_smem_probe(int32_t iters, uint32_t* sink) {
  extern __shared__ uint4 buf[];  // kProbeWords words of dynamic shared memory
  for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x)
    buf[i] = make_uint4((uint32_t)i, (uint32_t)i * 3u, (uint32_t)i * 5u, (uint32_t)i * 7u);
  __syncthreads();
  const uint4* p = buf + threadIdx.x;  // threadIdx.x < 1024 = kProbeWords / 4
  uint32_t a = 0u, b = 0u, c = 0u, d = 0u;
  for (int32_t k = 0; k < iters; ++k) {
    const uint4 v0 = p[0], v1 = p[1024], v2 = p[2048], v3 = p[3072];
    a ^= v0.x ^ v1.y ^ v2.z ^ v3.w;
    b ^= v0.y ^ v1.z ^ v2.w ^ v3.x;
    c ^= v0.z ^ v1.w ^ v2.x ^ v3.y;
    d ^= v0.w ^ v1.x ^ v2.y ^ v3.z;
    // a different (still conflict-free) pairing each iteration, so the
    // loads are not loop invariant
    p = buf + ((threadIdx.x + 32u * (uint32_t)(k + 1)) & 1023u);
  }
  const uint32_t r = a ^ b ^ c ^ d;
  if (r == 0x9e3779b9u) sink[blockIdx.x] = r;  // practically never: keeps r alive
}

cudaError_t launch_smem_probe(int grid, int32_t iters, uint32_t* sink, cudaStream_t s) {
  const int bytes = kProbeWords * (int)sizeof(uint4);  // above the 48 KB default: opt in
  cudaError_t e = cudaFuncSetAttribute(k_smem_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_smem_probe<<<grid, kProbeThreads, bytes, s>>>(iters, sink);
  return cudaGetLastError();
}

int smem_probe_threads() { return kProbeThreads; }

}  // namespace mqo
