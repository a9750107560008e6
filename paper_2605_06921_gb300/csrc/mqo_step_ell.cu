// mqo_step_ell.cu -- the shared-memory step kernel (mqo_step_smem.cuh) with
// the sliced-ELL neighbour stream, for 2-byte x: unweighted MaxCut, and MIS
// with bfloat16 x (whose checker needs no rounding words).  Its own
// translation unit so that it compiles beside the CSR instances.
#include "mqo_step_smem.cuh"

namespace mqo {

cudaError_t launch_smem_ell(const StepArgs& a, bool wide, size_t smem, bool mis, const int4* ell, const int2* ell_pos,
                            int grid, int x_dtype, int v_dtype, cudaStream_t s) {
  if (!mis && a.g.w != nullptr) return cudaErrorInvalidValue;  // the stream carries no weights
  if (x_dtype == DT_BF16 && v_dtype == DT_BF16)
    return launch_smem<__nv_bfloat16, __nv_bfloat16, true>(a.B, wide, smem, mis, a, ell, ell_pos, grid, s);
  if (x_dtype == DT_BF16 && v_dtype == DT_F32)
    return launch_smem<__nv_bfloat16, float, true>(a.B, wide, smem, mis, a, ell, ell_pos, grid, s);
  if (!mis && x_dtype == DT_F16 && v_dtype == DT_F16)
    return launch_smem<__half, __half, true>(a.B, wide, smem, mis, a, ell, ell_pos, grid, s);
  if (!mis && x_dtype == DT_F16 && v_dtype == DT_F32)
    return launch_smem<__half, float, true>(a.B, wide, smem, mis, a, ell, ell_pos, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace mqo

namespace mqo {

// One CTA per item: the item's rows in groups of rpw positions of the
// processing order; group q's vectors start at pos[first position].x and
// number pos[..].y per row (4 entries each); entries past a row's end, and
// whole rows past the item's end, hold the dummy neighbour (local id ng).
__global__ void k_ell_fill(GraphDev g, int rpw, int pitch, const int2* __restrict__ pos, int4* __restrict__ ell) {
  const Item item = g.items[blockIdx.x];
  const int nrows = item.v1 - item.v0;
  const int32_t off = g.node_off[item.g];
  const int dummy = (g.node_off[item.g + 1] - off) * pitch;
  const int ngrp = (nrows + rpw - 1) / rpw;
  for (int i = threadIdx.x; i < ngrp * rpw; i += blockDim.x) {
    const int q = i / rpw, r = i - q * rpw;
    const int2 ep = pos[item.v0 + q * rpw];
    int rs = 0, re = 0;
    if (i < nrows) {
      const int v = g.order[item.v0 + i];
      rs = g.row_ptr[v];
      re = g.row_ptr[v + 1];
    }
    for (int c = 0; c < ep.y; ++c) {
      int e[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = rs + 4 * c + k;
        e[k] = j < re ? (g.col[j] - off) * pitch : dummy;
      }
      ell[(int64_t)ep.x + (int64_t)c * rpw + r] = make_int4(e[0], e[1], e[2], e[3]);
    }
  }
}

cudaError_t launch_ell_fill(const GraphDev& g, int rpw, int pitch, const int2* pos, int4* ell, cudaStream_t s) {
  if (g.num_items <= 0) return cudaSuccess;
  k_ell_fill<<<g.num_items, 256, 0, s>>>(g, rpw, pitch, pos, ell);
  return cudaGetLastError();
}

}  // namespace mqo
