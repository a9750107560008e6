// mqo_step.cu -- the dispatch of a tick's step to the shared-memory kernel
// (mqo_step_smem.cuh; here with column indices from the CSR arrays, in
// mqo_step_ell.cu with the sliced-ELL stream), the staged-gather kernel
// (mqo_step_staged.cu) or the global-memory kernel (mqo_step_generic.cu).
// The step itself (gradient, momentum, projection, rounding, exact
// evaluation) is described in mqo_step.cuh.
#include "mqo_step_smem.cuh"

namespace mqo {

// the shared-memory kernel with the sliced-ELL stream (mqo_step_ell.cu)
cudaError_t launch_smem_ell(const StepArgs& a, bool wide, size_t smem, bool mis, const int4* ell, const int2* ell_pos,
                            int grid, int x_dtype, int v_dtype, cudaStream_t s);

size_t step_smem_bytes(int B, int x_dtype, int problem, int max_ng) {
  const size_t sx = x_dtype == DT_F32 ? 4 : 2;
  const size_t rowb = (size_t)B * sx;
  const size_t pitch = rowb == 64 ? 128 : rowb;
  const size_t xb = ((size_t)(max_ng + 1) * pitch + 15) & ~(size_t)15;
  const size_t zb = problem == PROB_MIS ? (((size_t)(max_ng + 1) * ((B + 31) / 32) * 4 + 15) & ~(size_t)15) : 0;
  return xb + zb + ((3 * (size_t)B * 8 + 15) & ~(size_t)15) + (size_t)kItemMaxNodes * 16;
}

bool step_wide_possible(int B, int x_dtype) { return x_dtype != DT_F32 ? (B == 32 || B == 64 || B == 128) : (B == 32 || B == 64); }

template <typename TX, typename TV>
static cudaError_t launch_tv(bool wide, size_t smem, bool mis, const StepArgs& a, int grid, cudaStream_t s) {
  return launch_smem<TX, TV, false>(a.B, wide, smem, mis, a, nullptr, nullptr, grid, s);
}

cudaError_t launch_step(const SolverDev& S, Counters* cnt, const int32_t* act, const int32_t* gflag_step,
                        size_t smem, cudaStream_t stream, const int4* ell, const int2* ell_pos) {
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
  a.slices = S.slices;
  if (!S.step_c16) a.g.col16 = nullptr;
  a.num_slices = S.num_slices;
  a.slice_rows = S.slice_rows;
  a.slice_cols = S.slice_cols;
  const int xd = S.p.x_dtype, vd = S.p.v_dtype;
  if (smem == 0 && S.step_staged) {
    // staged-gather kernel: one CTA per slice
    const int vec = S.step_vec > 0 ? S.step_vec : default_staged_vec(S.B, xd);
    const int sx = xd == DT_F32 ? 4 : 2, sv = vd == DT_F32 ? 4 : 2;
    const size_t qs = staged_layout(S.B, sx, sv, S.slice_cols, S.slice_rows,
                                    S.g.w != nullptr && S.p.problem != PROB_MIS)
                          .total;
    return launch_step_staged(a, vec, xd, vd, qs, stream);
  }
  if (smem == 0) {
    // global-memory kernel; few items (a handful of member graphs): several CTAs per item
    const int vec = S.step_vec > 0 ? S.step_vec : default_step_vec(S.B, xd);
    a.split = S.split;
    return launch_step_generic(a, vec, xd, vd, S.g.num_items * a.split, stream);
  }
  const bool wide = S.step_wide != 0;
  const bool mis = S.p.problem == PROB_MIS;
  const int grid = S.g.num_items;
  if (ell) return launch_smem_ell(a, wide, smem, mis, ell, ell_pos, grid, xd, vd, stream);
  if (xd == DT_F32) return launch_tv<float, float>(wide, smem, mis, a, grid, stream);
  if (xd == DT_BF16 && vd == DT_BF16) return launch_tv<__nv_bfloat16, __nv_bfloat16>(wide, smem, mis, a, grid, stream);
  if (xd == DT_BF16 && vd == DT_F32) return launch_tv<__nv_bfloat16, float>(wide, smem, mis, a, grid, stream);
  if (xd == DT_F16 && vd == DT_F16) return launch_tv<__half, __half>(wide, smem, mis, a, grid, stream);
  if (xd == DT_F16 && vd == DT_F32) return launch_tv<__half, float>(wide, smem, mis, a, grid, stream);
  return cudaErrorInvalidValue;
}

}  // namespace mqo
