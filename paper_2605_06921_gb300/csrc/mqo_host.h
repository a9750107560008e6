// mqo_host.h -- launchers shared by the host runtime of the mQO library.
#pragma once

#include <cuda_runtime.h>

#include "../../include/mqo.h"
#include "mqo_dev.cuh"

namespace mqo {

constexpr int kPairThreads = 256;  // pair kernels: (node, trajectory) per thread

enum CtrlMode : int { CTRL_MACHINE = 0, CTRL_LS_BEGIN = 1, CTRL_LS = 2, CTRL_RESET = 3 };

// smem > 0: the shared-memory kernel with that much dynamic shared memory,
// with the sliced-ELL neighbour stream when `ell` is given (build_ell)
cudaError_t launch_step(const SolverDev& S, Counters* cnt, const int32_t* act, const int32_t* gflag_step,
                        size_t smem, cudaStream_t stream, const int4* ell = nullptr, const int2* ell_pos = nullptr);
// the sliced-ELL stream of the shared-memory step kernel (mqo_step_smem.cuh)
// for `rpw` rows per warp and x rows `pitch` bytes apart, from the group
// table `pos` (one entry per processing position)
cudaError_t launch_ell_fill(const GraphDev& g, int rpw, int pitch, const int2* pos, int4* ell, cudaStream_t s);
bool step_wide_possible(int B, int x_dtype);
int default_step_vec(int B, int x_dtype);
bool staged_vec_ok(int B, int x_dtype, int vec);
int default_staged_vec(int B, int x_dtype);
size_t step_smem_bytes(int B, int x_dtype, int problem, int max_ng);

cudaError_t launch_ctrl(const SolverDev& S, int mode, const uint8_t* mask, cudaStream_t stream);
cudaError_t launch_apply(const SolverDev& S, cudaStream_t stream);
cudaError_t launch_disc(const SolverDev& S, int pass, cudaStream_t stream);
size_t disc_graph_smem_bytes(int B, int max_ng);
cudaError_t launch_disc_graph(const SolverDev& S, size_t smem, cudaStream_t stream);
cudaError_t launch_tick_end(const SolverDev& S, cudaStream_t stream);
cudaError_t launch_round_bits(const SolverDev& S, uint32_t* z, cudaStream_t stream);
cudaError_t launch_eval(const SolverDev& S, const uint32_t* z, Counters* out, cudaStream_t stream);
cudaError_t launch_counters_out(const SolverDev& S, const Counters* c, int64_t* value, int64_t* a, int64_t* b,
                                int kind, cudaStream_t stream);
cudaError_t launch_objective(const SolverDev& S, double* out, cudaStream_t stream);
cudaError_t launch_ls_merge(const SolverDev& S, const TrajState* saved, cudaStream_t stream);
cudaError_t launch_state_init(const SolverDev& S, cudaStream_t stream);
cudaError_t launch_any_pending(const SolverDev& S, int32_t* out, cudaStream_t stream);
// device check of the CSR entries (range, no self loop, strictly ascending
// rows, weights in {-1,+1}, no edge between member graphs, a reverse entry
// with the same weight): *bad_row <- the smallest row with a bad entry
// (unchanged if none); synchronous
cudaError_t launch_validate_csr(const int32_t* rp, const int32_t* col, const int8_t* w, const int32_t* node_off,
                                int32_t G, int32_t n, int32_t* bad_row, int sms, cudaStream_t stream);
cudaError_t launch_pool_ctrl(const SolverDev& S, cudaStream_t stream);
// 16-bit member-local copies of the column indices (every member graph below 65536 nodes)
cudaError_t launch_col16(const GraphDev& g, uint16_t* col16, cudaStream_t stream);
cudaError_t launch_pool_apply(const SolverDev& S, cudaStream_t stream);

// graph-level kernels (autograd path)
struct HeavyPlan {
  const int32_t* light_rows;  // rows handled whole
  int32_t num_light;
  const int32_t* heavy_row;   // per chunk: row
  const int32_t* heavy_j0;    // per chunk: first entry
  const int32_t* heavy_j1;    // per chunk: end entry
  int32_t num_chunks;
  const int32_t* heavy_rows;  // distinct heavy rows
  const int32_t* heavy_first; // per heavy row: first chunk
  int32_t num_heavy;
  // light rows in segments of consecutive rows (no heavy row inside) of
  // about kFbSegEntries entries: {first row, end row, first entry, end entry}
  const int4* segs;
  int32_t num_segs;
};
constexpr int kFbSegEntries = 512;

// the shared-memory bandwidth probe (mqo_probe.cu): `grid` CTAs of
// smem_probe_threads() threads, `iters` iterations of four 16-byte loads each
cudaError_t launch_smem_probe(int grid, int32_t iters, uint32_t* sink, cudaStream_t s);
int smem_probe_threads();

cudaError_t launch_fb(const GraphDev& g, const HeavyPlan& hp, const float* X, int B, float lambda_,
                      const float* gout, float* G, double* obj, float* scratch, int grid, cudaStream_t stream);
cudaError_t launch_momentum(float* x, float* v, const float* grad, int64_t n, float lr, float mu, float lo,
                            float hi, cudaStream_t stream);
cudaError_t launch_adam(float* x, float* m, float* u, const float* grad, int64_t n, float lr, float b1, float b2,
                        float eps, int64_t t, float lo, float hi, cudaStream_t stream);

// read-only view of a graph's device CSR and its long-row statistics
// (rows longer than 512 entries, and their 512-entry chunks)
struct GraphCsrView {
  const int32_t* row_ptr;
  const int32_t* col;
  const int8_t* w;
  int32_t n;
  int32_t long_rows;
  int64_t long_chunks;
  int32_t sms;  // multiprocessors of the device the graph was created on
};

}  // namespace mqo

struct mqo_graph_s;
void graph_csr_view(mqo_graph_s* g, mqo::GraphCsrView* out);
mqo_status set_last_error(mqo_status status, const char* msg);
