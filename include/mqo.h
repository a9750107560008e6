/*
 * mqo.h -- C ABI of the GB300 (sm_103a) implementation of the mQO hot path.
 *
 * Method: "Mutation-Guided Differentiable Quadratic Combinatorial
 * Optimization" (mQO).  The library runs batched projected momentum
 * gradient ascent on the box-relaxed MIS objective
 *     h(x)   = 1^T x - (gamma/2) x^T A x,   x in [0,1]^n   (Eq. 3)
 * and the perturbed-bias MaxCut objective
 *     f_B(x) = -lambda 1^T x - x^T A x,     x in [-1,1]^n  (Eq. 7)
 * fused with threshold rounding and exact integer evaluation, inside the
 * per-trajectory mutation/reset/local-search machine of Alg. 1 (MIS) and
 * Alg. 2 (MaxCut), B independent trajectories per graph (pmQO, Alg. 3/4).
 *
 * Conventions for every entry point:
 *  - Status: every call returns an mqo_status; no C++ exception crosses
 *    the ABI.  mqo_last_error() returns a thread-local message for the last
 *    failure on the calling thread.  After MQO_ECUDA the solver is poisoned
 *    and later calls on it return MQO_ESTATE.
 *  - Streams: `cuda_stream` is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream).  Work is enqueued asynchronously unless the
 *    call says it synchronises.
 *  - Ownership: the library deep-copies graphs into device memory it owns.
 *    Every pointer the caller passes stays owned by the caller; device
 *    output arrays are caller-allocated and never freed by the library.
 *  - Layouts: node-major.  A relaxed block X holds n x B values, row v
 *    (node) contiguous over its B trajectories: X[v*B + b].  Binary vectors
 *    of a solver are bit-packed node-major: with Bw = ceil(B/32) words per
 *    node, trajectory b of node v is bit (b % 32) of word v*Bw + b/32.
 *  - Trajectory ids: for a graph packed from G member graphs, trajectory
 *    t = g*B + b (member graph g, batch slot b); random draws are keyed by
 *    (seed, t) and local node ids, so a trajectory's result does not depend
 *    on which other graphs share the batch.
 */
#ifndef MQO_H
#define MQO_H

#include <stdint.h>

#if defined(__GNUC__)
#define MQO_API __attribute__((visibility("default")))
#else
#define MQO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mqo_graph_s* mqo_graph;
typedef struct mqo_solver_s* mqo_solver;

typedef enum {
  MQO_OK = 0,
  MQO_EINVAL = -1,  /* bad argument (null pointer, size, unsupported option) */
  MQO_EGRAPH = -2,  /* CSR failed validation (see mqo_last_error) */
  MQO_ENOMEM = -3,  /* device or host allocation failed */
  MQO_ECUDA = -4,   /* a CUDA call failed; the solver is poisoned */
  MQO_ETIMEOUT = -5,/* reserved: no entry point waits on the device */
  MQO_ESTATE = -6   /* solver poisoned by an earlier failure */
} mqo_status;

typedef enum { MQO_MIS = 0, MQO_MAXCUT = 1 } mqo_problem;
/* MaxCut relaxation descended by the solver (Sec. 3):
 *   MQO_OBJ_FB  f_B(x) = -lambda 1'x - x'Ax        (Eq. 7; the default)
 *   MQO_OBJ_FL  f_L(x) = 1/4 x'Lx, L = D - A       (Eq. 4)
 *   MQO_OBJ_FP  f_P(x) = x'(L + lambda I)x         (perturbed Laplacian)
 *   MQO_OBJ_FA  f_A(x) = -x'Ax                     (adjacency form)
 * Each equals an affine function of the cut on {-1,1}^n; they differ in
 * which binary points are PGA fixed points (Thm 3.3, Prop. 3.4, Thm 3.6). */
typedef enum { MQO_OBJ_FB = 0, MQO_OBJ_FL = 1, MQO_OBJ_FP = 2, MQO_OBJ_FA = 3 } mqo_objective;
typedef enum { MQO_F32 = 0, MQO_BF16 = 1, MQO_F16 = 2 } mqo_dtype;

/* Trajectory phases reported by mqo_traj_state. */
/* MQO_PH_WAIT (pool mode only): the trajectory holds a finished set until
 * every trajectory of its member graph has one (Alg. 3/4 steps 3-4). */
typedef enum { MQO_PH_DESCENT = 0, MQO_PH_REPAIR = 1, MQO_PH_LS = 2, MQO_PH_WAIT = 3 } mqo_phase;

/*
 * Solver parameters.  Paper symbols: alpha (step size), momentum (MGA,
 * Sec. 5 and App. F), gamma > 1 (edge penalty of h, Eq. 3),
 * lambda in (0,2) (bias of f_B, Thm 3.6; 0.001 in Sec. 5), rho in (0,1)
 * (reset fraction, |R| = floor(rho n), Sec. 4), t_gs (global-reset rounds
 * per outer iteration, Alg. 1 step 5), sigma (init noise std, Alg. 1
 * step 2).
 */
typedef struct {
  int32_t problem;      /* mqo_problem */
  int32_t batch;        /* B trajectories per graph: a power of two in [1, 128] */
  int32_t x_dtype;      /* storage of X: mqo_dtype (arithmetic is FP32) */
  int32_t v_dtype;      /* storage of the momentum V: MQO_F32 or x_dtype */
  float alpha;
  float momentum;
  float gamma;          /* MIS only */
  float lambda_;        /* MaxCut only */
  double rho;           /* |R| = floor(rho * n_g), evaluated in double */
  float sigma;          /* init_kind 1 noise std */
  int32_t t_gs;         /* >= 0 */
  int32_t descent_cap;  /* >= 1: descent steps before a descent is cut off */
  int32_t init_kind;    /* 0: x ~ U(box); 1: degree-based centre + noise (Alg. 1/2 step 2) */
  int32_t local_search; /* 1: OneTwoSwap / OneTwoFlip after t_gs rounds (Alg. 1/2 step 11) */
  int32_t repair;       /* MIS: 1 = repair a capped descent into a maximal IS, 0 = discard it */
  uint64_t seed;
  int32_t objective;    /* MaxCut only: mqo_objective (gradient of the step and its fixed-point test) */
  int32_t pool_k;       /* 0: B independent trajectories per graph (Alg. 1/2); K in [1,64]: the B
                           trajectories of a graph share a pool of the K best sets (pmQO, Alg. 3/4) */
} mqo_params;

/* Per-trajectory machine state (host copy), see mqo_traj_state. */
typedef struct {
  int32_t phase;        /* mqo_phase */
  int32_t s;            /* descent steps taken in the current descent */
  int32_t r;            /* reset rounds started in the current outer iteration */
  int32_t o;            /* outer iteration (fresh initialisations so far) */
  int64_t best;         /* best exact value accepted so far, INT64_MIN if none */
  int64_t ticks;        /* machine ticks run */
  int32_t last_round;   /* discrete round type of the last tick (-1: a descent step) */
  int32_t pad0;
  int64_t last_commits; /* moves applied by that round */
  int64_t ev_value;     /* last exact evaluation: MIS size | cut value */
  int64_t ev_a;         /* MIS conflicting nodes | MaxCut nodes not f_B-fixed */
  int64_t ev_b;         /* MIS uncovered nodes | MaxCut nodes with a positive 1-flip gain */
  int64_t accepts;      /* strict improvements of best */
  int64_t descents;     /* finished descents */
  int64_t held;         /* pool mode: value of the set held while waiting, INT64_MIN if none
                           (or a capped, unrepaired MIS point, which is no candidate) */
  /* gains breakdown (the paper's appendix on where mQO's gains come from):
   * best = first_value + gain_descent + gain_ls once a set was accepted */
  int64_t first_value;  /* first accepted value (end of the first descent), INT64_MIN if none */
  int64_t gain_descent; /* sum of the strict improvements accepted from later descents
                           (global-reset rounds and restarts; pool merges in pool mode) */
  int64_t gain_ls;      /* sum of the strict improvements accepted from local search */
  int64_t steps;        /* descent steps taken in all (ticks that ran a gradient step) */
} mqo_traj_info;

/* ---------------------------------------------------------------- graphs */

/*
 * Create a graph from symmetric CSR (Sec. 2 notation: A, N(v), d(v)).
 * n nodes (1 <= n < 2^31), nnz directed entries (nnz < 2^31); row_ptr[n+1]
 * int64 (row_ptr[0] = 0, row_ptr[n] = nnz); col_idx[nnz] int32 sorted
 * strictly ascending within every row; weights[nnz] int8 in {-1,+1} with
 * w_uv == w_vu, or NULL for an unweighted graph.  The pattern must be
 * symmetric with no self loops.  is_device_ptr = 1 if the three arrays are
 * device pointers (row_ptr is copied to the host; the entries are copied
 * device to device).  The row pointers are checked on the host; the entries
 * (range, self loops, order, weights, symmetry, member graphs) by a kernel
 * after the upload when a GPU is present, else on the host, with the same
 * messages.  Validation failures return MQO_EGRAPH.  Synchronises cuda_stream.
 */
MQO_API mqo_status mqo_graph_create_csr(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                const int8_t* weights, int32_t is_device_ptr, void* cuda_stream,
                                mqo_graph* out);

/*
 * Create a block-diagonal batch of num_graphs independent graphs from one
 * packed CSR: node_offsets[num_graphs+1] (int64, node_offsets[0] = 0)
 * delimits the member graphs; row_ptr/col_idx/weights as in
 * mqo_graph_create_csr over all nodes, with global node ids; no edge may
 * join two member graphs.  Each member graph gets its own B trajectories.
 */
MQO_API mqo_status mqo_graph_create_packed(int32_t num_graphs, const int64_t* node_offsets, int64_t nnz,
                                   const int64_t* row_ptr, const int32_t* col_idx, const int8_t* weights,
                                   int32_t is_device_ptr, void* cuda_stream, mqo_graph* out);

/* Free a graph.  No solver created from it may be used afterwards. */
MQO_API mqo_status mqo_graph_destroy(mqo_graph g);

/* Node count, directed nnz and member-graph count of a graph (host). */
MQO_API mqo_status mqo_graph_info(mqo_graph g, int64_t* n, int64_t* nnz, int32_t* num_graphs);

/* ---------------------------------------------------------------- solver */

/*
 * Create a solver (all device state of G*B trajectories) on cuda_stream.
 * Rejects MIS on a weighted graph, batch not a power of two in [1,128],
 * descent_cap < 1, lambda outside (0,2) for MaxCut, gamma <= 1 for MIS.
 * The trajectories are initialised as by mqo_init.
 */
MQO_API mqo_status mqo_solver_create(mqo_graph g, const mqo_params* p, void* cuda_stream, mqo_solver* out);
MQO_API mqo_status mqo_solver_destroy(mqo_solver s);

/*
 * Initialise every trajectory (Alg. 1/2 step 2, outer iteration 0):
 * x from the Philox4x64-10 stream keyed (seed, trajectory), V = 0,
 * best = none, machine in its first descent.
 */
MQO_API mqo_status mqo_init(mqo_solver s);

/*
 * nsteps plain fused steps for every trajectory (the gradient of Eq. 3 / Eq. 7 as a CSR SpMM, the momentum step, the
 * projection onto the box, threshold rounding of Sec. 3 and the exact
 * evaluation of the rounded point, all in one kernel per step).  The
 * machine state is left untouched; mqo_step_stats reads the evaluation of
 * the last step.
 */
MQO_API mqo_status mqo_step(mqo_solver s, int32_t nsteps);

/*
 * Exact evaluation of z(x_t) made by the last mqo_step, per trajectory,
 * into device int64 arrays of length G*B (any may be NULL): value (MIS
 * size | cut), a (MIS conflicting nodes | MaxCut nodes that a PGA step of
 * the solver's relaxation would move, i.e. not fixed under it),
 * b (MIS uncovered nodes | MaxCut positive-gain nodes).
 */
MQO_API mqo_status mqo_step_stats(mqo_solver s, int64_t* value, int64_t* a, int64_t* b);

/*
 * nticks ticks of the full per-trajectory machine (Alg. 1 / Alg. 2 with a
 * tick budget in place of the wall clock): each tick every trajectory
 * takes one descent step or one discrete round; descents end at the
 * fixed-point test (Eq. 8; for MaxCut the fixed point of the
 * solver's relaxation, e.g. f_B, Thm 3.6) or at
 * descent_cap; strict acceptance (Alg. 1 steps 4/10); reset rounds from the
 * best set (steps 6-8); local search after t_gs rounds (step 11); a fresh
 * initialisation after local search.  The tick loop runs as a captured
 * CUDA graph.
 */
MQO_API mqo_status mqo_run(mqo_solver s, int64_t nticks);

/*
 * Force a mutation reset now (Alg. 1/2 steps 6-8) for the trajectories
 * whose byte in traj_mask (device, G*B bytes; NULL = all) is non-zero:
 * x <- best set (MIS 1/0, MaxCut +1/-1), x_R <- 0 with |R| = floor(rho n_g)
 * drawn from the trajectory's reset stream for round r+1, V <- 0, and the
 * trajectory starts a new descent.  MQO_EINVAL in pool mode, where resets
 * start from pool members chosen by the pool machine.
 */
MQO_API mqo_status mqo_reset(mqo_solver s, const uint8_t* traj_mask);

/* Threshold rounding (Sec. 3) of the current x into z_bits (device,
 * node-major bit layout, n*Bw uint32 words). */
MQO_API mqo_status mqo_round(mqo_solver s, uint32_t* z_bits);

/*
 * Exact integer evaluation of binary points z_bits (device, node-major bit
 * layout) per trajectory into device int64 arrays of length G*B (any may
 * be NULL).  MIS: value = |I|, conflicts = edges inside I, uncovered =
 * nodes outside I with no neighbour in I.  MaxCut: value = cut weight,
 * conflicts = nodes that are not f_B-fixed, uncovered = nodes with a
 * positive 1-flip gain.
 */
MQO_API mqo_status mqo_evaluate(mqo_solver s, const uint32_t* z_bits, int64_t* value, int64_t* conflicts,
                        int64_t* uncovered);

/*
 * Local search on the best set of every trajectory, run to convergence
 * (OneTwoSwap for MIS, OneTwoFlip for MaxCut; Sec. 4 and Defs. 2.3-2.5):
 * rounds are applied until none changes the set, then the result is
 * accepted if it is strictly better.  Synchronises the stream (the number
 * of rounds is data dependent; max_rounds bounds it).  MQO_EINVAL in pool
 * mode, where the pool machine runs its own local search (Alg. 3/4 step 13).
 */
MQO_API mqo_status mqo_local_search(mqo_solver s, int32_t max_rounds);

/*
 * As mqo_run, with the nticks ticks captured as one CUDA graph that holds
 * an event-record node between consecutive kernels on the solver's stream;
 * synchronises and writes, summed over the nticks ticks, the milliseconds
 * spent in each of the tick's seven kernels to phase_ms[7] (control, apply,
 * fused step, discrete pass A, pass B, count pass C, tick end), and the
 * number of kernel launches to *launches (either pointer may be NULL).
 * Used to profile the tick kernel by kernel.
 */
MQO_API mqo_status mqo_run_timed(mqo_solver s, int64_t nticks, double* phase_ms, int64_t* launches);

/* mqo_init followed by mqo_run(s, nticks). */
MQO_API mqo_status mqo_solve(mqo_solver s, int64_t nticks);

/*
 * Best-so-far readout (Alg. 1/2 output): values (host int64, G*B; may be
 * NULL) and the best sets (device, node-major bit layout; may be NULL).
 * Synchronises the stream.
 */
MQO_API mqo_status mqo_best(mqo_solver s, int64_t* values, uint32_t* z_bits);

/*
 * Pool readout (pool mode, pool_k = K > 0; pmQO, Alg. 3/4): for every member
 * graph g, counts[g] (host int32[G]) = pool members so far (<= K), values
 * (host int64[G*K]) = their exact values, best first (entries beyond
 * counts[g] undefined), merges (host int64[G]) = pool merges so far, and
 * bits (device, n*Kw uint32 words, Kw = ceil(K/32)) = the member sets,
 * node-major: member k of node v is bit k%32 of word v*Kw + k/32.  Any
 * pointer may be NULL.  MQO_EINVAL if the solver is not in pool mode.
 * Synchronises the stream.
 */
MQO_API mqo_status mqo_pool_state(mqo_solver s, int32_t* counts, int64_t* values, int64_t* merges, uint32_t* bits);

/* Per-trajectory machine state (host array of G*B mqo_traj_info).  Synchronises. */
MQO_API mqo_status mqo_traj_state(mqo_solver s, mqo_traj_info* out);

/*
 * Execution plan (chosen at creation or by mqo_autotune; host, any pointer
 * may be NULL): *step_kernel bit 0 = the fused step stages each member
 * graph's block of x in shared memory (every member graph fits; else the
 * global-memory kernel), bit 1 = the discrete passes run fused, one CTA per
 * member graph (else three node-parallel launches), bit 2 = the
 * shared-memory step kernel uses 16-byte lanes (twice the trajectories per
 * lane, twice the rows per warp), bit 3 = the global-memory step runs as the
 * staged-gather kernel (each CTA copies every neighbour row of x of a slice
 * of rows into shared memory before summing), bits 4..7 = trajectories per
 * lane of a global-memory step kernel (0 with bit 0), bits 8..15 = KB of
 * gathered rows of x per staged slice (0 without bit 3), bit 16 = the
 * shared-memory step kernel reads 16-bit member-local column indices (kept
 * by the graph when every member graph has fewer than 65535 nodes, 2 bytes
 * per entry of device memory), bit 17 = the shared-memory step kernel reads
 * its neighbours from the solver's sliced-ELL stream (the rows of a warp
 * padded to a common length, four neighbour offsets per 16-byte vector;
 * 2-byte x, MIS with bfloat16 x or unweighted MaxCut; about 4 bytes of
 * device memory per entry and lane width); *smem_bytes = the
 * shared-memory step kernel's dynamic shared memory per CTA; *items = work
 * items (node ranges of at most 256 nodes); *replicas = counter replicas per
 * trajectory.
 */
MQO_API mqo_status mqo_solver_info(mqo_solver s, int32_t* step_kernel, int64_t* smem_bytes, int32_t* items,
                                   int32_t* replicas);

/*
 * Autotuner of the launch plan: every plan the solver can run (shared-memory
 * or global-memory step kernel; for the former lane width and neighbour
 * stream, for the latter each choice of trajectories per lane, i.e. lanes
 * per row, and of staged slices; fused or node-parallel discrete passes)
 * runs `ticks` machine ticks from the current state; the state is restored
 * after every trial, so tuning changes no result (all plans compute the same
 * ticks bit for bit).  The current plan is timed first; another replaces it
 * only if more than 3 % faster.  The chosen plan is kept for later ticks.  Writes the
 * plan to *plan (the bits of mqo_solver_info's *step_kernel) and its time
 * per tick in milliseconds to *ms_per_tick
 * (either may be NULL).  Allocates a snapshot of the solver's state for the
 * duration of the call and synchronises.
 */
MQO_API mqo_status mqo_autotune(mqo_solver s, int32_t ticks, int32_t* plan, double* ms_per_tick);

/* Copy the current relaxed iterate X (n*B values of x_dtype, node-major)
 * to / from device memory.  During a discrete phase a trajectory's x is
 * not defined and mqo_get_x returns stale values for it. */
MQO_API mqo_status mqo_get_x(mqo_solver s, void* x_out);
MQO_API mqo_status mqo_set_x(mqo_solver s, const void* x_in);
/* Same for the momentum V (n*B values of v_dtype). */
MQO_API mqo_status mqo_get_v(mqo_solver s, void* v_out);

/*
 * Relaxed objective of the current x per trajectory, in double precision
 * (h of Eq. 3, or the solver's MaxCut relaxation: f_B of
 * Eq. 7, f_L, f_P or f_A of Sec. 3), into device double
 * out[G*B].  (Ax)_v is accumulated in float32 in CSR order; products and
 * sums are in double.
 */
MQO_API mqo_status mqo_objective_f64(mqo_solver s, double* out);

/* ------------------------------------------------------ graph-level kernels */

/*
 * Forward of f_B for a float32 block X (device, n*B node-major) of a graph
 * (the whole packed node range): obj[b] = -lambda sum_v x_vb
 * - sum_v x_vb (A x_b)_v in double (device double[B]).  Rows of degree above
 * an internal split are accumulated in chunks (fixed order).  B a power of
 * two in [1,256]; for B >= 32, X must be 16-byte aligned (rows are read in
 * 16-byte pieces), else MQO_EINVAL and nothing is launched.
 */
MQO_API mqo_status mqo_fb_forward(mqo_graph g, const float* X, int32_t B, float lambda_, double* obj, void* cuda_stream);

/*
 * Backward of f_B (gradient, Thm 3.6 proof: grad f_B = -lambda 1 - 2 A x):
 * G[v*B+b] = gout[b] * (-lambda - 2 (A X)_{vb}), float32, device arrays;
 * gout may be NULL (taken as 1).  Uses library-owned scratch for the
 * chunk partial sums of high-degree rows.  B and the alignment of X as for
 * mqo_fb_forward.
 */
MQO_API mqo_status mqo_spmm_grad(mqo_graph g, const float* X, const float* gout, float* G, int32_t B, float lambda_,
                         void* cuda_stream);

/*
 * Same result as mqo_spmm_grad, but the call allocates nothing.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc during the call -- applications whose device memory is already
 * held by their own pool or allocator, and loops that must not pay for
 * cudaMalloc / cudaFree, which can synchronise the device.  mqo_spmm_grad
 * keeps a scratch buffer for the partial sums of
 * long rows and allocates (or grows) it on first use; this variant keeps
 * those partial sums in one static device array of 4 MiB (1,048,576 32-bit
 * words) that every GPU loading the library holds until the process exits.
 *
 * Limit: 64 + 2*L + C*B words must fit in that array, where L is the number
 * of rows with more than 512 entries and C the number of their 512-entry
 * chunks; larger requests return MQO_EINVAL with the required size in
 * mqo_last_error() and launch nothing.  B is a power of two in [1, 256].
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call on a device shares the same array: calls
 * whose work overlaps on the GPU (on different streams without ordering)
 * race and give wrong results; calls ordered on one stream are safe.
 * Arguments, layouts and the returned gradient are those of mqo_spmm_grad.
 */
MQO_API mqo_status mqo_spmm_grad_static(mqo_graph g, const float* X, const float* gout, float* G, int32_t B,
                                        float lambda_, void* cuda_stream);

/*
 * Projected optimiser updates on device float32 arrays of length count,
 * ascending along grad and projecting onto [lo, hi] (the PGA update of
 * Sec. 3 with momentum or Adam):
 *   momentum: v <- mu v + grad;  x <- Pi(x + lr v)
 *   adam:     m <- b1 m + (1-b1) grad;  u <- b2 u + (1-b2) grad^2;
 *             x <- Pi(x + lr (m / (1-b1^t)) / (sqrt(u / (1-b2^t)) + eps))
 */
MQO_API mqo_status mqo_pga_momentum_step(float* x, float* v, const float* grad, int64_t count, float lr, float mu,
                                 float lo, float hi, void* cuda_stream);
MQO_API mqo_status mqo_pga_adam_step(float* x, float* m, float* u, const float* grad, int64_t count, float lr, float b1,
                             float b2, float eps, int64_t t, float lo, float hi, void* cuda_stream);

/*
 * Measured shared-memory load bandwidth of the current device (bytes per
 * second over all SMs, in GB/s, into host *gbs): two CTAs per SM stream
 * conflict-free 16-byte loads, `iters` iterations of four loads per thread,
 * one untimed launch then one timed with CUDA events.  The denominator of
 * the shared-memory step kernel's roofline (a measurement aid; no part of the
 * method).  Synchronises; MQO_EINVAL for iters < 1 or a null pointer.
 */
MQO_API mqo_status mqo_measure_smem_gbs(int32_t iters, double* gbs);

/* Thread-local message for the last failure on this thread ("" if none). */
MQO_API const char* mqo_last_error(void);

/* Library version string. */
MQO_API const char* mqo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MQO_H */
