/*
 * mqo_oracle.c -- plain, slow, single-threaded CPU oracle of the mQO hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it, to check the CUDA library against an independent
 * restatement of the method.  It shares no code, header, table or constant
 * generator with the CUDA sources.
 *
 * Method: "Mutation-Guided Differentiable Quadratic Combinatorial
 * Optimization" (mQO).  Every function cites the passage it follows.
 * Compile with -O2 -ffp-contract=off so that every float expression is
 * evaluated exactly as written (one IEEE round-to-nearest per operation).
 *
 * One graph, one trajectory at a time.  The graph is symmetric CSR with
 * rows sorted ascending, optional int8 edge weights in {-1,+1}.
 *
 * Parity status of each function (see the pins in tests/test_oracle_*.py):
 *   philox4x64_10            pinned: numpy.random.Philox outputs
 *   round_store              pinned: numpy float16 / torch bfloat16 casts
 *   eval_mis / eval_cut      pinned: brute force, textbook definitions
 *   descent_step             pinned: closed-form gradients, finite differences
 *   feistel_sigma            pinned: bijection + exact |R| by enumeration,
 *                            uniformity by chi-square
 *   repair / local search    pinned: invariants (independent, maximal,
 *                            swap-free / flip-free, exact gains), brute force
 *   orc_ls_*_sequential      pinned: the same invariants, move counts against
 *                            the value gained
 *   orc_init_x               pinned: exact projected centres of Alg. 1/2
 *                            step 2 at sigma = 0, noise mean and spread
 *   reset_from / accept      pinned through the machine: the first step after
 *                            a reset starts from the point of Alg. 1/2 steps
 *                            6-8; equal-valued candidates leave the best set
 *   run_trajectory           pinned through its parts + brute-force bound
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

enum { ORC_MIS = 0, ORC_MAXCUT = 1 };
enum { ORC_F_B = 0, ORC_F_L = 1, ORC_F_P = 2, ORC_F_A = 3 };
enum { ORC_F32 = 0, ORC_BF16 = 1, ORC_F16 = 2 };
enum { ORC_PH_DESCENT = 0, ORC_PH_REPAIR = 1, ORC_PH_LS = 2, ORC_PH_WAIT = 3 };
enum {
  ORC_R_NONE = -1,
  ORC_R_COUNT = 0,
  ORC_R_DROP = 1,
  ORC_R_COMPLETE = 2,
  ORC_R_SWAP = 3,
  ORC_R_FLIP1 = 4,
  ORC_R_FLIP2 = 5
};

typedef struct {
  int64_t n;
  const int64_t* row_ptr; /* n+1 */
  const int32_t* col;     /* nnz */
  const int8_t* w;        /* nnz or NULL (all ones) */
} orc_graph;

typedef struct {
  int32_t problem;
  int32_t batch;
  int32_t x_dtype;
  int32_t v_dtype;
  float alpha;
  float momentum;
  float gamma;
  float lambda_;
  double rho;
  float sigma;
  int32_t t_gs;
  int32_t descent_cap;
  int32_t init_kind;
  int32_t local_search;
  int32_t repair;
  uint64_t seed;
  int32_t pool_k;     /* 0: independent trajectories (Alg. 1/2); K >= 1: pmQO pool (Alg. 3/4) */
  int32_t objective;  /* MaxCut relaxation: ORC_F_B (Eq. 7), ORC_F_L (Eq. 4),
                         ORC_F_P (Eq. 5), ORC_F_A (Eq. 6) */
} orc_params;

/* Per-trajectory machine state, mirrored field by field for the tests. */
typedef struct {
  int32_t phase;
  int32_t s;          /* descent ticks completed in the current descent */
  int32_t r;          /* reset rounds started in this outer iteration */
  int32_t o;          /* outer iteration */
  int64_t best;       /* INT64_MIN until the first acceptance */
  int64_t ticks;
  int32_t last_round; /* discrete round type run in the last tick */
  int64_t last_commits;
  /* evaluation of the last tick (descent: of z(x_t); discrete: of zwork) */
  int64_t ev_value;   /* MIS size or cut */
  int64_t ev_a;       /* MIS: conflicting nodes; MaxCut: non-fixed nodes */
  int64_t ev_b;       /* MIS: uncovered (free) nodes; MaxCut: 1-flip candidates */
  int64_t accepts;
  int64_t descents;
  int64_t held;       /* pool mode: value of the set held while waiting, INT64_MIN if none */
  /* where the best value came from (the gains breakdown of the appendix on
   * mQO's gains): the first accepted value (the end of the first descent's
   * gradient updates), then the strict improvements accepted from later
   * descents (global resets and restarts) and from local search */
  int64_t first_value; /* INT64_MIN until the first acceptance */
  int64_t gain_descent;
  int64_t gain_ls;
  int64_t steps;       /* descent steps taken in all */
} orc_state;

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies */
/* with a Weyl-sequence key schedule.                                   */
/* ------------------------------------------------------------------ */
static void mul128(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

ORC_API void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B97F4A7C15ULL; /* golden ratio */
      k1 += 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul128(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
    mul128(0xCA5A826395121157ULL, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout of the two random draws the method makes.            */
/* key = (seed, trajectory id); ctr = (tag, outer iteration, a, b).      */
#define ORC_TAG_INIT 1ULL
#define ORC_TAG_RESET 2ULL
#define ORC_TAG_POOL 3ULL

/* top 24 bits of a 64-bit word as an exact float in [0,1) */
static float u24(uint64_t w) { return (float)(w >> 40) * (1.0f / 16777216.0f); }

/* ------------------------------------------------------------------ */
/* Storage rounding: IEEE round-to-nearest-even into bfloat16 / binary16 */
/* written from the format definitions.                                */
/* ------------------------------------------------------------------ */
static float to_bf16(float f) {
  /* bfloat16 keeps the float's sign and 8-bit exponent and 7 mantissa
   * bits: round the magnitude to a multiple of 2^(e-7) for 2^e <= |f|. */
  if (!isfinite(f) || f == 0.0f) return f;
  double a = fabs((double)f);
  int e;
  frexp(a, &e);       /* a = m * 2^e, m in [0.5,1) -> leading bit 2^(e-1) */
  int lead = e - 1;
  if (lead < -126) lead = -126; /* bfloat16 subnormals share float's */
  double q = ldexp(1.0, lead - 7);
  double r = rint(a / q) * q;   /* rint: ties to even in default mode */
  if (r >= ldexp(1.0, 128)) r = INFINITY;
  return (float)(f < 0 ? -r : r);
}

static float to_f16(float f) {
  /* binary16: 5-bit exponent (bias 15), 10 mantissa bits, subnormal
   * quantum 2^-24, largest finite 65504. */
  if (!isfinite(f) || f == 0.0f) return f;
  double a = fabs((double)f);
  int e;
  frexp(a, &e);
  int lead = e - 1;
  if (lead < -14) lead = -14;
  double q = ldexp(1.0, lead - 10);
  double r = rint(a / q) * q;
  if (r > 65504.0) r = INFINITY;
  return (float)(f < 0 ? -r : r);
}

ORC_API float orc_round_store(float x, int32_t dtype) {
  if (dtype == ORC_BF16) return to_bf16(x);
  if (dtype == ORC_F16) return to_f16(x);
  return x;
}

/* ------------------------------------------------------------------ */
/* Initialisation (Alg. 1 step 2 and Alg. 2 step 2; uniform option).    */
/* ------------------------------------------------------------------ */
static void box(const orc_params* p, float* lo, float* hi) {
  if (p->problem == ORC_MIS) { *lo = 0.0f; *hi = 1.0f; }
  else { *lo = -1.0f; *hi = 1.0f; }
}

static float clampf(float v, float lo, float hi) {
  /* projection onto [lo,hi] (the box Pi of Sec. 3) */
  if (v < lo) return lo;
  if (v > hi) return hi;
  return v;
}

ORC_API void orc_init_x(const orc_graph* g, const orc_params* p, int64_t traj, int64_t outer, float* x) {
  float lo, hi;
  box(p, &lo, &hi);
  int64_t dmax = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
    if (d > dmax) dmax = d;
  }
  uint64_t key[2] = {p->seed, (uint64_t)traj};
  for (int64_t v = 0; v < g->n; ++v) {
    uint64_t ctr[4] = {ORC_TAG_INIT, (uint64_t)outer, (uint64_t)v, 0};
    uint64_t r[4];
    orc_philox4x64_10(ctr, key, r);
    float val;
    if (p->init_kind == 0) {
      /* x ~ U(lo, hi) */
      float u = u24(r[0]);
      val = lo + (hi - lo) * u;
    } else {
      /* degree-based centre d_base (MIS: 1 - d/Delta; MaxCut:
       * 2(1 - d/Delta) - 1) plus Gaussian-like noise of std sigma:
       * a sum of four uniforms, centred and scaled to unit variance
       * (Irwin-Hall, variance 4/12). */
      int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
      float q = dmax > 0 ? (float)d / (float)dmax : 0.0f;
      float base = 1.0f - q;
      if (p->problem == ORC_MAXCUT) base = 2.0f * base - 1.0f;
      float s = u24(r[0]) + u24(r[1]);
      s = s + u24(r[2]);
      s = s + u24(r[3]);
      s = s - 2.0f;
      float eps = s * 1.7320508075688772f;
      eps = p->sigma * eps;
      val = clampf(base + eps, lo, hi);
    }
    x[v] = orc_round_store(val, p->x_dtype);
  }
}

/* ------------------------------------------------------------------ */
/* Reset set R (Sec. 4: |R| = floor(rho n), uniform without replacement) */
/* A keyed pseudo-random permutation sigma of {0..n-1} is built from an  */
/* alternating-width Feistel network on d = ceil(log2 n) bits with       */
/* cycle walking (the bijective-shuffle construction of Mitchell et al., */
/* "Bandwidth-optimal random shuffling for GPUs", 2022); the round       */
/* function is Wellons' "lowbias32" integer hash of (half ^ key_i).      */
/* R = { v : sigma(v) < floor(rho n) } has exactly floor(rho n) members. */
/* ------------------------------------------------------------------ */
static uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

ORC_API void orc_reset_keys(uint64_t seed, int64_t traj, int64_t outer, int64_t round, uint32_t keys[6]) {
  uint64_t key[2] = {seed, (uint64_t)traj};
  uint64_t ctr[4] = {ORC_TAG_RESET, (uint64_t)outer, (uint64_t)round, 0};
  uint64_t r[4];
  orc_philox4x64_10(ctr, key, r);
  for (int i = 0; i < 3; ++i) {
    keys[2 * i] = (uint32_t)(r[i] & 0xffffffffULL);
    keys[2 * i + 1] = (uint32_t)(r[i] >> 32);
  }
}

static int ceil_log2(int64_t n) {
  int d = 0;
  while (((int64_t)1 << d) < n) ++d;
  return d;
}

static uint64_t feistel(uint64_t v, int d, const uint32_t keys[6]) {
  int wl = d / 2;       /* left half width */
  int wr = d - wl;      /* right half width */
  uint64_t L = v >> wr;
  uint64_t R = v & ((1ULL << wr) - 1ULL);
  for (int i = 0; i < 6; ++i) {
    uint64_t f = (uint64_t)lowbias32((uint32_t)R ^ keys[i]) & ((1ULL << wl) - 1ULL);
    uint64_t nl = R, nr = L ^ f;
    int t = wl; wl = wr; wr = t;  /* new left has the old right width */
    L = nl; R = nr;
  }
  return (L << wr) | R;
}

ORC_API int64_t orc_feistel_sigma(int64_t n, const uint32_t keys[6], int64_t v) {
  if (n <= 1) return v;
  int d = ceil_log2(n);
  if (d < 2) d = 2;
  uint64_t y = feistel((uint64_t)v, d, keys);
  while (y >= (uint64_t)n) y = feistel(y, d, keys);
  return (int64_t)y;
}

ORC_API int64_t orc_reset_count(int64_t n, double rho) {
  return (int64_t)floor(rho * (double)n);
}

ORC_API void orc_reset_mask(int64_t n, double rho, uint64_t seed, int64_t traj, int64_t outer, int64_t round,
                            uint8_t* in_r) {
  uint32_t keys[6];
  orc_reset_keys(seed, traj, outer, round, keys);
  int64_t k = orc_reset_count(n, rho);
  for (int64_t v = 0; v < n; ++v) in_r[v] = orc_feistel_sigma(n, keys, v) < k;
}

/* ------------------------------------------------------------------ */
/* Exact evaluation of binary points (Def. 2.1/2.2, Eq. 1, Eq. 2,       */
/* checker Eq. 8).                                                      */
/* ------------------------------------------------------------------ */
static int8_t wt(const orc_graph* g, int64_t j) { return g->w ? g->w[j] : (int8_t)1; }

/* MIS: size = sum z; conflicting edges = edges with both ends in z;
 * conflicting nodes = z-nodes with a z-neighbour; uncovered = non-z nodes
 * with no z-neighbour.  The PGA fixed-point checker on binary z holds iff
 * conflicting nodes == 0 and uncovered == 0 (z is a maximal independent
 * set): with grad h = 1 - gamma A z and gamma > 1, an in-set node is fixed
 * iff (Az)_v <= 1/gamma, i.e. (Az)_v = 0, and an out-of-set node iff
 * (Az)_v >= 1/gamma, i.e. (Az)_v >= 1. */
ORC_API void orc_eval_mis(const orc_graph* g, const uint8_t* z, int64_t out[4]) {
  int64_t size = 0, conf_edges2 = 0, conf_nodes = 0, unc = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    int64_t c = 0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) c += z[g->col[j]] ? 1 : 0;
    if (z[v]) {
      size += 1;
      conf_edges2 += c;
      if (c > 0) conf_nodes += 1;
    } else if (c == 0) {
      unc += 1;
    }
  }
  out[0] = size;
  out[1] = conf_edges2 / 2;
  out[2] = conf_nodes;
  out[3] = unc;
}

/* MaxCut on z (1 = node in S, i.e. x_v = +1; 0 = in S-bar, x_v = -1).
 * cut = sum over undirected edges of w_uv [z_u != z_v].  gain_v = s_v (A s)_v
 * is the cut change of flipping v alone (proof of Prop. 3.4).  A binary
 * point is a PGA fixed point of f_B (Thm 3.6) iff for every v:
 * s_v = +1 and (As)_v <= -1, or s_v = -1 and (As)_v >= 0 (grad f_B =
 * -lambda 1 - 2 A s, 0 < lambda < 2, integer weights). */
/* The same with the fixed-point rule of another MaxCut relaxation, from
 * the sign of its gradient at the binary point s (d_v = sum of w_vu):
 *   f_L = 1/4 s'Ls:        grad = 1/2 (d_v s_v - (As)_v)
 *   f_P = s'(L + lambda I)s: grad = 2 (d_v s_v - (As)_v + lambda s_v)
 *   f_A = -s'As:           grad = -2 (As)_v
 * s_v = +1 is fixed iff grad_v >= 0 and s_v = -1 iff grad_v <= 0. */
ORC_API void orc_eval_cut_obj(const orc_graph* g, const uint8_t* z, int32_t objective, float lambda_,
                              int64_t out[4]) {
  int64_t cut2 = 0, nonfixed = 0, cand = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    int64_t as = 0, d = 0;
    int sv = z[v] ? 1 : -1;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      int32_t u = g->col[j];
      int su = z[u] ? 1 : -1;
      as += (int64_t)wt(g, j) * su;
      d += wt(g, j);
      if (z[u] != z[v]) cut2 += wt(g, j);
    }
    int64_t gain = sv * as;
    if (gain > 0) cand += 1;
    int fixed;
    switch (objective) {
      case ORC_F_L: fixed = (sv == 1) ? (as <= d) : (as >= -d); break;
      case ORC_F_P: fixed = (sv == 1) ? ((double)(as - d) <= (double)lambda_)
                                      : ((double)(-(as + d)) <= (double)lambda_); break;
      case ORC_F_A: fixed = (sv == 1) ? (as <= 0) : (as >= 0); break;
      default: fixed = (sv == 1) ? (as <= -1) : (as >= 0); break;
    }
    if (!fixed) nonfixed += 1;
  }
  out[0] = cut2 / 2;
  out[1] = nonfixed;
  out[2] = cand;
  out[3] = 0;
}

ORC_API void orc_eval_cut(const orc_graph* g, const uint8_t* z, int64_t out[4]) {
  orc_eval_cut_obj(g, z, ORC_F_B, 0.001f, out);
}

/* The ascent direction of a step at x_v given acc = (Ax)_v (float, CSR
 * order): MIS grad h = 1 - gamma (Ax)_v; MaxCut, by relaxation:
 *   f_B: -lambda - 2 (Ax)_v;   f_A: -2 (Ax)_v;
 *   f_L: 1/2 (d_v x_v - (Ax)_v);   f_P: 2 ((d_v x_v - (Ax)_v) + lambda x_v),
 * d_v the (weighted) degree; every operation rounds once, as written. */
static float step_grad(const orc_graph* g, const orc_params* p, int64_t v, float xv, float acc) {
  if (p->problem == ORC_MIS) {
    float t = p->gamma * acc;
    return 1.0f - t;
  }
  if (p->objective == ORC_F_B || p->objective == ORC_F_A) {
    float t = 2.0f * acc;
    return p->objective == ORC_F_B ? -p->lambda_ - t : -t;
  }
  int64_t d = 0;
  for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) d += wt(g, j);
  float t1 = (float)d * xv;
  float t2 = t1 - acc;
  if (p->objective == ORC_F_L) return 0.5f * t2;
  float t3 = p->lambda_ * xv;
  float t4 = t2 + t3;
  return 2.0f * t4;
}

/* threshold rounding (Sec. 3): MIS I = {x_v > 0.5}; MaxCut S = {x_v > 0} */
static uint8_t round_z(const orc_params* p, float x) {
  return p->problem == ORC_MIS ? (uint8_t)(x > 0.5f) : (uint8_t)(x > 0.0f);
}

/* ------------------------------------------------------------------ */
/* One projected momentum-gradient-ascent step (Sec. 3 PGA update,      */
/* MGA as used in Sec. 5), heavy-ball form V <- mu V + alpha grad,       */
/* x <- Pi(x + V).  Gradients: MIS grad h = 1 - gamma A x (Eq. 3);*/
/* MaxCut grad f_B = -lambda 1 - 2 A x (Eq. 7).          */
/* (Ax)_v is accumulated in float in CSR order, one rounding per add.    */
/* z of the incoming x is evaluated exactly (checker / cut).             */
/* ------------------------------------------------------------------ */
ORC_API void orc_descent_step(const orc_graph* g, const orc_params* p, const float* x, const float* V, float* x_new,
                              float* V_new, uint8_t* z_out, int64_t ev[4]) {
  float lo, hi;
  box(p, &lo, &hi);
  for (int64_t v = 0; v < g->n; ++v) z_out[v] = round_z(p, x[v]);
  int64_t tmp[4];
  if (p->problem == ORC_MIS) {
    orc_eval_mis(g, z_out, tmp);
    ev[0] = tmp[0]; ev[1] = tmp[2]; ev[2] = tmp[3]; ev[3] = 0;
  } else {
    orc_eval_cut_obj(g, z_out, p->objective, p->lambda_, tmp);
    ev[0] = tmp[0]; ev[1] = tmp[1]; ev[2] = tmp[2]; ev[3] = 0;
  }
  for (int64_t v = 0; v < g->n; ++v) {
    float acc = 0.0f;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      float xu = x[g->col[j]];
      if (wt(g, j) >= 0) acc = acc + xu;
      else acc = acc - xu;
    }
    float grad = step_grad(g, p, v, x[v], acc);
    float a = p->momentum * V[v];
    float b = p->alpha * grad;
    float vn = a + b;
    float xn = clampf(x[v] + vn, lo, hi);
    V_new[v] = orc_round_store(vn, p->v_dtype);
    x_new[v] = orc_round_store(xn, p->x_dtype);
  }
}

/* The same step restricted to the listed rows (for sampled checks on
 * graphs too large to step whole): x_new[k], V_new[k] for row rows[k]. */
ORC_API void orc_step_rows(const orc_graph* g, const orc_params* p, const float* x, const float* V,
                           const int64_t* rows, int64_t k, float* x_new, float* V_new) {
  float lo, hi;
  box(p, &lo, &hi);
  for (int64_t i = 0; i < k; ++i) {
    int64_t v = rows[i];
    float acc = 0.0f;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      float xu = x[g->col[j]];
      if (wt(g, j) >= 0) acc = acc + xu;
      else acc = acc - xu;
    }
    float grad = step_grad(g, p, v, x[v], acc);
    float a = p->momentum * V[v];
    float b = p->alpha * grad;
    float vn = a + b;
    float xn = clampf(x[v] + vn, lo, hi);
    V_new[i] = orc_round_store(vn, p->v_dtype);
    x_new[i] = orc_round_store(xn, p->x_dtype);
  }
}

/* ------------------------------------------------------------------ */
/* Discrete rounds.  Every decision in a round reads the snapshot of z   */
/* taken at the start of the round; the moves are applied afterwards.    */
/* Conflicts between simultaneous moves are resolved in favour of the    */
/* smallest node index, so each round equals applying its moves one by   */
/* one in index order, each a valid move of the definitions cited.       */
/* ------------------------------------------------------------------ */
static int adjacent(const orc_graph* g, int64_t a, int64_t b) {
  for (int64_t j = g->row_ptr[a]; j < g->row_ptr[a + 1]; ++j)
    if (g->col[j] == b) return 1;
  return 0;
}

/* Repair, part 1: drop every z-node that has a z-neighbour of smaller
 * index; afterwards z is independent (Def. 2.1 feasibility). */
ORC_API int64_t orc_round_drop(const orc_graph* g, uint8_t* z) {
  uint8_t* drop = calloc((size_t)g->n + 1, 1);
  int64_t k = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    if (!z[v]) continue;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      int32_t u = g->col[j];
      if (u < v && z[u]) { drop[v] = 1; break; }
    }
  }
  for (int64_t v = 0; v < g->n; ++v) if (drop[v]) { z[v] = 0; ++k; }
  free(drop);
  return k;
}

/* Repair, part 2 (and maximality step of local search): a free node has
 * no z-neighbour; add every free node with no free neighbour of smaller
 * index.  The added nodes are pairwise non-adjacent, so independence is
 * kept, and the smallest free node is always added. */
ORC_API int64_t orc_round_complete(const orc_graph* g, uint8_t* z) {
  uint8_t* fr = calloc((size_t)g->n + 1, 1);
  uint8_t* add = calloc((size_t)g->n + 1, 1);
  for (int64_t v = 0; v < g->n; ++v) {
    if (z[v]) continue;
    int any = 0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) if (z[g->col[j]]) { any = 1; break; }
    fr[v] = !any;
  }
  int64_t k = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    if (!fr[v]) continue;
    int ok = 1;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      int32_t u = g->col[j];
      if (u < v && fr[u]) { ok = 0; break; }
    }
    add[v] = (uint8_t)ok;
  }
  for (int64_t v = 0; v < g->n; ++v) if (add[v]) { z[v] = 1; ++k; }
  free(fr); free(add);
  return k;
}

/* (1,2)-swap round (Def. 2.3; OneTwoSwap of Sec. 4).  A non-z node u is
 * tight if exactly one z-neighbour exists.  A z-node v proposes removing
 * itself and adding the first pair (in CSR order of N(v)) of tight
 * neighbours a, b that are not adjacent; the set grows by exactly one.
 * Proposal v is applied unless a neighbour of a or b is proposed for
 * addition by a z-node of smaller index. */
ORC_API int64_t orc_round_swap(const orc_graph* g, uint8_t* z) {
  int64_t n = g->n;
  int32_t* c = calloc((size_t)n + 1, sizeof(int32_t));
  int32_t* owner = malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* pa = malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* pb = malloc(((size_t)n + 1) * sizeof(int32_t));
  uint8_t* commit = calloc((size_t)n + 1, 1);
  for (int64_t v = 0; v < n; ++v) {
    owner[v] = -1; pa[v] = -1; pb[v] = -1;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) c[v] += z[g->col[j]] ? 1 : 0;
  }
  for (int64_t v = 0; v < n; ++v) {
    if (!z[v]) continue;
    int found = 0;
    for (int64_t i = g->row_ptr[v]; i < g->row_ptr[v + 1] && !found; ++i) {
      int32_t a = g->col[i];
      if (z[a] || c[a] != 1) continue;
      for (int64_t j = i + 1; j < g->row_ptr[v + 1]; ++j) {
        int32_t b = g->col[j];
        if (z[b] || c[b] != 1) continue;
        if (!adjacent(g, a, b)) { pa[v] = a; pb[v] = b; found = 1; break; }
      }
    }
    if (found) { owner[pa[v]] = (int32_t)v; owner[pb[v]] = (int32_t)v; }
  }
  int64_t k = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (pa[v] < 0) continue;
    int ok = 1;
    int32_t ends[2] = {pa[v], pb[v]};
    for (int e = 0; e < 2 && ok; ++e) {
      int32_t a = ends[e];
      for (int64_t j = g->row_ptr[a]; j < g->row_ptr[a + 1]; ++j) {
        int32_t y = g->col[j];
        if (owner[y] >= 0 && owner[y] < v) { ok = 0; break; }
      }
    }
    commit[v] = (uint8_t)ok;
  }
  for (int64_t v = 0; v < n; ++v) {
    if (!commit[v]) continue;
    z[v] = 0; z[pa[v]] = 1; z[pb[v]] = 1; ++k;
  }
  free(c); free(owner); free(pa); free(pb); free(commit);
  return k;
}

static void gains(const orc_graph* g, const uint8_t* z, int64_t* gain) {
  for (int64_t v = 0; v < g->n; ++v) {
    int64_t as = 0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) as += (int64_t)wt(g, j) * (z[g->col[j]] ? 1 : -1);
    gain[v] = (z[v] ? 1 : -1) * as;
  }
}

/* 1-flip round (Def. 2.4): every node with positive flip gain and no
 * positive-gain neighbour of smaller index changes side; the cut grows by
 * the sum of their gains. */
ORC_API int64_t orc_round_flip1(const orc_graph* g, uint8_t* z) {
  int64_t* gain = malloc(((size_t)g->n + 1) * sizeof(int64_t));
  uint8_t* fl = calloc((size_t)g->n + 1, 1);
  gains(g, z, gain);
  int64_t k = 0;
  for (int64_t v = 0; v < g->n; ++v) {
    if (gain[v] <= 0) continue;
    int ok = 1;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      int32_t u = g->col[j];
      if (u < v && gain[u] > 0) { ok = 0; break; }
    }
    fl[v] = (uint8_t)ok;
  }
  for (int64_t v = 0; v < g->n; ++v) if (fl[v]) { z[v] ^= 1; ++k; }
  free(gain); free(fl);
  return k;
}

/* 2-flip round (Def. 2.5): swapping the sides of the endpoints of an
 * edge (a,b) with z_a != z_b changes the cut by gain_a + gain_b + 2 w_ab.
 * Node a proposes the first neighbour b > a (CSR order) on the other side
 * with a positive pair gain.  Each node is claimed by the smallest
 * proposer naming it; proposal a is applied if it holds both its claims
 * and no other neighbour of a or b is claimed by a smaller proposer. */
ORC_API int64_t orc_round_flip2(const orc_graph* g, uint8_t* z) {
  int64_t n = g->n;
  int64_t* gain = malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t* owner = malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* pb = malloc(((size_t)n + 1) * sizeof(int32_t));
  uint8_t* commit = calloc((size_t)n + 1, 1);
  gains(g, z, gain);
  for (int64_t v = 0; v < n; ++v) { owner[v] = -1; pb[v] = -1; }
  for (int64_t a = 0; a < n; ++a) {
    for (int64_t j = g->row_ptr[a]; j < g->row_ptr[a + 1]; ++j) {
      int32_t b = g->col[j];
      if (b <= a || z[b] == z[a]) continue;
      if (gain[a] + gain[b] + 2 * (int64_t)wt(g, j) > 0) { pb[a] = b; break; }
    }
  }
  for (int64_t a = 0; a < n; ++a) {
    if (pb[a] < 0) continue;
    if (owner[a] < 0 || a < owner[a]) owner[a] = (int32_t)a;
    if (owner[pb[a]] < 0 || a < owner[pb[a]]) owner[pb[a]] = (int32_t)a;
  }
  int64_t k = 0;
  for (int64_t a = 0; a < n; ++a) {
    if (pb[a] < 0) continue;
    int32_t b = pb[a];
    int ok = owner[a] == a && owner[b] == a;
    int32_t ends[2] = {(int32_t)a, b};
    for (int e = 0; e < 2 && ok; ++e) {
      int32_t t = ends[e];
      for (int64_t j = g->row_ptr[t]; j < g->row_ptr[t + 1]; ++j) {
        int32_t y = g->col[j];
        if (y == a || y == b) continue;
        if (owner[y] >= 0 && owner[y] < a) { ok = 0; break; }
      }
    }
    commit[a] = (uint8_t)ok;
  }
  for (int64_t a = 0; a < n; ++a) {
    if (!commit[a]) continue;
    z[a] ^= 1; z[pb[a]] ^= 1; ++k;
  }
  free(gain); free(owner); free(pb); free(commit);
  return k;
}

/* ------------------------------------------------------------------ */
/* Local search in the paper's order (Sec. 4: scan the nodes in index   */
/* order and restart after each move), for cross-checking the round-    */
/* based variant above: both must end at points with the same defining  */
/* properties.  Returns the number of moves; *adds (MIS) counts the      */
/* free nodes added.                                                     */
/* ------------------------------------------------------------------ */

/* OneTwoSwap: add free nodes (lowest index first) until maximal; then the
 * first set node v (index order) with a pair of non-adjacent tight
 * neighbours (the first such pair in CSR order of N(v)) swaps v for the
 * pair (Def. 2.3); repeat until no swap exists. */
ORC_API int64_t orc_ls_mis_sequential(const orc_graph* g, uint8_t* z, int64_t* adds) {
  const int64_t n = g->n;
  int64_t moves = 0, added = 0;
  int32_t* cnt = malloc(((size_t)n + 1) * sizeof(int32_t));
  for (;;) {
    for (int64_t v = 0; v < n; ++v) { /* completion */
      if (z[v]) continue;
      int any = 0;
      for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1] && !any; ++j) any = z[g->col[j]];
      if (!any) { z[v] = 1; ++added; }
    }
    for (int64_t v = 0; v < n; ++v) {
      cnt[v] = 0;
      for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) cnt[v] += z[g->col[j]];
    }
    int64_t fa = -1, fb = -1, fv = -1;
    for (int64_t v = 0; v < n && fv < 0; ++v) {
      if (!z[v]) continue;
      for (int64_t i = g->row_ptr[v]; i < g->row_ptr[v + 1] && fv < 0; ++i) {
        const int32_t a = g->col[i];
        if (z[a] || cnt[a] != 1) continue;
        for (int64_t j = i + 1; j < g->row_ptr[v + 1]; ++j) {
          const int32_t c = g->col[j];
          if (z[c] || cnt[c] != 1 || adjacent(g, a, c)) continue;
          fa = a; fb = c; fv = v;
          break;
        }
      }
    }
    if (fv < 0) break;
    z[fv] = 0; z[fa] = 1; z[fb] = 1;
    ++moves;
  }
  free(cnt);
  if (adds) *adds = added;
  return moves;
}

/* OneTwoFlip: the first node (index order) with a positive 1-flip gain
 * changes side (Def. 2.4), repeated until none; then the first edge (a,b),
 * a < b in CSR order, across the cut with gain_a + gain_b + 2 w_ab > 0
 * swaps sides (Def. 2.5), and the 1-flips resume; until neither applies. */
ORC_API int64_t orc_ls_cut_sequential(const orc_graph* g, uint8_t* z) {
  const int64_t n = g->n;
  int64_t moves = 0;
  int64_t* gain = malloc(((size_t)n + 1) * sizeof(int64_t));
  for (;;) {
    gains(g, z, gain);
    int64_t f = -1;
    for (int64_t v = 0; v < n && f < 0; ++v) if (gain[v] > 0) f = v;
    if (f >= 0) { z[f] ^= 1; ++moves; continue; }
    int64_t fa = -1, fb = -1;
    for (int64_t a = 0; a < n && fa < 0; ++a)
      for (int64_t j = g->row_ptr[a]; j < g->row_ptr[a + 1]; ++j) {
        const int32_t b = g->col[j];
        if (b <= a || z[b] == z[a]) continue;
        if (gain[a] + gain[b] + 2 * (int64_t)wt(g, j) > 0) { fa = a; fb = b; break; }
      }
    if (fa < 0) break;
    z[fa] ^= 1; z[fb] ^= 1;
    ++moves;
  }
  free(gain);
  return moves;
}

/* counts after a discrete round: MIS (size, conflicting nodes, free);
 * MaxCut (cut, non-fixed nodes, 1-flip candidates) */
static void disc_counts(const orc_graph* g, const orc_params* p, const uint8_t* z, orc_state* st) {
  int64_t t[4];
  if (p->problem == ORC_MIS) {
    orc_eval_mis(g, z, t);
    st->ev_value = t[0]; st->ev_a = t[2]; st->ev_b = t[3];
  } else {
    orc_eval_cut(g, z, t);
    st->ev_value = t[0]; st->ev_a = t[1]; st->ev_b = t[2];
  }
}

/* ------------------------------------------------------------------ */
/* The per-trajectory machine: Alg. 1 (MIS) / Alg. 2 (MaxCut) driven one */
/* tick at a time.  A tick is one unit of work for the trajectory: one   */
/* descent step (Alg. 1 steps 3 and 9), or one discrete round (repair of */
/* a capped descent, or one OneTwoSwap / OneTwoFlip round of step 11).   */
/* Descent ends when z(x_t) passes the fixed-point test (MIS checker,    */
/* Eq. 8; MaxCut f_B fixed point, Thm 3.6) or after           */
/* descent_cap steps.  Acceptance is strict (steps 4 and 10).  After     */
/* acceptance: reset round r+1 from the best set (steps 6-8), or after   */
/* T_gs rounds local search (step 11), then a new outer iteration        */
/* (step 2) with a fresh initialisation.  The wall-clock budget of the   */
/* paper is a tick budget here.                                          */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_graph* g;
  const orc_params* p;
  int64_t traj;
  float *x, *V, *xn, *Vn;
  uint8_t *zx_prev, *zbest, *zwork, *in_r;
  orc_state* st;
} orc_traj;

/* book a strict improvement of the best value by its source */
static void credit(orc_state* st, int64_t value, int from_ls) {
  if (st->best == INT64_MIN) st->first_value = value;
  else if (from_ls) st->gain_ls += value - st->best;
  else st->gain_descent += value - st->best;
}

static void accept(orc_traj* T, const uint8_t* src, int64_t value, int from_ls) {
  orc_state* st = T->st;
  if (value > st->best) {
    credit(st, value, from_ls);
    st->best = value;
    memcpy(T->zbest, src, (size_t)T->g->n);
    st->accepts += 1;
  }
}

static void start_outer(orc_traj* T) {
  orc_state* st = T->st;
  st->o += 1;
  st->r = 0;
  st->s = 0;
  st->phase = ORC_PH_DESCENT;
  orc_init_x(T->g, T->p, T->traj, st->o, T->x);
  for (int64_t v = 0; v < T->g->n; ++v) T->V[v] = 0.0f;
}

static void reset_from(orc_traj* T, const uint8_t* base) {
  /* Alg. 1 steps 6-8 / Alg. 2 steps 6-8: x from the base set (the best
   * set; a pool member in Alg. 3/4 step 7), then the coordinates in R are
   * set to 0; the momentum starts from zero. */
  const orc_params* p = T->p;
  orc_state* st = T->st;
  orc_reset_mask(T->g->n, p->rho, p->seed, T->traj, st->o, st->r, T->in_r);
  for (int64_t v = 0; v < T->g->n; ++v) {
    float val;
    if (p->problem == ORC_MIS) val = base[v] ? 1.0f : 0.0f;
    else val = base[v] ? 1.0f : -1.0f;
    if (T->in_r[v]) val = 0.0f;
    T->x[v] = val;
    T->V[v] = 0.0f;
  }
}

static void reset_from_best(orc_traj* T) { reset_from(T, T->zbest); }

/* returns the discrete round to run in this tick, or ORC_R_NONE */
static int after_accept(orc_traj* T) {
  orc_state* st = T->st;
  const orc_params* p = T->p;
  if (st->r < p->t_gs) {
    st->r += 1;
    st->s = 0;
    st->phase = ORC_PH_DESCENT;
    reset_from_best(T);
    return ORC_R_NONE;
  }
  if (p->local_search) {
    st->phase = ORC_PH_LS;
    memcpy(T->zwork, T->zbest, (size_t)T->g->n);
    return ORC_R_COUNT;
  }
  start_outer(T);
  return ORC_R_NONE;
}

static int64_t run_round(orc_traj* T, int kind) {
  switch (kind) {
    case ORC_R_DROP: return orc_round_drop(T->g, T->zwork);
    case ORC_R_COMPLETE: return orc_round_complete(T->g, T->zwork);
    case ORC_R_SWAP: return orc_round_swap(T->g, T->zwork);
    case ORC_R_FLIP1: return orc_round_flip1(T->g, T->zwork);
    case ORC_R_FLIP2: return orc_round_flip2(T->g, T->zwork);
    default: return 0;
  }
}

static void tick(orc_traj* T) {
  orc_state* st = T->st;
  const orc_params* p = T->p;
  int mis = p->problem == ORC_MIS;
  int round = ORC_R_NONE;
  int stepping = 0;

  /* ---- control: act on what the previous tick found ---- */
  if (st->phase == ORC_PH_DESCENT) {
    if (st->s > 0) {
      int pass = mis ? (st->ev_a == 0 && st->ev_b == 0) : (st->ev_a == 0);
      if (pass) {
        st->descents += 1;
        accept(T, T->zx_prev, st->ev_value, 0);
        round = after_accept(T);
      } else if (st->s >= p->descent_cap) {
        st->descents += 1;
        if (mis) {
          if (p->repair) {
            st->phase = ORC_PH_REPAIR;
            memcpy(T->zwork, T->zx_prev, (size_t)T->g->n);
            round = ORC_R_COUNT;
          } else {
            round = after_accept(T);
          }
        } else {
          accept(T, T->zx_prev, st->ev_value, 0);
          round = after_accept(T);
        }
      }
    }
  } else if (st->phase == ORC_PH_REPAIR) {
    if (st->ev_a > 0) round = ORC_R_DROP;
    else if (st->ev_b > 0) round = ORC_R_COMPLETE;
    else {
      accept(T, T->zwork, st->ev_value, 0);
      round = after_accept(T);
    }
  } else { /* local search */
    int done;
    if (mis) {
      if (st->ev_b > 0) { round = ORC_R_COMPLETE; done = 0; }
      else if (!(st->last_round == ORC_R_SWAP && st->last_commits == 0)) { round = ORC_R_SWAP; done = 0; }
      else done = 1;
    } else {
      if (st->ev_b > 0) { round = ORC_R_FLIP1; done = 0; }
      else if (!(st->last_round == ORC_R_FLIP2 && st->last_commits == 0)) { round = ORC_R_FLIP2; done = 0; }
      else done = 1;
    }
    if (done) {
      accept(T, T->zwork, st->ev_value, 1);
      start_outer(T);
      round = ORC_R_NONE;
    }
  }
  if (st->phase == ORC_PH_DESCENT) stepping = 1;

  /* ---- compute ---- */
  if (stepping) {
    int64_t ev[4];
    orc_descent_step(T->g, p, T->x, T->V, T->xn, T->Vn, T->zx_prev, ev);
    memcpy(T->x, T->xn, (size_t)T->g->n * sizeof(float));
    memcpy(T->V, T->Vn, (size_t)T->g->n * sizeof(float));
    st->ev_value = ev[0]; st->ev_a = ev[1]; st->ev_b = ev[2];
    st->s += 1;
    st->steps += 1;
    st->last_round = ORC_R_NONE;
    st->last_commits = 0;
  } else {
    int64_t k = run_round(T, round);
    disc_counts(T->g, p, T->zwork, st);
    st->last_round = round;
    st->last_commits = k;
  }
  st->ticks += 1;
}

ORC_API void orc_state_init(orc_state* st) {
  memset(st, 0, sizeof(*st));
  st->phase = ORC_PH_DESCENT;
  st->best = INT64_MIN;
  st->last_round = ORC_R_NONE;
  st->held = INT64_MIN;
  st->first_value = INT64_MIN;
}

/* Run one trajectory for `nticks` ticks from a fresh start (outer
 * iteration 0) or, if `resume` is set, from the state passed in.
 * x, V: n floats (in/out); zbest, zwork, zx_prev: n bytes (in/out).
 * If trace_x is not NULL it receives x after each of the first
 * trace_ticks ticks (trace_ticks * n floats). */
ORC_API void orc_run_trajectory(const orc_graph* g, const orc_params* p, int64_t traj, int64_t nticks, int32_t resume,
                                orc_state* st, float* x, float* V, uint8_t* zbest, uint8_t* zwork, uint8_t* zx_prev,
                                float* trace_x, int64_t trace_ticks) {
  int64_t n = g->n;
  orc_traj T;
  T.g = g; T.p = p; T.traj = traj; T.st = st;
  T.x = x; T.V = V; T.zbest = zbest; T.zwork = zwork; T.zx_prev = zx_prev;
  T.xn = malloc(((size_t)n + 1) * sizeof(float));
  T.Vn = malloc(((size_t)n + 1) * sizeof(float));
  T.in_r = malloc((size_t)n + 1);
  if (!resume) {
    orc_state_init(st);
    orc_init_x(g, p, traj, 0, x);
    for (int64_t v = 0; v < n; ++v) { V[v] = 0.0f; zbest[v] = 0; zwork[v] = 0; zx_prev[v] = 0; }
  }
  for (int64_t t = 0; t < nticks; ++t) {
    tick(&T);
    if (trace_x && t < trace_ticks) memcpy(trace_x + t * n, x, (size_t)n * sizeof(float));
  }
  free(T.xn); free(T.Vn); free(T.in_r);
}

/* ------------------------------------------------------------------ */
/* pmQO: Alg. 3 (MIS) and Alg. 4 (MaxCut).  The B trajectories of one   */
/* graph share a pool P_K of the K best sets found so far.  A round runs */
/* every trajectory to the end of its descent (and the repair of a      */
/* capped MIS descent); a trajectory whose descent is over holds its set */
/* and waits.  When all B wait, the graph merges them into the pool      */
/* (steps 4 and 11: P_K <- TopK(P_K U batch)), takes the best set from   */
/* the pool (steps 5 and 12), and then either starts the next round --   */
/* each trajectory draws its base set uniformly from the pool (step 7),  */
/* zeroes its reset set R (steps 8-9) and descends again (step 10) -- or */
/* after T_gs rounds runs local search (step 13: OneTwoSwap on the best  */
/* set for MIS, OneTwoFlip on every pool member for MaxCut), and then a  */
/* new outer iteration with fresh initialisations (step 2).  The pool     */
/* persists across outer iterations.  Ties in TopK keep the earlier      */
/* candidate (pool members in pool order, then the batch in trajectory   */
/* order).  Every trajectory's best set is the graph's best set.         */
/* ------------------------------------------------------------------ */
enum { ORC_EP_DESCENT = 0, ORC_EP_LS = 1 };
enum { ORC_DEC_NONE = 0, ORC_DEC_NEXT = 1, ORC_DEC_LS = 2, ORC_DEC_OUTER = 3 };

typedef struct {
  int32_t epoch;  /* ORC_EP_*: what the trajectories are finishing */
  int32_t count;  /* pool members (<= K) */
  int64_t best;   /* value of the graph's best set, INT64_MIN before the first */
  int64_t merges; /* pool merges so far */
} orc_pool;

/* Step 7: a pool index uniform in [0, count): the high word of u * count
 * for a 64-bit Philox word u keyed like the other draws. */
ORC_API int64_t orc_pool_pick(uint64_t seed, int64_t traj, int64_t outer, int64_t round, int64_t count) {
  if (count <= 0) return -1;
  uint64_t key[2] = {seed, (uint64_t)traj};
  uint64_t ctr[4] = {ORC_TAG_POOL, (uint64_t)outer, (uint64_t)round, 0};
  uint64_t r[4], hi, lo;
  orc_philox4x64_10(ctr, key, r);
  mul128(r[0], (uint64_t)count, &hi, &lo);
  return (int64_t)hi;
}

static void hold(orc_traj* T, const uint8_t* src, int64_t value) {
  if (src != T->zwork) memcpy(T->zwork, src, (size_t)T->g->n);
  T->st->held = value;
  T->st->phase = ORC_PH_WAIT;
}

/* one tick of one trajectory in pool mode; dec is the graph's decision
 * of this tick, base the set to reset from (NEXT) or to search from (LS,
 * when ls_me) */
static void tick_pool(orc_traj* T, int dec, const uint8_t* base, int ls_me) {
  orc_state* st = T->st;
  const orc_params* p = T->p;
  const int64_t n = T->g->n;
  int mis = p->problem == ORC_MIS;
  int round = ORC_R_NONE;

  if (st->phase == ORC_PH_WAIT) {
    if (dec == ORC_DEC_NEXT) {
      st->r += 1;
      st->s = 0;
      st->phase = ORC_PH_DESCENT;
      reset_from(T, base);
    } else if (dec == ORC_DEC_LS) {
      st->held = INT64_MIN;
      if (ls_me) {
        st->phase = ORC_PH_LS;
        memcpy(T->zwork, base, (size_t)n);
        round = ORC_R_COUNT;
      }
    } else if (dec == ORC_DEC_OUTER) {
      st->held = INT64_MIN;
      start_outer(T);
    }
  } else if (st->phase == ORC_PH_DESCENT) {
    if (st->s > 0) {
      int pass = mis ? (st->ev_a == 0 && st->ev_b == 0) : (st->ev_a == 0);
      if (pass) {
        st->descents += 1;
        hold(T, T->zx_prev, st->ev_value);
      } else if (st->s >= p->descent_cap) {
        st->descents += 1;
        if (mis && p->repair) {
          st->phase = ORC_PH_REPAIR;
          memcpy(T->zwork, T->zx_prev, (size_t)n);
          round = ORC_R_COUNT;
        } else {
          /* an unrepaired capped MIS point is not a candidate */
          hold(T, T->zx_prev, mis ? INT64_MIN : st->ev_value);
        }
      }
    }
  } else if (st->phase == ORC_PH_REPAIR) {
    if (st->ev_a > 0) round = ORC_R_DROP;
    else if (st->ev_b > 0) round = ORC_R_COMPLETE;
    else hold(T, T->zwork, st->ev_value);
  } else { /* local search */
    int done;
    if (mis) {
      if (st->ev_b > 0) { round = ORC_R_COMPLETE; done = 0; }
      else if (!(st->last_round == ORC_R_SWAP && st->last_commits == 0)) { round = ORC_R_SWAP; done = 0; }
      else done = 1;
    } else {
      if (st->ev_b > 0) { round = ORC_R_FLIP1; done = 0; }
      else if (!(st->last_round == ORC_R_FLIP2 && st->last_commits == 0)) { round = ORC_R_FLIP2; done = 0; }
      else done = 1;
    }
    if (done) hold(T, T->zwork, st->ev_value);
  }

  if (st->phase == ORC_PH_DESCENT) {
    int64_t ev[4];
    orc_descent_step(T->g, p, T->x, T->V, T->xn, T->Vn, T->zx_prev, ev);
    memcpy(T->x, T->xn, (size_t)n * sizeof(float));
    memcpy(T->V, T->Vn, (size_t)n * sizeof(float));
    st->ev_value = ev[0]; st->ev_a = ev[1]; st->ev_b = ev[2];
    st->s += 1;
    st->steps += 1;
    st->last_round = ORC_R_NONE;
    st->last_commits = 0;
  } else if (round != ORC_R_NONE) {
    int64_t k = run_round(T, round);
    disc_counts(T->g, p, T->zwork, st);
    st->last_round = round;
    st->last_commits = k;
  }
  /* a waiting trajectory does nothing this tick */
  st->ticks += 1;
}

static void set_best_all(orc_traj* T, int B, orc_pool* P, int64_t value, const uint8_t* bits, int from_ls) {
  P->best = value;
  for (int b = 0; b < B; ++b) {
    if (T[b].zbest != bits) memcpy(T[b].zbest, bits, (size_t)T[b].g->n);
    credit(T[b].st, value, from_ls);
    T[b].st->best = value;
    T[b].st->accepts += 1;
  }
}

/* The graph's step at the start of a tick, on the states left by the
 * previous tick.  Returns the decision and fills base[b] / ls[b]. */
static int pool_control(orc_traj* T, int B, orc_pool* P, uint8_t* pool_bits, int64_t* pool_vals, uint8_t* tmp,
                        const uint8_t* zero, const uint8_t** base, int* ls) {
  const orc_params* p = T[0].p;
  const int64_t n = T[0].g->n;
  const int K = p->pool_k;
  for (int b = 0; b < B; ++b) {
    base[b] = zero;
    ls[b] = 0;
    if (T[b].st->phase != ORC_PH_WAIT) return ORC_DEC_NONE;
  }
  if (P->epoch == ORC_EP_LS) {
    /* end of step 13: the best set takes the best search result */
    int win = -1;
    int64_t bv = P->best;
    for (int b = 0; b < B; ++b)
      if (T[b].st->held != INT64_MIN && T[b].st->held > bv) { bv = T[b].st->held; win = b; }
    if (win >= 0) {
      memcpy(tmp, T[win].zwork, (size_t)n);
      set_best_all(T, B, P, bv, tmp, 1);
    }
    P->epoch = ORC_EP_DESCENT;
    return ORC_DEC_OUTER;
  }
  /* steps 4 / 11: candidates = pool members (pool order), then the held
   * sets (trajectory order); stable selection of the K largest values */
  int nc = 0;
  int64_t* cv = malloc(sizeof(int64_t) * (size_t)(K + B));
  int* cs = malloc(sizeof(int) * (size_t)(K + B));
  for (int j = 0; j < P->count; ++j) { cv[nc] = pool_vals[j]; cs[nc] = j; ++nc; }
  for (int b = 0; b < B; ++b)
    if (T[b].st->held != INT64_MIN) { cv[nc] = T[b].st->held; cs[nc] = K + b; ++nc; }
  for (int i = 1; i < nc; ++i) { /* insertion sort, descending, stable */
    int64_t v = cv[i];
    int c = cs[i], j = i - 1;
    while (j >= 0 && cv[j] < v) { cv[j + 1] = cv[j]; cs[j + 1] = cs[j]; --j; }
    cv[j + 1] = v;
    cs[j + 1] = c;
  }
  int keep = nc < K ? nc : K;
  uint8_t* newbits = malloc((size_t)K * (size_t)n + 1);
  for (int s = 0; s < keep; ++s) {
    const uint8_t* src = cs[s] < K ? pool_bits + (size_t)cs[s] * (size_t)n : T[cs[s] - K].zwork;
    memcpy(newbits + (size_t)s * (size_t)n, src, (size_t)n);
  }
  memcpy(pool_bits, newbits, (size_t)keep * (size_t)n);
  for (int s = 0; s < keep; ++s) pool_vals[s] = cv[s];
  P->count = keep;
  P->merges += 1;
  free(newbits); free(cv); free(cs);
  /* steps 5 / 12 */
  if (P->count > 0 && pool_vals[0] > P->best) set_best_all(T, B, P, pool_vals[0], pool_bits, 0);
  const orc_state* s0 = T[0].st;
  if (s0->r < p->t_gs) {
    for (int b = 0; b < B; ++b) {
      int64_t k = orc_pool_pick(p->seed, T[b].traj, s0->o, s0->r + 1, P->count);
      base[b] = k >= 0 ? pool_bits + (size_t)k * (size_t)n : zero;
    }
    return ORC_DEC_NEXT;
  }
  if (p->local_search) {
    P->epoch = ORC_EP_LS;
    for (int b = 0; b < B; ++b) {
      if (p->problem == ORC_MIS) {
        ls[b] = b == 0;
        base[b] = T[0].zbest;
      } else {
        ls[b] = b < P->count;
        base[b] = b < P->count ? pool_bits + (size_t)b * (size_t)n : zero;
      }
    }
    return ORC_DEC_LS;
  }
  return ORC_DEC_OUTER;
}

/* Run the B trajectories traj0 .. traj0+B-1 of one graph in pool mode for
 * nticks ticks, from a fresh start or (resume) from the state passed in.
 * st: B states; x, V: B*n floats; zbest, zwork, zx_prev: B*n bytes;
 * pool_bits: K*n bytes; pool_vals: K values. */
ORC_API void orc_run_pool(const orc_graph* g, const orc_params* p, int64_t traj0, int32_t B, int64_t nticks,
                          int32_t resume, orc_state* st, float* x, float* V, uint8_t* zbest, uint8_t* zwork,
                          uint8_t* zx_prev, orc_pool* P, uint8_t* pool_bits, int64_t* pool_vals) {
  const int64_t n = g->n;
  orc_traj* T = calloc((size_t)B, sizeof(orc_traj));
  const uint8_t** base = calloc((size_t)B, sizeof(uint8_t*));
  int* ls = calloc((size_t)B, sizeof(int));
  uint8_t* zero = calloc((size_t)n + 1, 1);
  uint8_t* tmp = malloc((size_t)n + 1);
  for (int b = 0; b < B; ++b) {
    T[b].g = g; T[b].p = p; T[b].traj = traj0 + b; T[b].st = st + b;
    T[b].x = x + (size_t)b * (size_t)n; T[b].V = V + (size_t)b * (size_t)n;
    T[b].zbest = zbest + (size_t)b * (size_t)n; T[b].zwork = zwork + (size_t)b * (size_t)n;
    T[b].zx_prev = zx_prev + (size_t)b * (size_t)n;
    T[b].xn = malloc(((size_t)n + 1) * sizeof(float));
    T[b].Vn = malloc(((size_t)n + 1) * sizeof(float));
    T[b].in_r = malloc((size_t)n + 1);
    if (!resume) {
      orc_state_init(T[b].st);
      orc_init_x(g, p, T[b].traj, 0, T[b].x);
      for (int64_t v = 0; v < n; ++v) { T[b].V[v] = 0.0f; T[b].zbest[v] = 0; T[b].zwork[v] = 0; T[b].zx_prev[v] = 0; }
    }
  }
  if (!resume) {
    P->epoch = ORC_EP_DESCENT;
    P->count = 0;
    P->best = INT64_MIN;
    P->merges = 0;
  }
  for (int64_t t = 0; t < nticks; ++t) {
    int dec = pool_control(T, B, P, pool_bits, pool_vals, tmp, zero, base, ls);
    for (int b = 0; b < B; ++b) tick_pool(&T[b], dec, base[b], ls[b]);
  }
  for (int b = 0; b < B; ++b) { free(T[b].xn); free(T[b].Vn); free(T[b].in_r); }
  free(T); free(base); free(ls); free(zero); free(tmp);
}

/* ------------------------------------------------------------------ */
/* Relaxed objectives in double precision (Eq. 3, Eq. 7) and the f_B  */
/* gradient -lambda 1 - 2 A x.                                         */
/* ------------------------------------------------------------------ */
ORC_API double orc_objective_f64(const orc_graph* g, int32_t problem, double gamma, double lambda_, const double* x) {
  double lin = 0.0, quad = 0.0;
  for (int64_t v = 0; v < g->n; ++v) {
    double ax = 0.0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) ax += (double)wt(g, j) * x[g->col[j]];
    lin += x[v];
    quad += x[v] * ax;
  }
  if (problem == ORC_MIS) return lin - 0.5 * gamma * quad;
  return -lambda_ * lin - quad;
}

/* The four MaxCut relaxations of Sec. 3 in double precision, written from
 * their definitions: f_L = 1/4 x'Lx (on {-1,1}^n equal to 1/2 sum over
 * undirected edges of w(1 - x_u x_v), the cut), f_P = x'(L + lambda I)x,
 * f_A = -x'Ax, f_B = -lambda 1'x - x'Ax, with L = D - A; and their
 * gradients (derived: 1/2 Lx, 2(L + lambda I)x, -2Ax, -lambda 1 - 2Ax). */
ORC_API double orc_cut_objective_f64(const orc_graph* g, int32_t objective, double lambda_, const double* x) {
  double xax = 0.0, xdx = 0.0, xx = 0.0, lin = 0.0;
  for (int64_t v = 0; v < g->n; ++v) {
    double d = 0.0, ax = 0.0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      const double w = (double)wt(g, j);
      d += w;
      ax += w * x[g->col[j]];
    }
    xax += x[v] * ax;
    xdx += d * x[v] * x[v];
    xx += x[v] * x[v];
    lin += x[v];
  }
  switch (objective) {
    case ORC_F_L: return 0.25 * (xdx - xax);
    case ORC_F_P: return (xdx - xax) + lambda_ * xx;
    case ORC_F_A: return -xax;
    default: return -lambda_ * lin - xax;
  }
}

ORC_API void orc_cut_gradient_f64(const orc_graph* g, int32_t objective, double lambda_, const double* x,
                                  double* grad) {
  for (int64_t v = 0; v < g->n; ++v) {
    double d = 0.0, ax = 0.0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      d += (double)wt(g, j);
      ax += (double)wt(g, j) * x[g->col[j]];
    }
    switch (objective) {
      case ORC_F_L: grad[v] = 0.5 * (d * x[v] - ax); break;
      case ORC_F_P: grad[v] = 2.0 * (d * x[v] - ax + lambda_ * x[v]); break;
      case ORC_F_A: grad[v] = -2.0 * ax; break;
      default: grad[v] = -lambda_ - 2.0 * ax; break;
    }
  }
}

ORC_API void orc_gradient_f64(const orc_graph* g, int32_t problem, double gamma, double lambda_, const double* x,
                              double* grad) {
  for (int64_t v = 0; v < g->n; ++v) {
    double ax = 0.0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) ax += (double)wt(g, j) * x[g->col[j]];
    grad[v] = problem == ORC_MIS ? 1.0 - gamma * ax : -lambda_ - 2.0 * ax;
  }
}

/* ------------------------------------------------------------------ */
/* Brute force over all 2^n binary points (n <= 26): optimum of the     */
/* MIS ILP and of the cut ILP, for pinning.                             */
/* ------------------------------------------------------------------ */
ORC_API int64_t orc_brute_mis(const orc_graph* g) {
  int64_t n = g->n, best = 0;
  uint64_t* nb = calloc((size_t)n + 1, sizeof(uint64_t));
  for (int64_t v = 0; v < n; ++v)
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) nb[v] |= 1ULL << g->col[j];
  for (uint64_t s = 0; s < (1ULL << n); ++s) {
    int ok = 1;
    for (int64_t v = 0; v < n && ok; ++v) if (((s >> v) & 1ULL) && (nb[v] & s)) ok = 0;
    if (ok) {
      int64_t c = __builtin_popcountll(s);
      if (c > best) best = c;
    }
  }
  free(nb);
  return best;
}

ORC_API int64_t orc_brute_maxcut(const orc_graph* g) {
  int64_t n = g->n, best = INT64_MIN;
  for (uint64_t s = 0; s < (1ULL << n); ++s) {
    int64_t c2 = 0;
    for (int64_t v = 0; v < n; ++v)
      for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j)
        if (((s >> v) & 1ULL) != ((s >> g->col[j]) & 1ULL)) c2 += wt(g, j);
    if (c2 / 2 > best) best = c2 / 2;
  }
  return best;
}
