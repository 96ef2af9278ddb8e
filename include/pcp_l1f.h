/*
 * pcp_l1f.h -- C ABI of the GB300 (sm_103a) l1-filtering PCP library.
 *
 * Principal Component Pursuit (Eq. PCP): given M (m x n) find L (low rank)
 * and S (sparse) with M = L + S minimising ||L||_* + lambda ||S||_1.  The
 * l1 filtering method (Algorithm 2) solves it in four stages:
 *   1. sample a seed submatrix M^s = M[I_s, J_s] of (s_r r) x (s_c r)
 *      entries (Section 3.1);
 *   2. solve the small PCP of Eq. SPCP on M^s (here: inexact ALM in FP64 on
 *      the device) and keep its skinny SVD L^s = U^s Sigma^s V^sT;
 *   3. l1 filtering (Section 3.2, Algorithm 1): every column of
 *      M^c = M[I_s, ~J_s] is an l1 regression on U^s (Eq. l1c') and every
 *      row of M^r = M[~I_s, J_s] an l1 regression on V^s (Eq. l1r');
 *   4. represent the rest by the generalized Nystrom formula
 *      L~^s = P~^T (Sigma^s)^{-1} Q~ (Eq. l1s') and output S = M - L.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major (Fortran/BLAS order) with an explicit leading
 *     dimension >= the row count.  Indices are 0-based.
 *   - "d" pointers are device pointers (cudaMalloc / torch CUDA tensors) and
 *     "h" pointers host pointers.  The caller owns every buffer it passes;
 *     the library never frees or retains them past the call except where a
 *     function says so.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; unless stated, calls are
 *     asynchronous with respect to the host.
 *   - Errors are returned as pcp_status; nothing aborts or traps.  The
 *     message of the last error on the calling thread is available from
 *     pcp_last_error().  On an error no output is guaranteed.
 *   - Floating point: M, S and the L factors are FP32.  The seed PCP keeps
 *     its ALM state (S, Y, G), the Ritz values and the final skinny SVD of
 *     L^s in FP64 (U^s, V^s orthonormal to FP64 rounding); inside the ALM
 *     the k x k Cholesky and Jacobi steps are FP32 and, while the residual
 *     is above 1e-6, so are the tall and rank-k products.
 */
#ifndef PCP_L1F_H
#define PCP_L1F_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pcp_status {
  PCP_OK = 0,
  PCP_ERR_ARG = -1,           /* invalid argument (size, pointer, index set) */
  PCP_ERR_NOMEM = -2,         /* device or pinned-host allocation failed */
  PCP_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  PCP_ERR_NONFINITE = -4,     /* NaN or Inf found in the seed block of M */
  PCP_ERR_RANK_TEST = -5,     /* Eq. rank_test failed: m'/r' < s_r or
                                 n'/r' < s_c, or r' = 0; results written */
  PCP_ERR_SEED_NOCONV = -6,   /* seed PCP hit seed_max_iter; results written */
  PCP_ERR_FILTER_NOCONV = -7, /* some l1 problems hit filter_max_iter;
                                 results written, see pcp_info */
  PCP_ERR_BUSY = -8,          /* serving: request still in flight */
  PCP_ERR_TIMEOUT = -9,       /* a bounded device wait ran out */
  PCP_ERR_CANCELLED = -10,    /* serving: request dropped at shutdown */
  PCP_ERR_UNSUPPORTED = -11   /* option not available on this device */
} pcp_status;

/* Arithmetic of Algorithm 1 (the seed PCP is the same in every mode). */
typedef enum pcp_precision {
  PCP_FP32 = 0,          /* FP32-accurate, kernel chosen by the library:
                            split-TF32 tensor-core products (three passes,
                            ~2^-21 relative), or, where both kernels take
                            the shape (p <= 256, r <= 32), the SIMT FP32
                            kernel where the compiled-in tuning table says
                            it is faster (pcp_l1_filter_kernel) */
  PCP_BF16_REFINED = 1,  /* one-pass BF16 tensor-core products (inputs
                            rounded to BF16, FP32 accumulation) for the
                            first lowp_iters iterations, then split-TF32
                            products until filter_tol, as below */
  PCP_TF32_REFINED = 2,  /* one-pass TF32 tensor-core products with FP32
                            accumulation for the first lowp_iters
                            iterations, then split-TF32 products (three
                            passes, ~2^-21 relative, the FP32 refinement)
                            until filter_tol */
  PCP_FP64 = 3,          /* reserved: PCP_ERR_UNSUPPORTED */
  PCP_FP32_TENSOR = 4,   /* split-TF32 tensor-core products, always */
  PCP_FP32_SIMT = 5      /* FP32 FMA on the CUDA cores (p <= 256, r <= 32) */
} pcp_precision;

/* Parameters of one solve.  Fill with pcp_params_default() first. */
typedef struct pcp_params {
  int64_t m, n;             /* size of M */
  int32_t r;                /* target rank; sizes the seed (Section 3.1) */
  int32_t precision;        /* pcp_precision */
  double lambda;            /* full-problem lambda of Eq. PCP; <= 0 means
                               1/sqrt(max(m,n)).  Reported only: the
                               filtering stage has no lambda. */
  double lambda_seed;       /* lambda~ of Eq. SPCP; <= 0 means
                               1/sqrt(max(m',n')) */
  double s_r, s_c;          /* oversampling rates, default 10 (Section 3.1);
                               m' = round(s_r r), n' = round(s_c r) */
  double seed_tol;          /* ||M^s-L^s-S^s||_F/||M^s||_F stop, default 1e-7
                               (Section 4.1.1) */
  double seed_rho;          /* ALM penalty growth, default 1.5 */
  double seed_mu_scale;     /* mu_0 = seed_mu_scale/||M^s||_2, default 1.25 */
  double seed_mu_max_ratio; /* mu_max = ratio * mu_0, default 1e7 */
  double rank_cut;          /* singular values of L^s below rank_cut * the
                               largest are dropped, default 1e-6 (the seed is
                               resolved only to ~1e-7 of its norm) */
  double filter_tol;        /* epsilon of Algorithm 1's stop test (see
                               pcp_l1_filter), default 3e-6 */
  double filter_rho;        /* rho of Algorithm 1, default 1.5 */
  double beta0_scale;       /* beta_0 = beta0_scale/||x||_inf, default 1 */
  double beta_bar_ratio;    /* beta_bar = ratio * beta_0, default 1e10 */
  int32_t seed_max_iter;    /* default 500 */
  int32_t filter_max_iter;  /* default 500 */
  int32_t seed_subspace;    /* initial subspace size of the seed's partial
                               SVD; <= 0 means r + max(6, r/4), rounded up to
                               even */
  int32_t lowp_iters;       /* PCP_TF32_REFINED: Algorithm 1 iterations with
                               one-pass TF32 products before the FP32-
                               accurate refinement, default 12 */
  uint64_t rng_seed;        /* seed sampling when seed_rows/cols are NULL */
  const int64_t* seed_rows; /* optional host array, m' distinct row indices */
  const int64_t* seed_cols; /* optional host array, n' distinct col indices */
  const int64_t* row_order; /* optional host array, a permutation of 0..m-1:
                               the seed rows are its first m' entries
                               (sorted); excludes seed_rows */
  const int64_t* col_order; /* same for the columns; excludes seed_cols */
  int32_t seed_m, seed_n;   /* > 0: seed size m', n' instead of s_r r, s_c r */
  int32_t grow_seed;        /* 1: on a failed Eq. rank_test, grow the seed to
                               (s_r r') x (s_c r') and solve again, until the
                               test holds or the seed would pass half of a
                               side (Section 3.5); needs seeds taken by order
                               (row_order / col_order or the library's own
                               sampling, not seed_rows / seed_cols) and a
                               pcp_info for the solve */
  int32_t seed_ctas;        /* team of the seed PCP: 1..16 = one thread-
                               block cluster of that many CTAs (hardware
                               cluster barrier; the grid form below when the
                               device cannot hold it), more = a cooperative
                               grid of that many CTAs (software grid barrier,
                               up to the co-resident limit), 0 = the
                               library's choice (a cluster of 16 for seeds
                               up to 64 x 64, else the grid).  The result
                               does not depend on it (fixed partial-sum
                               slots). */
  int64_t wait_timeout_ns;  /* limit of each bounded device wait of the seed
                               stage (its grid barrier), in ns; <= 0 means
                               2 s.  A wait that runs out ends the seed
                               kernel on every CTA and the solve returns
                               PCP_ERR_TIMEOUT (the device stays usable). */
} pcp_params;

/* Diagnostics of one solve. */
typedef struct pcp_info {
  int32_t rank;             /* r' = numerical rank of L^s kept (<= r) */
  int32_t rank_ok;          /* 1 if Eq. rank_test holds */
  int32_t seed_iters;       /* ALM iterations of the seed PCP */
  int32_t filter_iters_max; /* most Algorithm 1 iterations of any problem */
  int64_t seed_m, seed_n;   /* m', n' */
  int64_t problems;         /* (n - n') column + (m - m') row problems */
  int64_t problems_unconverged;
  double seed_residual;     /* final ||M^s-L^s-S^s||_F/||M^s||_F */
  double lambda;            /* full-problem lambda used/reported */
  float t_seed_ms;          /* gather + seed PCP + factor assembly */
  float t_filter_ms;        /* column and row filtering */
  float t_spass_ms;         /* S = M - L */
  float t_total_ms;         /* whole solve (batched and served forms: the
                               batch / request end to end) */
  int32_t status;           /* pcp_status of this solve */
  int32_t seed_rank_raw;    /* rank of L^s before the cap at r (Eq.
                               rank_test uses it) */
  double filter_iters_mean; /* mean Algorithm 1 iterations per problem */
  int32_t filter_kernel;    /* Algorithm 1 kernel of the column filter
                               (PCP_KERNEL_SIMT or PCP_KERNEL_TENSOR); the
                               row filter's is pcp_l1_filter_kernel(n', r,
                               precision) */
  int32_t launches;         /* kernels this call launched on the device
                               (every stage, seed growth included) */
  int32_t seed_team;        /* the seed PCP's team of CTAs: c > 0 for one
                               thread-block cluster of c CTAs, -g for a
                               cooperative grid of g CTAs */
  int32_t pad_info;
} pcp_info;

/* One instance of a batched or served solve: its parameters and buffers
 * (same meaning and layout as the arguments of pcp_l1filter_solve). */
typedef struct pcp_problem {
  pcp_params params;
  const float* dM;
  int64_t ldm;
  float* dLu;
  float* dLv;
  float* dS; /* may be NULL */
  int64_t lds;
} pcp_problem;

typedef struct pcp_plan pcp_plan;

/* Fill *p with the defaults listed above for an m x n problem of target
 * rank r.  Returns PCP_ERR_ARG if p is NULL. */
pcp_status pcp_params_default(pcp_params* p, int64_t m, int64_t n, int32_t r);

/* Human-readable message of the last error on the calling thread. */
const char* pcp_last_error(void);

/* Library version string. */
const char* pcp_version(void);

/* ------------------------------------------------------------------------
 * Whole solve (Algorithm 2).
 * ---------------------------------------------------------------------- */

/* Validate *params and allocate the device workspace for problems of that
 * size (seed buffers, index sets, per-problem status).  The plan copies
 * *params (and the optional seed index arrays) and owns its workspace until
 * pcp_plan_destroy().  One plan serves any number of sequential solves of
 * the same shape; concurrent solves need separate plans.  Limits: r <= 64,
 * seeds up to 512 x 512 and smaller than M in both sides (PCP_ERR_ARG). */
pcp_status pcp_l1filter_plan(const pcp_params* params, pcp_plan** out);

/* Run Algorithm 2 on M.
 *   dM  (m x n, ldm >= m), FP32, read only.
 *   dLu (m x r, ld m) and dLv (n x r, ld n), FP32, written: the factored
 *       low-rank part with W = (Sigma^s)^{-1} folded in, L = Lu * Lv^T:
 *         Lu[I_s]  = U^s,               Lu[~I_s] = P~^T (Sigma^s)^{-1},
 *         Lv[J_s]  = V^s Sigma^s,       Lv[~J_s] = Q~^T,
 *       columns r'..r-1 zero when the seed rank r' < r.
 *   dS  (m x n, lds >= m), FP32, written with S = M - Lu Lv^T.  May be NULL
 *       to skip the S pass (factors only).
 *   h_seed_rows_out / h_seed_cols_out: optional host arrays of m' / n'
 *       entries receiving I_s and J_s (with grow_seed: room for
 *       min(512, m/2) / min(512, n/2) entries; info->seed_m / seed_n give
 *       the sizes of the seed the solve ended with).
 *   info: optional.  When non-NULL the call synchronises the stream and
 *       fills *info (stage times by CUDA events); when NULL the call is
 *       asynchronous except for the seed index upload.
 * Returns PCP_ERR_RANK_TEST / PCP_ERR_SEED_NOCONV / PCP_ERR_FILTER_NOCONV
 * only when info is non-NULL (the checks need the device results). */
pcp_status pcp_l1filter_solve(pcp_plan* plan, const float* dM, int64_t ldm,
                              float* dLu, float* dLv, float* dS, int64_t lds,
                              int64_t* h_seed_rows_out,
                              int64_t* h_seed_cols_out, pcp_info* info,
                              void* stream);

/* pcp_l1filter_solve (Algorithm 2) on host buffers, with the copies
 * overlapped with the compute.  hM (m x n, ldm >= m) is host memory; page-locked memory
 * (cudaHostAlloc / cudaHostRegister) is read in place by the seed gather so
 * the seed starts while M is still being copied, and the copies run
 * asynchronously; pageable memory works with the copies serialised.
 * hLu (m x r, ld m), hLv (n x r, ld n) and hS (m x n, lds >= m; NULL to
 * skip S) receive the results: the factors while the S pass runs, S in
 * column chunks while the next chunk is computed.  The plan keeps device
 * copies of M, S and the factors (allocated on the first call, freed by
 * pcp_plan_destroy) and a copy stream; successive calls on one stream reuse
 * them in order.  info and the status codes as for pcp_l1filter_solve
 * (with info, t_spass_ms includes the last copies of S).  Without info the
 * call returns before the copies finish: synchronise `stream` before
 * reading the outputs or reusing hM. */
pcp_status pcp_l1filter_solve_host(pcp_plan* plan, const float* hM,
                                   int64_t ldm, float* hLu, float* hLv,
                                   float* hS, int64_t lds, pcp_info* info,
                                   void* stream);

/* Asynchronous solves (info == NULL, either call above) run as a CUDA graph:
 * the first call on a plan runs directly, the second with the same buffers
 * (device pointers and leading dimensions, or host pointers) is captured
 * into a graph of its launches and copies and later calls with the same
 * buffers replay it on `stream`; other buffers are captured anew.  A solve
 * that cannot be captured runs directly and graphs stay off for that plan.
 * Returns the number of graph launches so far, or -1 when graphs are off. */
int64_t pcp_plan_graph_launches(const pcp_plan* plan);

void pcp_plan_destroy(pcp_plan* plan);

/* Batched form of Algorithm 2 (Section 3.2: the column and row problems of
 * every instance are independent): `count` independent instances of any
 * sizes, each stage one launch over all of them (batched gather; all seed
 * PCPs in one launch, side by side: a large seed on a team of CTAs, the
 * others one CTA each; batched factor assembly; one Algorithm 1 launch per
 * kernel shape over every instance's column and row problems), then the S
 * pass per instance.  Every parameter is per instance, and an instance's
 * result does not depend on the other instances of the batch (a seed sums
 * its partials in the same fixed slots on any team); its rounding differs
 * from pcp_l1filter_solve's (whole-GPU seed, more slots) by reduction
 * order only.  Workspace is stream-ordered (cudaMallocAsync /
 * cudaFreeAsync on `stream`); the caller's buffers must stay valid until
 * the stream reaches the end of the batch.  With infos (count entries) the
 * call synchronises and fills one pcp_info per instance, including its
 * status; the return value is then the first non-OK status.  With infos,
 * an instance with grow_seed whose seed fails Eq. rank_test grows (Section
 * 3.5) and runs again, until none grows; its first round's filters are
 * skipped on the device, so only the last round writes its outputs.
 * Without infos the call is asynchronous and nothing grows.  Limits: count
 * <= 65535, r <= 64, seeds up to 512 x 512; violations give PCP_ERR_ARG
 * before any device work. */
pcp_status pcp_l1filter_batch(int32_t count, const pcp_problem* probs,
                              pcp_info* infos, void* stream);

/* Batch plans: pcp_l1filter_batch with its workspace allocated once and its
 * launches (batched gather, seed teams, assembly, one Algorithm 1 launch
 * per kernel shape over every instance's problems, diagnostics, S passes)
 * captured into a CUDA graph that each run replays.
 *
 * pcp_l1filter_batch_plan runs the batch once directly (on `stream`,
 * synchronising it; instances with grow_seed settle their seed size as
 * Section 3.5 says), then fixes every instance's seed at the size it ended
 * with, allocates the workspace (cudaMalloc), uploads the index sets and
 * captures the launches.  The plan copies the pcp_problem array and the
 * host index arrays it points to; the device buffers (dM, dLu, dLv, dS)
 * must stay valid for the plan's lifetime, and each run reads M and writes
 * the outputs again.  PCP_ERR_ARG / PCP_ERR_CUDA / PCP_ERR_NOMEM on
 * failure (no plan); a per-instance status such as PCP_ERR_RANK_TEST does
 * not stop the plan (that instance keeps its last seed).
 *
 * pcp_l1filter_batch_run replays the graph on `stream`.  Without infos the
 * call is asynchronous; with infos (count entries) it synchronises and
 * fills one pcp_info per instance (t_total_ms = the replay; stage times 0)
 * and returns the first non-OK status.  Runs of one plan must not overlap
 * on the GPU (they share its workspace); different plans may. */
typedef struct pcp_batch_plan pcp_batch_plan;
pcp_status pcp_l1filter_batch_plan(int32_t count, const pcp_problem* probs,
                                   void* stream, pcp_batch_plan** out);
pcp_status pcp_l1filter_batch_run(pcp_batch_plan* plan, pcp_info* infos,
                                  void* stream);
void pcp_batch_plan_destroy(pcp_batch_plan* plan);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of independent solves (no counterpart in
 * the paper, which solves one matrix at a time; built on the batched form).
 *
 * A server owns a scheduler thread and `streams` CUDA streams on the device
 * current at creation.  pcp_serve_submit queues a request and returns at
 * once with a ticket.  The scheduler admits queued requests in arrival
 * order while their summed device workspace stays within hbm_budget_bytes
 * and at most max_slots requests are in flight, launches each admitted
 * group as one batched solve on a free stream, and keeps admitting while
 * earlier groups run, so requests that arrive during a solve join the next
 * group instead of waiting for the device to drain.  A request whose
 * workspace alone exceeds the budget completes with PCP_ERR_NOMEM.  The
 * result of a request does not depend on which other requests share its
 * group.  A request with grow_seed whose seed fails Eq. rank_test (its
 * filters skipped on the device) goes back to the head of the queue with
 * the grown seed (Section 3.5) and completes when a seed passes or the
 * growth gives up.  The caller's buffers (pcp_problem pointers) must stay
 * valid and untouched until the request completes; the optional seed index
 * arrays are copied at submission.
 * ---------------------------------------------------------------------- */
typedef struct pcp_server pcp_server;

/* Create a server.  hbm_budget_bytes > 0; max_slots >= 1;
 * 1 <= streams <= 16.  PCP_ERR_ARG on bad arguments, PCP_ERR_CUDA if a
 * stream cannot be created. */
pcp_status pcp_serve_create(size_t hbm_budget_bytes, int32_t max_slots,
                            int32_t streams, pcp_server** out);

/* Queue one request (validated now: PCP_ERR_ARG before queueing on bad
 * sizes or pointers).  *ticket receives its id.  PCP_ERR_CANCELLED once
 * pcp_serve_destroy has begun. */
pcp_status pcp_serve_submit(pcp_server* server, const pcp_problem* prob,
                            uint64_t* ticket);

/* Non-blocking: PCP_ERR_BUSY while the request is queued or running;
 * otherwise the request's own status, *info filled (if non-NULL; its
 * t_total_ms is submission to completion), and the ticket is released.
 * PCP_ERR_ARG for an unknown or already released ticket. */
pcp_status pcp_serve_poll(pcp_server* server, uint64_t ticket,
                          pcp_info* info);

/* Blocking form of pcp_serve_poll. */
pcp_status pcp_serve_wait(pcp_server* server, uint64_t ticket,
                          pcp_info* info);

/* Stop admitting: requests not yet launched complete with
 * PCP_ERR_CANCELLED, running groups are finished and the scheduler thread
 * is joined.  Every ticket stays pollable afterwards; later submissions
 * return PCP_ERR_CANCELLED.  Idempotent. */
pcp_status pcp_serve_stop(pcp_server* server);

/* pcp_serve_stop, then release the server (its streams and any results
 * never polled).  No other call on this server may be in progress or made
 * afterwards.  NULL is accepted. */
pcp_status pcp_serve_destroy(pcp_server* server);

/* ------------------------------------------------------------------------
 * Stage entry points (the rows of the hot path, callable one by one).
 * Index arrays are device int32 arrays.
 * ---------------------------------------------------------------------- */

/* Stage 1 gather (Eq. partition): dMs[i + j*mp] = (double) dM[rows[i] +
 * cols[j]*ldm] for i < mp, j < np.  Returns PCP_ERR_ARG on bad sizes. */
pcp_status pcp_gather_seed(const float* dM, int64_t ldm, const int32_t* d_rows,
                           int32_t mp, const int32_t* d_cols, int32_t np,
                           double* dMs, void* stream);

/* Bytes of device workspace pcp_seed_pcp needs for an mp x np seed whose
 * partial SVD may grow to kmax vectors (kmax <= min(mp, np), kmax <= 128). */
size_t pcp_seed_workspace_bytes(int32_t mp, int32_t np, int32_t kmax);

/* Stage 2: seed PCP (Eq. SPCP) by inexact ALM in FP64 with a partial SVD
 * for the singular value thresholding (Eq. SVT), one persistent cooperative
 * launch.  dD is mp x np (ld mp), FP64, read only.  On return (the call
 * synchronises `stream`):
 *   dU (mp x kmax, ld mp), dSigma (kmax), dV (np x kmax, ld np): the skinny
 *   SVD of the recovered L^s, columns sorted by decreasing singular value,
 *   entries past *h_rank zero;  *h_rank = r' (singular values above
 *   rank_cut * largest, capped at r_cap when r_cap > 0);
 *   *h_iters, *h_residual: ALM iterations and final relative residual.
 * lambda <= 0 means 1/sqrt(max(mp,np)).  k0 is the initial subspace size
 * (even, <= kmax); kmax is even, <= 64 and <= min(mp, np); 2 <= mp, np <=
 * 512.  The SVT equals the full-SVD one while the subspace holds every
 * singular value above 1/mu; a subspace started below the SVT's rank cuts
 * it until it grows (another ALM path).  d_work must hold
 * pcp_seed_workspace_bytes() bytes.
 * Returns PCP_ERR_SEED_NOCONV when max_iter is reached (outputs written),
 * PCP_ERR_TIMEOUT if a device barrier wait ran out. */
pcp_status pcp_seed_pcp(const double* dD, int32_t mp, int32_t np,
                        double lambda, double tol, double rho,
                        double mu_scale, double mu_max_ratio, int32_t max_iter,
                        int32_t k0, int32_t kmax, double rank_cut,
                        int32_t r_cap, void* d_work, double* dU,
                        double* dSigma, double* dV, int32_t* h_rank,
                        int32_t* h_iters, double* h_residual, void* stream);

/* Allocation-free seed PCP (the paper has no counterpart; this is a
 * deployment convenience).  Same arguments, results and errors as
 * pcp_seed_pcp, without d_work: the workspace is a fixed 3 MiB array in
 * device memory owned by the library, for callers that cannot call
 * cudaMalloc (host frameworks that give out all device memory from their own
 * pool, latency-bound loops that cannot afford cudaMalloc's implicit device
 * synchronisation, processes whose memory budget is committed up front).
 *   - Limit: seeds whose pcp_seed_workspace_bytes(mp, np, kmax) is at most
 *     3 MiB (e.g. 200 x 200 with kmax = 52; not 256 x 256 with kmax = 64);
 *     larger sizes return PCP_ERR_ARG with the byte counts in the message.
 *   - Every GPU that loads the library holds the array until process exit.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device); make that first call before
 *     any stream capture.
 *   - All calls share the array: calls whose work overlaps on the GPU (other
 *     streams, other threads) race and must be serialised by the caller.
 *     Each call clears the control words it relies on, so the contents left
 *     by the previous call do no harm. */
pcp_status pcp_seed_pcp_static(const double* dD, int32_t mp, int32_t np,
                               double lambda, double tol, double rho,
                               double mu_scale, double mu_max_ratio,
                               int32_t max_iter, int32_t k0, int32_t kmax,
                               double rank_cut, int32_t r_cap, double* dU,
                               double* dSigma, double* dV, int32_t* h_rank,
                               int32_t* h_iters, double* h_residual,
                               void* stream);

/* Tracing of the seed stage: copy block 0's phase records of the last seed
 * solve that ran in d_work (pcp_seed_pcp's workspace) into h_out, up to
 * `cap` records of two uint64 each: (globaltimer ns, phase code).  Phase
 * codes: 1 prologue norms, 2 T = G^T Omega, 3 Gram of T, 4 Cholesky QR of T,
 * 5 P = G Psi, 6 Gram of P, 7 power-step orthonormalisation, 8 Jacobi
 * eigen-solve, 9 rotation to Ritz vectors, 10 ALM start, 11 ALM update,
 * 12 set-up of the eigen-solve, 13 / 14 FP64 refinement of the Ritz basis
 * (Gram, rotation), 15 the final FP64 skinny SVD of L^s.
 * Synchronises `stream`.  Returns the number of records, -1 on error. */
int32_t pcp_seed_trace(const void* d_work, int32_t mp, int32_t np,
                       int32_t kmax, uint64_t* h_out, int32_t cap,
                       void* stream);

/* Same for the seed stage of the last pcp_l1filter_solve on this plan. */
int32_t pcp_plan_seed_trace(const pcp_plan* plan, uint64_t* h_out,
                            int32_t cap, void* stream);

/* Stage 3/4: Algorithm 1 on N independent problems (columns or rows of M),
 * FP32.  Problem j reads its p entries x_j[t] = dM[pidx[t]*sp + qidx[j]*sq]
 * (column problems: pidx = I_s, sp = 1, qidx = ~J_s, sq = ldm; row problems:
 * pidx = J_s, sp = ldm, qidx = ~I_s, sq = 1) and is regressed on
 * dA (p x r, ld lda, FP32, orthonormal columns).  The solution z_j is
 * written as dZ[qidx[j] + k*ldz] = z_j[k] * (d_scale ? d_scale[k] : 1) for
 * k < r (so the result lands directly in a row of Lv or Lu).  The rank is
 * read from *d_rank when d_rank is non-NULL (device int32, <= r; columns
 * past it are written as zero).  d_iters (N int32, optional) receives each
 * problem's iteration count, negated when it hit max_iter.
 * precision: PCP_FP32 / PCP_FP32_TENSOR (split TF32), PCP_TF32_REFINED
 * (lowp_iters one-pass TF32 iterations, then split TF32 until eps) or
 * PCP_FP32_SIMT; the stop test is only taken on FP32-accurate iterations.
 * Stop test (FP32 reading of Algorithm 1's): a problem stops when
 * ||x - A z - e||_inf < eps * max(||x - e||_inf, 1e-3 ||x||_inf); the paper
 * divides by ||x||_inf, which lets the fit of x - e be as loose as
 * eps times the largest outlier.
 * Limits: p <= 512, r <= 64 (PCP_FP32_SIMT: p <= 256, r <= 32). */
pcp_status pcp_l1_filter(const float* dM, const int32_t* d_pidx, int32_t p,
                         int64_t sp, const int32_t* d_qidx, int32_t N,
                         int64_t sq, const float* dA, int32_t lda, int32_t r,
                         const int32_t* d_rank, const float* d_scale,
                         float* dZ, int64_t ldz, double eps, double rho,
                         double beta0_scale, double beta_bar_ratio,
                         int32_t max_iter, int32_t precision,
                         int32_t lowp_iters, int32_t* d_iters,
                         void* stream);

/* Algorithm 1 kernels (pcp_info.filter_kernel, pcp_l1_filter_kernel). */
enum {
  PCP_KERNEL_SIMT = 1,   /* adm_f32_kernel: FP32 FMA on the CUDA cores */
  PCP_KERNEL_TENSOR = 2  /* adm_tc_kernel: mma.sync tensor-core products */
};

/* The Algorithm 1 kernel pcp_l1_filter (and every solve) runs for problems
 * of length p, rank r and the given precision: PCP_KERNEL_SIMT or
 * PCP_KERNEL_TENSOR, or PCP_ERR_ARG for sizes or a precision it refuses.
 * For PCP_FP32 the choice is fixed per (p, r) class by a table compiled
 * into the library (written by a committed tuning run that timed both
 * kernels on GB300), so the same inputs give the same bits in every
 * process; the batched and served forms use the same table. */
int32_t pcp_l1_filter_kernel(int32_t p, int32_t r, int32_t precision);

/* Stage 5: factor assembly (Eq. l1s').  From the seed's FP64 skinny SVD
 * (dU mp x ku ld mp, dSigma, dV np x ku ld np, rank *d_rank) write
 *   Lu[rows[i] + k*ldu] = U[i,k],  Lv[cols[j] + k*ldv] = V[j,k]*sigma_k,
 * the FP32 copies dU32 (mp x r, ld mp) and dV32 (np x r, ld np) used as A by
 * the filters, and d_inv_sigma32[k] = 1/sigma_k (0 past the rank), for
 * k < r.  Columns k >= rank of Lu/Lv rows outside the seed are zeroed by the
 * filters; rows inside the seed are written here. */
pcp_status pcp_assemble_factors(const double* dU, const double* dSigma,
                                const double* dV, int32_t mp, int32_t np,
                                int32_t ku, const int32_t* d_rank, int32_t r,
                                const int32_t* d_rows, const int32_t* d_cols,
                                float* dLu, int64_t ldu, float* dLv,
                                int64_t ldv, float* dU32, float* dV32,
                                float* d_inv_sigma32, void* stream);

/* Stage 6, the S pass (Algorithm 2 output): dS = dM - dLu * dLv^T over the
 * full m x n matrix, FP32, with dLu m x r (ld ldu) and dLv n x r (ld ldv).
 * dS may alias dM only if lds == ldm (in-place update).  Same as
 * pcp_spass_impl(..., PCP_SPASS_AUTO, stream). */
pcp_status pcp_spass(const float* dM, int64_t ldm, const float* dLu,
                     int64_t ldu, const float* dLv, int64_t ldv, int32_t r,
                     float* dS, int64_t lds, int64_t m, int64_t n,
                     void* stream);

/* S-pass kernels.  PCP_SPASS_TENSOR: tcgen05 tensor cores (split TF32, FP32
 * accumulation, ~2^-21 relative error per product) with TMA tiles of M and
 * S; needs 1 <= r <= 64, m >= 128, n >= 64, dM and dS 16-byte aligned and
 * ldm, lds multiples of 4, else PCP_ERR_UNSUPPORTED.  PCP_SPASS_SIMT: FP32
 * FMA, any shape.  PCP_SPASS_AUTO: the tensor form where it applies. */
enum {
  PCP_SPASS_AUTO = 0,
  PCP_SPASS_SIMT = 1,
  PCP_SPASS_TENSOR = 2
};
pcp_status pcp_spass_impl(const float* dM, int64_t ldm, const float* dLu,
                          int64_t ldu, const float* dLv, int64_t ldv,
                          int32_t r, float* dS, int64_t lds, int64_t m,
                          int64_t n, int32_t impl, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCP_L1F_H */
