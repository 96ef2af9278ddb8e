// Host side of the C ABI: parameters, plans, the whole solve (Algorithm 2),
// error reporting and seed sampling.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace pcp {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

pcp_status cuda_fail(cudaError_t e, const char* what, const char* file,
                     int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) return PCP_ERR_NOMEM;
  return PCP_ERR_CUDA;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
      cudaSuccess)
    return 0;
  return sms;
}

// defined in seed.cu / spass.cu
size_t seed_workspace_bytes(int mp, int np, int kmax);
pcp_status seed_pcp_async(const double* dD, int mp, int np, double lam,
                          double tol, double rho, double mu_scale,
                          double mu_max_ratio, int max_iter, int k0, int kmax,
                          double rank_cut, int r_cap, void* d_work,
                          double* dU, double* dSigma, double* dV,
                          cudaStream_t st, int** d_rank_out, int ctas,
                          unsigned long long timeout_ns, int* launches,
                          int* team_out);
pcp_status seed_read_ctl(void* d_work, int mp, int np, int kmax,
                         cudaStream_t st, int* rank, int* iters,
                         double* residual, int* converged, int* error,
                         int* rank_raw);
pcp_status gather_seed(const float* dM, int64_t ldm, const int32_t* d_rows,
                       int32_t mp, const int32_t* d_cols, int32_t np,
                       double* dMs, int32_t* d_bad, cudaStream_t st);
pcp_status spass_tc_read_timeouts(int* out);

// splitmix64: the library's own generator for seed sampling.
static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// k distinct values of [0, n), sorted (partial Fisher-Yates on a map-free
// rejection scheme for k << n, full shuffle otherwise).
static std::vector<int64_t> sample_sorted(int64_t n, int64_t k,
                                          uint64_t seed) {
  std::vector<int64_t> out;
  uint64_t s = seed;
  if (k * 4 >= n) {
    std::vector<int64_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    for (int64_t i = 0; i < k; ++i) {
      const int64_t j = i + (int64_t)(splitmix64(s) % (uint64_t)(n - i));
      std::swap(all[i], all[j]);
    }
    out.assign(all.begin(), all.begin() + k);
  } else {
    std::vector<char> taken(n, 0);
    while ((int64_t)out.size() < k) {
      const int64_t v = (int64_t)(splitmix64(s) % (uint64_t)n);
      if (!taken[v]) {
        taken[v] = 1;
        out.push_back(v);
      }
    }
  }
  std::sort(out.begin(), out.end());
  return out;
}

// A random permutation of [0, n) (Fisher-Yates on splitmix64): the library's
// sampling order when seeds may grow (every prefix is a uniform sample).
static std::vector<int64_t> sample_order(int64_t n, uint64_t seed) {
  std::vector<int64_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  uint64_t s = seed;
  for (int64_t i = 0; i + 1 < n; ++i) {
    const int64_t j = i + (int64_t)(splitmix64(s) % (uint64_t)(n - i));
    std::swap(all[i], all[j]);
  }
  return all;
}

static std::vector<int64_t> sorted_prefix(const std::vector<int64_t>& order,
                                          int64_t k) {
  std::vector<int64_t> v(order.begin(), order.begin() + k);
  std::sort(v.begin(), v.end());
  return v;
}

}  // namespace pcp

// S-pass column chunks of a host-buffer solve (each chunk's S goes back to
// the host while the next chunk is computed) and the events that order the
// copy stream against the compute stream.
constexpr int kHostChunks = 8;
constexpr int kHostEvents = kHostChunks + 4;

struct pcp_plan {
  pcp_params p;
  std::vector<int64_t> given_rows, given_cols;
  std::vector<int64_t> row_order, col_order;  // seeds by order (prefixes)
  pcp_plan* child = nullptr;                   // grown seed (Section 3.5)
  // the last solve on this plan stopped after the seed (a failed rank test
  // checked before the filters), so its outputs were not written
  bool stopped_after_seed = false;
  int64_t m, n;
  int r, mp, np, kmax, k0;
  double lam_seed, lam_full;
  int device;
  // device memory (one allocation)
  void* d_base = nullptr;
  size_t d_bytes = 0;
  int32_t *d_rows = nullptr, *d_cols = nullptr, *d_rbar = nullptr,
          *d_cbar = nullptr;
  double *d_Ms = nullptr, *d_U = nullptr, *d_Sigma = nullptr, *d_V = nullptr;
  float *d_U32 = nullptr, *d_V32 = nullptr, *d_inv_sigma = nullptr;
  int32_t *d_iters = nullptr, *d_bad = nullptr;
  void* d_seed_work = nullptr;
  // pinned staging of the index sets
  int32_t* h_idx = nullptr;
  bool idx_uploaded = false;
  std::vector<int64_t> cur_rows, cur_cols;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // host-buffer solves (pcp_l1filter_solve_host), allocated on first use:
  // device copies of M, S and the factors, a copy stream and its events
  float *hd_M = nullptr, *hd_S = nullptr, *hd_Lu = nullptr, *hd_Lv = nullptr;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t cev[kHostEvents] = {};
  // asynchronous solves (info == NULL) replay a CUDA graph of the solve's
  // launches and copies, captured on the second call with the same buffers
  cudaStream_t cap_st = nullptr;
  // the row filter runs on a second stream beside the column filter (the
  // two launches are independent; together they fill the last wave)
  cudaStream_t side_st = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<uintptr_t> gkey;
  int async_calls = 0;
  int64_t graph_launches = 0;
  bool graph_off = false;
  // kernels launched since the public entry point began (pcp_info.launches)
  int launches = 0;
  int seed_team = 0;  // the last seed launch's team (pcp_info.seed_team)
};

extern "C" const char* pcp_last_error(void) { return pcp::g_err; }

extern "C" const char* pcp_version(void) {
  return "pcp_l1f 0.1 (sm_103a)";
}

extern "C" pcp_status pcp_params_default(pcp_params* p, int64_t m, int64_t n,
                                         int32_t r) {
  if (!p) {
    pcp::set_error("pcp_params_default: null pointer");
    return PCP_ERR_ARG;
  }
  std::memset(p, 0, sizeof(*p));
  p->m = m;
  p->n = n;
  p->r = r;
  p->precision = PCP_FP32;
  p->lambda = 0.0;
  p->lambda_seed = 0.0;
  p->s_r = 10.0;
  p->s_c = 10.0;
  p->seed_tol = 1e-7;
  p->seed_rho = 1.5;
  p->seed_mu_scale = 1.25;
  p->seed_mu_max_ratio = 1e7;
  p->rank_cut = 1e-6;
  p->filter_tol = 3e-6;
  p->filter_rho = 1.5;
  p->beta0_scale = 1.0;
  p->beta_bar_ratio = 1e10;
  p->seed_max_iter = 500;
  p->filter_max_iter = 500;
  p->seed_subspace = 0;
  p->lowp_iters = 12;
  p->rng_seed = 0x1108535900000001ull;
  p->seed_rows = nullptr;
  p->seed_cols = nullptr;
  return PCP_OK;
}

static pcp_status check_index_set(const int64_t* v, int64_t k, int64_t n,
                                  const char* what) {
  std::vector<char> seen(n, 0);
  for (int64_t i = 0; i < k; ++i) {
    if (v[i] < 0 || v[i] >= n || seen[v[i]]) {
      pcp::set_error("%s: index %lld at %lld out of range or repeated", what,
                     (long long)v[i], (long long)i);
      return PCP_ERR_ARG;
    }
    seen[v[i]] = 1;
  }
  return PCP_OK;
}

extern "C" pcp_status pcp_l1filter_plan(const pcp_params* params,
                                        pcp_plan** out) {
  PCP_ARG(params && out, "pcp_l1filter_plan: null pointer");
  *out = nullptr;
  const pcp_params& q = *params;
  PCP_ARG(q.m >= 2 && q.n >= 2 && q.m < (1LL << 31) && q.n < (1LL << 31),
          "pcp_l1filter_plan: m=%lld n=%lld out of range", (long long)q.m,
          (long long)q.n);
  PCP_ARG(q.r >= 1 && q.r <= 64, "pcp_l1filter_plan: r=%d outside [1, 64]",
          q.r);
  PCP_ARG(q.s_r > 0 && q.s_c > 0, "pcp_l1filter_plan: oversampling <= 0");
  PCP_ARG(q.precision == PCP_FP32 || q.precision == PCP_TF32_REFINED ||
              q.precision == PCP_BF16_REFINED ||
              q.precision == PCP_FP32_TENSOR || q.precision == PCP_FP32_SIMT,
          "pcp_l1filter_plan: precision %d not available", q.precision);
  PCP_ARG(q.lowp_iters >= 0, "pcp_l1filter_plan: lowp_iters < 0");
  PCP_ARG(q.seed_ctas >= 0, "pcp_l1filter_plan: seed_ctas < 0");
  const int mp = q.seed_m > 0 ? q.seed_m : (int)std::llround(q.s_r * q.r);
  const int np = q.seed_n > 0 ? q.seed_n : (int)std::llround(q.s_c * q.r);
  PCP_ARG(!(q.row_order && q.seed_rows) && !(q.col_order && q.seed_cols),
          "pcp_l1filter_plan: give seed_rows or row_order, not both (same "
          "for columns)");
  PCP_ARG(!q.grow_seed || (!q.seed_rows && !q.seed_cols),
          "pcp_l1filter_plan: grow_seed needs seeds taken by order "
          "(row_order / col_order or sampling), not seed_rows / seed_cols");
  PCP_ARG(mp >= 2 && np >= 2 && mp < q.m && np < q.n,
          "pcp_l1filter_plan: seed %dx%d does not fit in %lldx%lld", mp, np,
          (long long)q.m, (long long)q.n);
  PCP_ARG(mp <= 512 && np <= 512,
          "pcp_l1filter_plan: seed %dx%d larger than 512", mp, np);
  PCP_ARG(q.precision != PCP_FP32_SIMT || (q.r <= 32 && mp <= 256 && np <= 256),
          "pcp_l1filter_plan: PCP_FP32_SIMT takes r <= 32 and seeds up to "
          "256 (r=%d, seed %dx%d)", q.r, mp, np);
  PCP_ARG(q.filter_tol > 0 && q.filter_rho > 1 && q.beta0_scale > 0 &&
              q.beta_bar_ratio >= 1 && q.filter_max_iter >= 1,
          "pcp_l1filter_plan: bad filter parameters");
  PCP_ARG(q.seed_tol > 0 && q.seed_rho > 1 && q.seed_mu_scale > 0 &&
              q.seed_mu_max_ratio >= 1 && q.seed_max_iter >= 1,
          "pcp_l1filter_plan: bad seed parameters");
  if (q.seed_rows) {
    pcp_status s = check_index_set(q.seed_rows, mp, q.m, "seed_rows");
    if (s != PCP_OK) return s;
  }
  if (q.seed_cols) {
    pcp_status s = check_index_set(q.seed_cols, np, q.n, "seed_cols");
    if (s != PCP_OK) return s;
  }
  if (q.row_order) {
    pcp_status s = check_index_set(q.row_order, q.m, q.m, "row_order");
    if (s != PCP_OK) return s;
  }
  if (q.col_order) {
    pcp_status s = check_index_set(q.col_order, q.n, q.n, "col_order");
    if (s != PCP_OK) return s;
  }

  pcp_plan* P = new pcp_plan();
  P->p = q;
  if (q.seed_rows) P->given_rows.assign(q.seed_rows, q.seed_rows + mp);
  if (q.seed_cols) P->given_cols.assign(q.seed_cols, q.seed_cols + np);
  if (q.row_order)
    P->row_order.assign(q.row_order, q.row_order + q.m);
  else if (q.grow_seed)
    P->row_order = pcp::sample_order(q.m, q.rng_seed);
  if (q.col_order)
    P->col_order.assign(q.col_order, q.col_order + q.n);
  else if (q.grow_seed)
    P->col_order = pcp::sample_order(q.n, q.rng_seed ^ 0xC01C01C0ull);
  P->p.seed_rows = nullptr;
  P->p.seed_cols = nullptr;
  P->p.row_order = nullptr;
  P->p.col_order = nullptr;
  P->m = q.m;
  P->n = q.n;
  P->r = q.r;
  P->mp = mp;
  P->np = np;
  int k0 = q.seed_subspace > 0 ? q.seed_subspace
                               : q.r + std::max(6, q.r / 4);
  k0 = (k0 + 1) / 2 * 2;
  const int kcap = std::min(std::min(mp, np) / 2 * 2, 64);
  k0 = std::min(k0, kcap);
  P->k0 = k0;
  P->kmax = std::min(kcap, std::max(k0 + 16, 2 * k0) / 2 * 2);
  P->lam_seed = q.lambda_seed > 0 ? q.lambda_seed
                                  : 1.0 / std::sqrt((double)std::max(mp, np));
  P->lam_full = q.lambda > 0
                    ? q.lambda
                    : 1.0 / std::sqrt((double)std::max(q.m, q.n));
  if (cudaGetDevice(&P->device) != cudaSuccess) P->device = 0;

  // one device allocation, carved up
  const int64_t nrb = q.m - mp, ncb = q.n - np;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_rows = take(sizeof(int32_t) * mp);
  const size_t o_cols = take(sizeof(int32_t) * np);
  const size_t o_rbar = take(sizeof(int32_t) * nrb);
  const size_t o_cbar = take(sizeof(int32_t) * ncb);
  const size_t o_Ms = take(sizeof(double) * mp * np);
  const size_t o_U = take(sizeof(double) * mp * P->kmax);
  const size_t o_Sig = take(sizeof(double) * P->kmax);
  const size_t o_V = take(sizeof(double) * np * P->kmax);
  const size_t o_U32 = take(sizeof(float) * mp * q.r);
  const size_t o_V32 = take(sizeof(float) * np * q.r);
  const size_t o_isg = take(sizeof(float) * q.r);
  const size_t o_it = take(sizeof(int32_t) * (nrb + ncb));
  const size_t o_bad = take(sizeof(int32_t) * 4);
  const size_t o_sw = take(pcp::seed_workspace_bytes(mp, np, P->kmax));
  P->d_bytes = off;
  cudaError_t e = cudaMalloc(&P->d_base, off);
  if (e != cudaSuccess) {
    delete P;
    return pcp::cuda_fail(e, "cudaMalloc(plan workspace)", __FILE__, __LINE__);
  }
  char* base = static_cast<char*>(P->d_base);
  P->d_rows = reinterpret_cast<int32_t*>(base + o_rows);
  P->d_cols = reinterpret_cast<int32_t*>(base + o_cols);
  P->d_rbar = reinterpret_cast<int32_t*>(base + o_rbar);
  P->d_cbar = reinterpret_cast<int32_t*>(base + o_cbar);
  P->d_Ms = reinterpret_cast<double*>(base + o_Ms);
  P->d_U = reinterpret_cast<double*>(base + o_U);
  P->d_Sigma = reinterpret_cast<double*>(base + o_Sig);
  P->d_V = reinterpret_cast<double*>(base + o_V);
  P->d_U32 = reinterpret_cast<float*>(base + o_U32);
  P->d_V32 = reinterpret_cast<float*>(base + o_V32);
  P->d_inv_sigma = reinterpret_cast<float*>(base + o_isg);
  P->d_iters = reinterpret_cast<int32_t*>(base + o_it);
  P->d_bad = reinterpret_cast<int32_t*>(base + o_bad);
  P->d_seed_work = base + o_sw;
  e = cudaMallocHost(&P->h_idx, sizeof(int32_t) * (q.m + q.n));
  if (e != cudaSuccess) {
    cudaFree(P->d_base);
    delete P;
    return pcp::cuda_fail(e, "cudaMallocHost(index staging)", __FILE__,
                          __LINE__);
  }
  for (auto& ev : P->ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
      pcp_plan_destroy(P);
      return pcp::cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__);
    }
  }
  if ((e = cudaStreamCreateWithFlags(&P->side_st, cudaStreamNonBlocking)) !=
          cudaSuccess ||
      (e = cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming)) !=
          cudaSuccess ||
      (e = cudaEventCreateWithFlags(&P->join_ev, cudaEventDisableTiming)) !=
          cudaSuccess) {
    pcp_plan_destroy(P);
    return pcp::cuda_fail(e, "plan streams", __FILE__, __LINE__);
  }
  *out = P;
  return PCP_OK;
}

extern "C" void pcp_plan_destroy(pcp_plan* P) {
  if (!P) return;
  pcp_plan_destroy(P->child);
  for (auto& ev : P->ev)
    if (ev) cudaEventDestroy(ev);
  if (P->h_idx) cudaFreeHost(P->h_idx);
  if (P->d_base) cudaFree(P->d_base);
  for (auto& ev : P->cev)
    if (ev) cudaEventDestroy(ev);
  if (P->copy_st) cudaStreamDestroy(P->copy_st);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->cap_st) cudaStreamDestroy(P->cap_st);
  if (P->side_st) cudaStreamDestroy(P->side_st);
  if (P->fork_ev) cudaEventDestroy(P->fork_ev);
  if (P->join_ev) cudaEventDestroy(P->join_ev);
  cudaFree(P->hd_M);
  cudaFree(P->hd_S);
  cudaFree(P->hd_Lu);
  cudaFree(P->hd_Lv);
  delete P;
}

// Upload I_s, J_s and their sorted complements (only when they changed).
static pcp_status upload_indices(pcp_plan* P, cudaStream_t st) {
  std::vector<int64_t> rows =
      !P->row_order.empty()
          ? pcp::sorted_prefix(P->row_order, P->mp)
          : (P->given_rows.empty()
                 ? pcp::sample_sorted(P->m, P->mp, P->p.rng_seed)
                 : P->given_rows);
  std::vector<int64_t> cols =
      !P->col_order.empty()
          ? pcp::sorted_prefix(P->col_order, P->np)
          : (P->given_cols.empty()
                 ? pcp::sample_sorted(P->n, P->np,
                                      P->p.rng_seed ^ 0xC01C01C0ull)
                 : P->given_cols);
  if (P->idx_uploaded && rows == P->cur_rows && cols == P->cur_cols)
    return PCP_OK;
  // the previous upload may still be read by in-flight work on this stream
  PCP_CUDA(cudaStreamSynchronize(st));
  int32_t* h = P->h_idx;
  std::vector<char> in_r(P->m, 0), in_c(P->n, 0);
  int64_t o = 0;
  for (int i = 0; i < P->mp; ++i) {
    h[o++] = (int32_t)rows[i];
    in_r[rows[i]] = 1;
  }
  for (int j = 0; j < P->np; ++j) {
    h[o++] = (int32_t)cols[j];
    in_c[cols[j]] = 1;
  }
  for (int64_t i = 0; i < P->m; ++i)
    if (!in_r[i]) h[o++] = (int32_t)i;
  for (int64_t j = 0; j < P->n; ++j)
    if (!in_c[j]) h[o++] = (int32_t)j;
  // the four arrays are contiguous pieces of one allocation, but each is
  // 256-byte aligned; copy them one by one.
  PCP_CUDA(cudaMemcpyAsync(P->d_rows, h, sizeof(int32_t) * P->mp,
                           cudaMemcpyHostToDevice, st));
  PCP_CUDA(cudaMemcpyAsync(P->d_cols, h + P->mp, sizeof(int32_t) * P->np,
                           cudaMemcpyHostToDevice, st));
  PCP_CUDA(cudaMemcpyAsync(P->d_rbar, h + P->mp + P->np,
                           sizeof(int32_t) * (P->m - P->mp),
                           cudaMemcpyHostToDevice, st));
  PCP_CUDA(cudaMemcpyAsync(P->d_cbar, h + P->mp + P->np + (P->m - P->mp),
                           sizeof(int32_t) * (P->n - P->np),
                           cudaMemcpyHostToDevice, st));
  P->cur_rows = rows;
  P->cur_cols = cols;
  P->idx_uploaded = true;
  return PCP_OK;
}

// Host buffers of a pcp_l1filter_solve_host call.
struct HostIO {
  const float* hM;     // host M (column-major, ld ldm)
  const float* gM;     // device-accessible address of hM, or null (pageable)
  int64_t ldm;
  float *hLu, *hLv;    // host factors (ld m / ld n)
  float* hS;           // host S (ld lds) or null
  int64_t lds;
};

static pcp_status solve_once(pcp_plan* P, const float* dM, int64_t ldm,
                             float* dLu, float* dLv, float* dS, int64_t lds,
                             int64_t* h_seed_rows_out,
                             int64_t* h_seed_cols_out, pcp_info* info,
                             void* stream, const HostIO* hio = nullptr,
                             bool rank_first = false);

static pcp_status grow_loop(pcp_plan* P, const float* dM, int64_t ldm,
                            float* dLu, float* dLv, float* dS, int64_t lds,
                            int64_t* h_seed_rows_out,
                            int64_t* h_seed_cols_out, pcp_info* info,
                            void* stream, pcp_status st);

// Asynchronous solves through a CUDA graph: the first call runs directly
// (it settles the filter autotuner and any first-use allocation), the
// second with the same buffers is captured on the plan's capture stream and
// instantiated, and later calls with the same buffers replay the graph on
// the caller's stream.  A solve that cannot be captured (an index upload
// that has to synchronise, or anything the CUDA driver refuses to capture) runs
// directly and turns graphs off for the plan.
template <typename Run>
static pcp_status solve_async(pcp_plan* P, std::vector<uintptr_t> key,
                              void* stream, Run run) {
  cudaStream_t st = (cudaStream_t)stream;
  if (P->graph_off || P->async_calls++ == 0) return run(st);
  if (P->gexec && key == P->gkey) {
    PCP_CUDA(cudaGraphLaunch(P->gexec, st));
    ++P->graph_launches;
    return PCP_OK;
  }
  if (!P->cap_st)
    PCP_CUDA(cudaStreamCreateWithFlags(&P->cap_st, cudaStreamNonBlocking));
  // the capture stream must not start before the caller's earlier work
  // when the captured work is replayed: the graph is launched on `st`, so
  // ordering is by the launch; nothing is enqueued on cap_st outside capture
  if (cudaStreamBeginCapture(P->cap_st, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    cudaGetLastError();
    P->graph_off = true;
    return run(st);
  }
  pcp_status s = run(P->cap_st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(P->cap_st, &g);
  cudaGraphExec_t ex = nullptr;
  const bool ok = s == PCP_OK && e == cudaSuccess && g &&
                  cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    if (ex) cudaGraphExecDestroy(ex);
    P->graph_off = true;
    return run(st);
  }
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  P->gexec = ex;
  P->gkey = std::move(key);
  PCP_CUDA(cudaGraphLaunch(P->gexec, st));
  ++P->graph_launches;
  return PCP_OK;
}

extern "C" int64_t pcp_plan_graph_launches(const pcp_plan* P) {
  if (!P) return 0;
  return P->graph_off ? -1 : P->graph_launches;
}

extern "C" pcp_status pcp_l1filter_solve(pcp_plan* P, const float* dM,
                                         int64_t ldm, float* dLu, float* dLv,
                                         float* dS, int64_t lds,
                                         int64_t* h_seed_rows_out,
                                         int64_t* h_seed_cols_out,
                                         pcp_info* info, void* stream) {
  if (P) P->launches = 0;
  if (P && !info) {
    if (h_seed_rows_out || h_seed_cols_out) {
      pcp_status s0 = upload_indices(P, (cudaStream_t)stream);
      if (s0 != PCP_OK) return s0;
      if (h_seed_rows_out)
        std::copy(P->cur_rows.begin(), P->cur_rows.end(), h_seed_rows_out);
      if (h_seed_cols_out)
        std::copy(P->cur_cols.begin(), P->cur_cols.end(), h_seed_cols_out);
    }
    return solve_async(
        P,
        {(uintptr_t)dM, (uintptr_t)ldm, (uintptr_t)dLu, (uintptr_t)dLv,
         (uintptr_t)dS, (uintptr_t)lds},
        stream, [&](cudaStream_t s) {
          return solve_once(P, dM, ldm, dLu, dLv, dS, lds, nullptr, nullptr,
                            nullptr, s);
        });
  }
  pcp_status st = solve_once(P, dM, ldm, dLu, dLv, dS, lds, h_seed_rows_out,
                             h_seed_cols_out, info, stream, nullptr,
                             P && P->p.grow_seed);
  return grow_loop(P, dM, ldm, dLu, dLv, dS, lds, h_seed_rows_out,
                   h_seed_cols_out, info, stream, st);
}

static pcp_status grow_loop(pcp_plan* P, const float* dM, int64_t ldm,
                            float* dLu, float* dLv, float* dS, int64_t lds,
                            int64_t* h_seed_rows_out,
                            int64_t* h_seed_cols_out, pcp_info* info,
                            void* stream, pcp_status st) {
  if (!P || !info || !P->p.grow_seed) return st;
  // Section 3.5: a seed whose rank r' fails Eq. rank_test grows to
  // (s_r r') x (s_c r') (prefixes of the same orders) and the solve repeats,
  // until the test holds or the seed would pass half of a side.
  const pcp_params& q = P->p;
  pcp_plan* cur = P;
  while (st == PCP_ERR_RANK_TEST) {
    const int rr = info->seed_rank_raw;
    const int gm = std::max(cur->mp, (int)std::llround(q.s_r * rr));
    const int gn = std::max(cur->np, (int)std::llround(q.s_c * rr));
    if (rr < 1 || (gm == cur->mp && gn == cur->np) || 2 * (int64_t)gm > q.m ||
        2 * (int64_t)gn > q.n || gm > 512 || gn > 512)
      break;
    if (!P->child || P->child->mp != gm || P->child->np != gn) {
      pcp_plan_destroy(P->child);
      P->child = nullptr;
      pcp_params q2 = q;
      q2.seed_m = gm;
      q2.seed_n = gn;
      q2.grow_seed = 0;
      q2.row_order = P->row_order.data();
      q2.col_order = P->col_order.data();
      pcp_status s2 = pcp_l1filter_plan(&q2, &P->child);
      if (s2 != PCP_OK) return s2;
    }
    cur = P->child;
    P->child->launches = P->launches;  // info->launches counts every attempt
    st = solve_once(P->child, dM, ldm, dLu, dLv, dS, lds, h_seed_rows_out,
                    h_seed_cols_out, info, stream, nullptr, true);
    P->launches = P->child->launches;
  }
  if (st == PCP_ERR_RANK_TEST && cur->stopped_after_seed) {
    // growth gave up: the last seed's solve runs in full, so that the
    // outputs are written as without growth
    cur->launches = P->launches;
    st = solve_once(cur, dM, ldm, dLu, dLv, dS, lds, h_seed_rows_out,
                    h_seed_cols_out, info, stream, nullptr, false);
    P->launches = cur->launches;
  }
  return st;
}

// Device buffers, copy stream and events of host-buffer solves.
static pcp_status ensure_host_buffers(pcp_plan* P, bool want_S) {
  // each resource on its own, so a call after a failed allocation retries
  // only what is missing
  const size_t mn = sizeof(float) * (size_t)P->m * (size_t)P->n;
  if (!P->hd_M) PCP_CUDA(cudaMalloc(&P->hd_M, mn));
  if (!P->hd_Lu)
    PCP_CUDA(cudaMalloc(&P->hd_Lu, sizeof(float) * (size_t)P->m * P->r));
  if (!P->hd_Lv)
    PCP_CUDA(cudaMalloc(&P->hd_Lv, sizeof(float) * (size_t)P->n * P->r));
  if (!P->copy_st)
    PCP_CUDA(cudaStreamCreateWithFlags(&P->copy_st, cudaStreamNonBlocking));
  for (auto& ev : P->cev)
    if (!ev) PCP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  if (want_S && !P->hd_S) PCP_CUDA(cudaMalloc(&P->hd_S, mn));
  return PCP_OK;
}

extern "C" pcp_status pcp_l1filter_solve_host(pcp_plan* P, const float* hM,
                                              int64_t ldm, float* hLu,
                                              float* hLv, float* hS,
                                              int64_t lds, pcp_info* info,
                                              void* stream) {
  PCP_ARG(P && hM && hLu && hLv, "pcp_l1filter_solve_host: null pointer");
  PCP_ARG(ldm >= P->m, "pcp_l1filter_solve_host: ldm < m");
  PCP_ARG(!hS || lds >= P->m, "pcp_l1filter_solve_host: lds < m");
  pcp_status s = ensure_host_buffers(P, hS != nullptr);
  if (s != PCP_OK) return s;
  P->launches = 0;
  // a page-locked M is read in place by the seed gather (the device reads
  // host memory directly), so the seed need not wait for the whole copy
  HostIO io{hM, nullptr, ldm, hLu, hLv, hS, lds};
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, hM) == cudaSuccess &&
      pa.type == cudaMemoryTypeHost && pa.devicePointer)
    io.gM = static_cast<const float*>(pa.devicePointer);
  else
    cudaGetLastError();  // pageable memory: clear the query's error
  cudaStream_t st = (cudaStream_t)stream;
  if (!info)
    return solve_async(
        P,
        {1, (uintptr_t)hM, (uintptr_t)ldm, (uintptr_t)hLu, (uintptr_t)hLv,
         (uintptr_t)hS, (uintptr_t)lds, (uintptr_t)io.gM},
        stream, [&](cudaStream_t s) {
          return solve_once(P, P->hd_M, P->m, P->hd_Lu, P->hd_Lv,
                            hS ? P->hd_S : nullptr, P->m, nullptr, nullptr,
                            nullptr, s, &io);
        });
  pcp_status r = solve_once(P, P->hd_M, P->m, P->hd_Lu, P->hd_Lv,
                            hS ? P->hd_S : nullptr, P->m, nullptr, nullptr,
                            info, stream, &io);
  if (r == PCP_ERR_RANK_TEST && info && P->p.grow_seed) {
    // Section 3.5 growth on the data already on the device, then the
    // grown solve's outputs back to the host
    r = grow_loop(P, P->hd_M, P->m, P->hd_Lu, P->hd_Lv,
                  hS ? P->hd_S : nullptr, P->m, nullptr, nullptr, info,
                  stream, r);
    PCP_CUDA(cudaMemcpyAsync(hLu, P->hd_Lu, sizeof(float) * P->m * P->r,
                             cudaMemcpyDeviceToHost, st));
    PCP_CUDA(cudaMemcpyAsync(hLv, P->hd_Lv, sizeof(float) * P->n * P->r,
                             cudaMemcpyDeviceToHost, st));
    if (hS)
      PCP_CUDA(cudaMemcpy2DAsync(hS, sizeof(float) * lds, P->hd_S,
                                 sizeof(float) * P->m, sizeof(float) * P->m,
                                 P->n, cudaMemcpyDeviceToHost, st));
    PCP_CUDA(cudaStreamSynchronize(st));
  }
  return r;
}

static pcp_status solve_once(pcp_plan* P, const float* dM, int64_t ldm,
                             float* dLu, float* dLv, float* dS, int64_t lds,
                             int64_t* h_seed_rows_out,
                             int64_t* h_seed_cols_out, pcp_info* info,
                             void* stream, const HostIO* hio,
                             bool rank_first) {
  PCP_ARG(P, "pcp_l1filter_solve: null plan");
  PCP_ARG(dM && dLu && dLv, "pcp_l1filter_solve: null pointer");
  PCP_ARG(ldm >= P->m, "pcp_l1filter_solve: ldm < m");
  PCP_ARG(!dS || lds >= P->m, "pcp_l1filter_solve: lds < m");
  cudaStream_t st = (cudaStream_t)stream;
  const pcp_params& q = P->p;
  pcp_status s = upload_indices(P, st);
  if (s != PCP_OK) return s;
  if (h_seed_rows_out)
    std::copy(P->cur_rows.begin(), P->cur_rows.end(), h_seed_rows_out);
  if (h_seed_cols_out)
    std::copy(P->cur_cols.begin(), P->cur_cols.end(), h_seed_cols_out);
  const bool timed = info != nullptr;
  if (timed) PCP_CUDA(cudaEventRecord(P->ev[0], st));

  // host buffers: M goes to the device on the copy stream (after whatever
  // this stream still runs on the device copy), overlapping the seed
  cudaEvent_t* cev = P->cev;
  if (hio) {
    PCP_CUDA(cudaEventRecord(cev[0], st));
    PCP_CUDA(cudaStreamWaitEvent(P->copy_st, cev[0], 0));
    PCP_CUDA(cudaMemcpy2DAsync(
        const_cast<float*>(dM), sizeof(float) * ldm, hio->hM,
        sizeof(float) * hio->ldm, sizeof(float) * P->m, P->n,
        cudaMemcpyHostToDevice, P->copy_st));
    PCP_CUDA(cudaEventRecord(cev[1], P->copy_st));
    if (!hio->gM) PCP_CUDA(cudaStreamWaitEvent(st, cev[1], 0));
  }
  // stage 1: gather the seed (FP64) and count non-finite entries (from the
  // page-locked host M itself when the device can read it)
  pcp::NvtxStages nvtx("pcp.seed");
  PCP_CUDA(cudaMemsetAsync(P->d_bad, 0, sizeof(int32_t), st));
  s = (hio && hio->gM)
          ? pcp::gather_seed(hio->gM, hio->ldm, P->d_rows, P->mp, P->d_cols,
                             P->np, P->d_Ms, P->d_bad, st)
          : pcp::gather_seed(dM, ldm, P->d_rows, P->mp, P->d_cols, P->np,
                             P->d_Ms, P->d_bad, st);
  if (s != PCP_OK) return s;
  ++P->launches;
  // stage 2: seed PCP (FP64)
  int* d_rank = nullptr;
  s = pcp::seed_pcp_async(P->d_Ms, P->mp, P->np, P->lam_seed, q.seed_tol,
                          q.seed_rho, q.seed_mu_scale, q.seed_mu_max_ratio,
                          q.seed_max_iter, P->k0, P->kmax, q.rank_cut, P->r,
                          P->d_seed_work, P->d_U, P->d_Sigma, P->d_V, st,
                          &d_rank, q.seed_ctas,
                          q.wait_timeout_ns > 0
                              ? (unsigned long long)q.wait_timeout_ns
                              : 0ull,
                          &P->launches, &P->seed_team);
  if (s != PCP_OK) return s;
  // stage 5 (seed rows of the factors) + FP32 bases for the filters
  s = pcp_assemble_factors(P->d_U, P->d_Sigma, P->d_V, P->mp, P->np, P->kmax,
                           d_rank, P->r, P->d_rows, P->d_cols, dLu, P->m, dLv,
                           P->n, P->d_U32, P->d_V32, P->d_inv_sigma, st);
  if (s != PCP_OK) return s;
  ++P->launches;
  if (timed) PCP_CUDA(cudaEventRecord(P->ev[1], st));
  P->stopped_after_seed = false;
  if (rank_first && timed && !hio) {
    // Section 3.5 with seed growth on: the seed's rank decides whether this
    // seed is kept, so it is read now and a seed that fails Eq. rank_test
    // (and will grow) does not pay for the filters and the S pass
    int rank = 0, iters = 0, conv = 0, err = 0, rank_raw = 0;
    double resid = 0;
    s = pcp::seed_read_ctl(P->d_seed_work, P->mp, P->np, P->kmax, st, &rank,
                           &iters, &resid, &conv, &err, &rank_raw);
    if (s != PCP_OK) return s;
    int32_t bad = 0;
    PCP_CUDA(cudaMemcpy(&bad, P->d_bad, sizeof(int32_t),
                        cudaMemcpyDeviceToHost));
    const bool ok = rank_raw >= 1 &&
                    (double)P->mp / rank_raw >= q.s_r - 1e-9 &&
                    (double)P->np / rank_raw >= q.s_c - 1e-9;
    if (!err && !bad && conv && !ok) {
      float t01 = 0.0f;
      cudaEventElapsedTime(&t01, P->ev[0], P->ev[1]);
      std::memset(info, 0, sizeof(*info));
      info->rank = rank;
      info->seed_iters = iters;
      info->seed_residual = resid;
      info->seed_m = P->mp;
      info->seed_n = P->np;
      info->seed_rank_raw = rank_raw;
      info->lambda = P->lam_full;
      info->rank_ok = 0;
      info->status = (int32_t)PCP_ERR_RANK_TEST;
      info->launches = P->launches;
      info->seed_team = P->seed_team;
      info->t_seed_ms = t01;
      info->t_total_ms = t01;
      P->stopped_after_seed = true;
      pcp::set_error("rank test failed: seed rank %d for a %dx%d seed",
                     rank_raw, P->mp, P->np);
      return PCP_ERR_RANK_TEST;
    }
  }
  if (hio) PCP_CUDA(cudaStreamWaitEvent(st, cev[1], 0));  // all of M landed
  // stages 3 and 4: column and row filtering (Algorithm 1), the row filter
  // on the plan's second stream so that both launches share the GPU
  const int64_t ncb = P->n - P->np, nrb = P->m - P->mp;
  nvtx.next("pcp.filter");
  PCP_CUDA(cudaEventRecord(P->fork_ev, st));
  PCP_CUDA(cudaStreamWaitEvent(P->side_st, P->fork_ev, 0));
  s = pcp_l1_filter(dM, P->d_rows, P->mp, 1, P->d_cbar, (int32_t)ncb, ldm,
                    P->d_U32, P->mp, P->r, d_rank, nullptr, dLv, P->n,
                    q.filter_tol, q.filter_rho, q.beta0_scale,
                    q.beta_bar_ratio, q.filter_max_iter, q.precision,
                    q.lowp_iters, P->d_iters, st);
  if (s != PCP_OK) return s;
  P->launches += ncb > 0;
  s = pcp_l1_filter(dM, P->d_cols, P->np, ldm, P->d_rbar, (int32_t)nrb, 1,
                    P->d_V32, P->np, P->r, d_rank, P->d_inv_sigma, dLu, P->m,
                    q.filter_tol, q.filter_rho, q.beta0_scale,
                    q.beta_bar_ratio, q.filter_max_iter, q.precision,
                    q.lowp_iters, P->d_iters + ncb, P->side_st);
  if (s != PCP_OK) return s;
  P->launches += nrb > 0;
  PCP_CUDA(cudaEventRecord(P->join_ev, P->side_st));
  PCP_CUDA(cudaStreamWaitEvent(st, P->join_ev, 0));
  if (timed) PCP_CUDA(cudaEventRecord(P->ev[2], st));
  if (hio) {
    // the factors go back while the S pass runs
    PCP_CUDA(cudaEventRecord(cev[2], st));
    PCP_CUDA(cudaStreamWaitEvent(P->copy_st, cev[2], 0));
    PCP_CUDA(cudaMemcpyAsync(hio->hLu, dLu, sizeof(float) * P->m * P->r,
                             cudaMemcpyDeviceToHost, P->copy_st));
    PCP_CUDA(cudaMemcpyAsync(hio->hLv, dLv, sizeof(float) * P->n * P->r,
                             cudaMemcpyDeviceToHost, P->copy_st));
  }
  nvtx.next("pcp.spass");
  // stage 6: S = M - Lu Lv^T (host buffers: in column chunks of a multiple
  // of 64 columns, each chunk's S copied back while the next is computed)
  if (dS && hio) {
    const int64_t w = std::max<int64_t>(
        64, (P->n + kHostChunks - 1) / kHostChunks / 64 * 64 + 64);
    int c = 0;
    for (int64_t j0 = 0; j0 < P->n; j0 += w, ++c) {
      const int64_t nc = std::min(w, P->n - j0);
      s = pcp_spass(dM + j0 * ldm, ldm, dLu, P->m, dLv + j0, P->n, P->r,
                    dS + j0 * lds, lds, P->m, nc, st);
      if (s != PCP_OK) return s;
      ++P->launches;
      PCP_CUDA(cudaEventRecord(cev[4 + c], st));
      PCP_CUDA(cudaStreamWaitEvent(P->copy_st, cev[4 + c], 0));
      PCP_CUDA(cudaMemcpy2DAsync(hio->hS + j0 * hio->lds,
                                 sizeof(float) * hio->lds, dS + j0 * lds,
                                 sizeof(float) * lds, sizeof(float) * P->m,
                                 nc, cudaMemcpyDeviceToHost, P->copy_st));
    }
  } else if (dS) {
    s = pcp_spass(dM, ldm, dLu, P->m, dLv, P->n, P->r, dS, lds, P->m, P->n,
                  st);
    if (s != PCP_OK) return s;
    ++P->launches;
  }
  if (hio) {
    // this stream's later work (and its synchronisation) follows the copies
    PCP_CUDA(cudaEventRecord(cev[3], P->copy_st));
    PCP_CUDA(cudaStreamWaitEvent(st, cev[3], 0));
  }
  if (!timed) return PCP_OK;
  PCP_CUDA(cudaEventRecord(P->ev[3], st));

  // diagnostics
  int rank = 0, iters = 0, conv = 0, err = 0, rank_raw = 0;
  double resid = 0;
  s = pcp::seed_read_ctl(P->d_seed_work, P->mp, P->np, P->kmax, st, &rank,
                         &iters, &resid, &conv, &err, &rank_raw);
  if (s != PCP_OK) return s;
  if (dS) {
    // bounded waits of the tensor-core S pass that ran out since the last
    // check (a device-wide counter)
    static std::atomic<int> seen{0};
    int tmo = 0;
    s = pcp::spass_tc_read_timeouts(&tmo);
    if (s != PCP_OK) return s;
    if (tmo > seen.exchange(tmo)) {
      pcp::set_error("S pass: a device wait timed out");
      return PCP_ERR_TIMEOUT;
    }
  }
  std::vector<int32_t> it(ncb + nrb);
  int32_t bad = 0;
  PCP_CUDA(cudaMemcpy(it.data(), P->d_iters, sizeof(int32_t) * it.size(),
                      cudaMemcpyDeviceToHost));
  PCP_CUDA(cudaMemcpy(&bad, P->d_bad, sizeof(int32_t),
                      cudaMemcpyDeviceToHost));
  std::memset(info, 0, sizeof(*info));
  info->rank = rank;
  info->seed_iters = iters;
  info->seed_residual = resid;
  info->seed_m = P->mp;
  info->seed_n = P->np;
  info->seed_rank_raw = rank_raw;
  info->problems = ncb + nrb;
  info->lambda = P->lam_full;
  int imax = 0;
  int64_t unconv = 0;
  double isum = 0.0;
  for (int32_t v : it) {
    imax = std::max(imax, v < 0 ? -v : v);
    unconv += (v < 0);
    isum += v < 0 ? -v : v;
  }
  info->filter_iters_max = imax;
  info->problems_unconverged = unconv;
  info->filter_iters_mean = it.empty() ? 0.0 : isum / (double)it.size();
  info->filter_kernel =
      pcp_l1_filter_kernel(P->mp, P->r, q.precision) == PCP_KERNEL_SIMT
          ? PCP_KERNEL_SIMT
          : PCP_KERNEL_TENSOR;
  info->launches = P->launches;
  info->seed_team = P->seed_team;
  // Eq. rank_test on the numerical rank before the cap at the target r
  info->rank_ok = (rank_raw >= 1 &&
                   (double)P->mp / rank_raw >= q.s_r - 1e-9 &&
                   (double)P->np / rank_raw >= q.s_c - 1e-9)
                      ? 1
                      : 0;
  float t01 = 0, t12 = 0, t23 = 0, t03 = 0;
  cudaEventElapsedTime(&t01, P->ev[0], P->ev[1]);
  cudaEventElapsedTime(&t12, P->ev[1], P->ev[2]);
  cudaEventElapsedTime(&t23, P->ev[2], P->ev[3]);
  cudaEventElapsedTime(&t03, P->ev[0], P->ev[3]);
  info->t_seed_ms = t01;
  info->t_filter_ms = t12;
  info->t_spass_ms = t23;
  info->t_total_ms = t03;
  pcp_status result = PCP_OK;
  if (err) result = PCP_ERR_TIMEOUT;
  else if (bad) result = PCP_ERR_NONFINITE;
  else if (!conv) result = PCP_ERR_SEED_NOCONV;
  else if (!info->rank_ok) result = PCP_ERR_RANK_TEST;
  else if (unconv) result = PCP_ERR_FILTER_NOCONV;
  info->status = (int32_t)result;
  if (err) {
    pcp::set_error("seed PCP: device barrier wait timed out");
    return PCP_ERR_TIMEOUT;
  }
  if (bad) {
    pcp::set_error("seed block of M holds %d non-finite entries", bad);
    return PCP_ERR_NONFINITE;
  }
  if (!conv) {
    pcp::set_error("seed PCP did not converge in %d iterations", iters);
    return PCP_ERR_SEED_NOCONV;
  }
  if (!info->rank_ok) {
    pcp::set_error("rank test failed: seed rank %d for a %dx%d seed",
                   rank_raw, P->mp, P->np);
    return PCP_ERR_RANK_TEST;
  }
  if (unconv) {
    pcp::set_error("%lld l1 problems hit filter_max_iter",
                   (long long)unconv);
    return PCP_ERR_FILTER_NOCONV;
  }
  return PCP_OK;
}

extern "C" int32_t pcp_plan_seed_trace(const pcp_plan* P, uint64_t* h_out,
                                       int32_t cap, void* stream) {
  if (!P) return -1;
  return pcp_seed_trace(P->d_seed_work, P->mp, P->np, P->kmax, h_out, cap,
                        stream);
}
