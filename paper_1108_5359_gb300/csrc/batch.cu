// Many independent PCP solves at once (the batched form of Algorithm 2).
//
// Every stage runs as one launch over all instances: a batched gather, one
// CTA per seed PCP (the seeds of different instances run side by side), a
// batched factor assembly, and a single Algorithm 1 launch whose tile list
// covers the column and row problems of every instance (Section 3.2: all
// these problems are independent).  The S pass runs per instance.  The
// launch half (batch_launch) is asynchronous and is shared with the serving
// loop; batch_finish reads the per-instance diagnostics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "internal.cuh"

namespace pcp {

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

std::vector<int64_t> sample(int64_t n, int64_t k, uint64_t seed) {
  std::vector<int64_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  uint64_t s = seed;
  for (int64_t i = 0; i < k; ++i) {
    const int64_t j = i + (int64_t)(splitmix(s) % (uint64_t)(n - i));
    std::swap(all[i], all[j]);
  }
  std::vector<int64_t> out(all.begin(), all.begin() + k);
  std::sort(out.begin(), out.end());
  return out;
}

// Index block of one instance, written on the device: the seed rows and
// columns in their given order, then the other rows and columns in
// ascending order.  src holds rows, cols and sorted copies of both; a
// non-seed index i goes to position i - (number of seed indices below i).
struct ComplementTask {
  const int32_t* src;  // rows (mp), cols (np), sorted rows, sorted cols
  int32_t* idx;        // rows, cols, rbar (m - mp), cbar (n - np)
  int m, n, mp, np;
};

__device__ __forceinline__ int lower_bound_i32(const int32_t* v, int len,
                                               int x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void complement_batched_kernel(
    const ComplementTask* __restrict__ tasks) {
  const ComplementTask t = tasks[blockIdx.y];
  const int32_t* srows = t.src + t.mp + t.np;
  const int32_t* scols = srows + t.mp;
  int32_t* rbar = t.idx + t.mp + t.np;
  int32_t* cbar = rbar + (t.m - t.mp);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < t.m + t.n;
       e += gridDim.x * blockDim.x) {
    if (e < t.mp + t.np) t.idx[e] = t.src[e];
    if (e < t.m) {
      const int c = lower_bound_i32(srows, t.mp, e);
      if (c == t.mp || srows[c] != e) rbar[e - c] = e;
    } else {
      const int j = e - t.m;
      const int c = lower_bound_i32(scols, t.np, j);
      if (c == t.np || scols[c] != j) cbar[j - c] = j;
    }
  }
}

struct SummaryTask {
  const SeedCtl* ctl;
  const int32_t* iters;
  int64_t nprob;
  const int32_t* bad;
  int32_t* skip;      // written by batch_gate_kernel
  int mp, np;         // seed size
  int64_t m, n;
  double s_r, s_c;
  int gate;           // grow_seed on and the caller grows failed seeds
};

// Section 3.5 on the device, before the filters: an instance whose seed
// failed Eq. rank_test and will grow to (s_r r') x (s_c r') skips its
// filters (the same test and grown size as the host's, so the host grows
// exactly the skipped instances; it runs again without the gate any
// skipped instance it does not grow).
__global__ void batch_gate_kernel(const SummaryTask* __restrict__ tasks,
                                  int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const SummaryTask t = tasks[i];
  int skip = 0;
  if (t.gate) {
    const int rr = t.ctl->rank_raw;
    const bool rank_ok = rr >= 1 && (double)t.mp / rr >= t.s_r - 1e-9 &&
                         (double)t.np / rr >= t.s_c - 1e-9;
    int gm = 0, gn = 0;
    if (t.ctl->converged && *t.bad == 0 && !rank_ok)
      skip = grown_seed_dims(rr, t.mp, t.np, t.m, t.n, t.s_r, t.s_c, &gm, &gn);
  }
  *t.skip = skip;
}

// Per-instance diagnostics reduced on the device, so that batch_finish
// reads the whole batch with one copy.
__global__ void batch_summary_kernel(const SummaryTask* __restrict__ tasks,
                                     BatchSummary* __restrict__ out) {
  const SummaryTask t = tasks[blockIdx.x];
  const int skipped = *t.skip;
  const int64_t nprob = skipped ? 0 : t.nprob;  // no filter ran
  int imax = 0;
  long long unconv = 0, isum = 0;
  for (int64_t j = threadIdx.x; j < nprob; j += blockDim.x) {
    const int v = t.iters[j];
    imax = max(imax, v < 0 ? -v : v);
    unconv += (v < 0);
    isum += v < 0 ? -v : v;
  }
  __shared__ int smax[8];
  __shared__ long long scnt[8], ssum[8];
  for (int o = 16; o > 0; o >>= 1) {
    imax = max(imax, __shfl_xor_sync(0xffffffffu, imax, o));
    unconv += __shfl_xor_sync(0xffffffffu, unconv, o);
    isum += __shfl_xor_sync(0xffffffffu, isum, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    smax[w] = imax;
    scnt[w] = unconv;
    ssum[w] = isum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    BatchSummary r;
    r.iters_max = 0;
    r.unconverged = 0;
    r.iters_sum = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      r.iters_max = max(r.iters_max, smax[q]);
      r.unconverged += scnt[q];
      r.iters_sum += ssum[q];
    }
    r.rank = t.ctl->rank;
    r.iters = t.ctl->iters;
    r.converged = t.ctl->converged;
    r.rank_raw = t.ctl->rank_raw;
    r.residual = t.ctl->residual;
    r.bad = *t.bad;
    r.skipped = skipped;
    out[blockIdx.x] = r;
  }
}

}  // namespace

// The whole sampling order behind sample(): its first k entries, sorted,
// are sample(n, k, seed), so seeds grown along it keep their first rows.
std::vector<int64_t> sample_order(int64_t n, uint64_t seed) {
  std::vector<int64_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  uint64_t s = seed;
  for (int64_t i = 0; i + 1 < n; ++i) {
    const int64_t j = i + (int64_t)(splitmix(s) % (uint64_t)(n - i));
    std::swap(all[i], all[j]);
  }
  return all;
}

bool grown_seed_size(const pcp_params& q, const pcp_info& inf, int* gm,
                     int* gn) {
  return grown_seed_dims(inf.seed_rank_raw, (int)inf.seed_m, (int)inf.seed_n,
                         q.m, q.n, q.s_r, q.s_c, gm, gn);
}

pcp_status batch_validate(const pcp_problem& pr, BatchInstance* bi) {
  const pcp_params& q = pr.params;
  PCP_ARG(q.m >= 2 && q.n >= 2 && q.m < (1LL << 31) && q.n < (1LL << 31),
          "batch: m=%lld n=%lld out of range", (long long)q.m, (long long)q.n);
  PCP_ARG(q.r >= 1 && q.r <= 64, "batch: r=%d outside [1, 64]", q.r);
  PCP_ARG(q.precision == PCP_FP32 || q.precision == PCP_TF32_REFINED ||
              q.precision == PCP_BF16_REFINED ||
              q.precision == PCP_FP32_TENSOR || q.precision == PCP_FP32_SIMT,
          "batch: precision %d not available", q.precision);
  PCP_ARG(q.lowp_iters >= 0, "batch: lowp_iters < 0");
  PCP_ARG(pr.dM && pr.dLu && pr.dLv && pr.ldm >= q.m &&
              (!pr.dS || pr.lds >= q.m),
          "batch: null pointer or leading dimension too small");
  const int mp = q.seed_m > 0 ? q.seed_m : (int)std::llround(q.s_r * q.r);
  const int np = q.seed_n > 0 ? q.seed_n : (int)std::llround(q.s_c * q.r);
  PCP_ARG(!(q.row_order && q.seed_rows) && !(q.col_order && q.seed_cols),
          "batch: give seed_rows or row_order, not both");
  PCP_ARG(!q.grow_seed || (!q.seed_rows && !q.seed_cols),
          "batch: grow_seed needs seeds taken by order (row_order / "
          "col_order or sampling), not seed_rows / seed_cols");
  PCP_ARG(mp >= 2 && np >= 2 && mp < q.m && np < q.n && mp <= 512 && np <= 512,
          "batch: seed %dx%d invalid for %lldx%lld", mp, np, (long long)q.m,
          (long long)q.n);
  PCP_ARG(q.precision != PCP_FP32_SIMT || (q.r <= 32 && mp <= 256 && np <= 256),
          "batch: PCP_FP32_SIMT takes r <= 32 and seeds up to 256");
  PCP_ARG(q.filter_tol > 0 && q.filter_rho > 1 && q.seed_tol > 0 &&
              q.seed_rho > 1 && q.seed_max_iter >= 1 &&
              q.filter_max_iter >= 1 && q.beta0_scale > 0 &&
              q.beta_bar_ratio >= 1 && q.seed_mu_scale > 0 &&
              q.seed_mu_max_ratio >= 1,
          "batch: bad tolerances or penalty constants");
  bi->mp = mp;
  bi->np = np;
  int k0 = q.seed_subspace > 0 ? q.seed_subspace : q.r + std::max(6, q.r / 4);
  k0 = (k0 + 1) / 2 * 2;
  const int kcap = std::min(std::min(mp, np) / 2 * 2, 64);
  bi->k0 = std::min(k0, kcap);
  // Room for one growth step of the subspace (k0 + max(8, k0 / 4)): a seed
  // that passes Eq. rank_test keeps r' <= r < k0 values, and the batched
  // seeds share one launch whose shared memory is sized by the largest
  // kmax; at r = 30 this keeps it at ~78 KB (two CTAs per SM) instead of
  // ~116 KB for kmax = 64 (one).
  bi->kmax = std::min(kcap, (bi->k0 + std::max(8, bi->k0 / 4) + 1) / 2 * 2);
  bi->lam_seed = q.lambda_seed > 0
                     ? q.lambda_seed
                     : 1.0 / std::sqrt((double)std::max(mp, np));
  bi->lam_full = q.lambda > 0 ? q.lambda
                              : 1.0 / std::sqrt((double)std::max(q.m, q.n));
  auto check = [&](const int64_t* v, int64_t k, int64_t n) {
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < k; ++i) {
      if (v[i] < 0 || v[i] >= n || seen[v[i]]) return false;
      seen[v[i]] = 1;
    }
    return true;
  };
  PCP_ARG(!q.seed_rows || check(q.seed_rows, mp, q.m),
          "batch: seed_rows out of range or repeated");
  PCP_ARG(!q.seed_cols || check(q.seed_cols, np, q.n),
          "batch: seed_cols out of range or repeated");
  PCP_ARG(!q.row_order || check(q.row_order, q.m, q.m),
          "batch: row_order is not a permutation");
  PCP_ARG(!q.col_order || check(q.col_order, q.n, q.n),
          "batch: col_order is not a permutation");
  return PCP_OK;
}

size_t batch_footprint(const pcp_problem& pr, const BatchInstance& bi) {
  const pcp_params& q = pr.params;
  const int64_t nrb = q.m - bi.mp, ncb = q.n - bi.np;
  size_t b = 0;
  b += align256(sizeof(int32_t) * (q.m + q.n));                  // indices
  b += sizeof(int32_t) * 2 * (bi.mp + bi.np) + 64;                // staged seeds
  b += align256(sizeof(double) * bi.mp * bi.np);                 // M^s
  b += align256(seed_workspace_bytes_cta(bi.mp, bi.np, bi.kmax));
  b += align256(sizeof(double) * (bi.mp + bi.np + 1) * bi.kmax); // U, S, V
  b += align256(sizeof(float) * ((bi.mp + bi.np) * q.r + q.r));  // FP32 copies
  b += align256(sizeof(int32_t) * (nrb + ncb + 2));  // iters, bad, skip
  return b + 8192;  // share of the batch-wide argument blocks
}

pcp_status batch_launch(int count, const pcp_problem* probs, cudaStream_t st,
                        BatchHandle* h, bool timed,
                        const unsigned char* grow_gate) {
  PCP_ARG(count >= 1 && count <= 65535,
          "batch: count %d outside [1, 65535]", count);
  h->count = count;
  h->inst.assign(count, BatchInstance());
  h->probs.assign(probs, probs + count);
  if (!h->prealloc) h->d_base = nullptr;  // a plan's workspace stays
  for (int i = 0; i < count; ++i) {
    pcp_status s = batch_validate(probs[i], &h->inst[i]);
    if (s != PCP_OK) {
      set_error("batch instance %d: %s", i, pcp_last_error());
      return s;
    }
  }
  // ---- device layout ------------------------------------------------------
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  std::vector<size_t> o_idx(count), o_Ms(count), o_work(count), o_U(count),
      o_Sig(count), o_V(count), o_U32(count), o_V32(count), o_isg(count),
      o_it(count);
  int64_t seed_total = 0;  // staged seed indices, 2 (m' + n') per instance
  for (int i = 0; i < count; ++i) {
    const pcp_params& q = probs[i].params;
    const BatchInstance& b = h->inst[i];
    o_idx[i] = take(sizeof(int32_t) * (q.m + q.n));
    seed_total += 2 * (b.mp + b.np);
    o_Ms[i] = take(sizeof(double) * b.mp * b.np);
    o_work[i] = take(seed_workspace_bytes_cta(b.mp, b.np, b.kmax));
    o_U[i] = take(sizeof(double) * b.mp * b.kmax);
    o_Sig[i] = take(sizeof(double) * b.kmax);
    o_V[i] = take(sizeof(double) * b.np * b.kmax);
    o_U32[i] = take(sizeof(float) * b.mp * q.r);
    o_V32[i] = take(sizeof(float) * b.np * q.r);
    o_isg[i] = take(sizeof(float) * q.r);
    o_it[i] = take(sizeof(int32_t) * ((q.m - b.mp) + (q.n - b.np)));
  }
  const size_t o_bad = take(sizeof(int32_t) * count);
  const size_t o_skip = take(sizeof(int32_t) * count);
  const size_t o_seeds = take(sizeof(int32_t) * (size_t)seed_total);
  const size_t o_ctask = take(sizeof(ComplementTask) * count);
  const size_t o_sargs = take(seed_batched_args_bytes(count));
  const size_t o_gat = take(sizeof(GatherTask) * count);
  const size_t o_asm = take(sizeof(AssembleTask) * count);
  const size_t o_stask = take(sizeof(SummaryTask) * count);
  const size_t o_sum = take(sizeof(BatchSummary) * count);
  // filter sets: two per instance
  std::vector<FilterSet> sets(2 * count);
  for (int i = 0; i < count; ++i) {
    const pcp_params& q = probs[i].params;
    const BatchInstance& b = h->inst[i];
    sets[2 * i].N = (int)(q.n - b.np);
    sets[2 * i + 1].N = (int)(q.m - b.mp);
  }
  const size_t fbytes = filter_batch_bytes(sets.data(), 2 * count);
  const size_t o_filt = take(fbytes);
  if (h->size_only) {
    h->bytes = off;
    return PCP_OK;
  }
  if (h->prealloc) {
    PCP_ARG(h->d_base && h->bytes >= off,
            "batch: workspace of %zu bytes, %zu needed", h->bytes, off);
  } else {
    h->bytes = off;
    PCP_CUDA(cudaMallocAsync(&h->d_base, off, st));
  }
  char* base = static_cast<char*>(h->d_base);

  // ---- host staging: seed indices, then the argument blocks ---------------
  // Only the seed rows and columns (and sorted copies) go to the device;
  // complement_batched_kernel writes each instance's whole index block.
  std::vector<int32_t> hseeds((size_t)seed_total);
  h->h_ctask.resize(sizeof(ComplementTask) * count);
  ComplementTask* ctask = reinterpret_cast<ComplementTask*>(h->h_ctask.data());
  int64_t pos = 0;
  int64_t widest = 1;
  for (int i = 0; i < count; ++i) {
    const pcp_params& q = probs[i].params;
    BatchInstance& b = h->inst[i];
    auto prefix = [](const int64_t* order, int64_t k) {
      std::vector<int64_t> v(order, order + k);
      std::sort(v.begin(), v.end());
      return v;
    };
    std::vector<int64_t> rows =
        q.seed_rows ? std::vector<int64_t>(q.seed_rows, q.seed_rows + b.mp)
                    : (q.row_order ? prefix(q.row_order, b.mp)
                                   : sample(q.m, b.mp, q.rng_seed));
    std::vector<int64_t> cols =
        q.seed_cols ? std::vector<int64_t>(q.seed_cols, q.seed_cols + b.np)
                    : (q.col_order ? prefix(q.col_order, b.np)
                                   : sample(q.n, b.np,
                                            q.rng_seed ^ 0xC01C01C0ull));
    int32_t* hp = hseeds.data() + pos;
    int64_t o = 0;
    for (int64_t v : rows) hp[o++] = (int32_t)v;
    for (int64_t v : cols) hp[o++] = (int32_t)v;
    std::vector<int64_t> srt(rows);
    std::sort(srt.begin(), srt.end());
    for (int64_t v : srt) hp[o++] = (int32_t)v;
    srt.assign(cols.begin(), cols.end());
    std::sort(srt.begin(), srt.end());
    for (int64_t v : srt) hp[o++] = (int32_t)v;
    b.rows = std::move(rows);
    b.cols = std::move(cols);
    ctask[i] = ComplementTask{
        reinterpret_cast<const int32_t*>(base + o_seeds) + pos,
        reinterpret_cast<int32_t*>(base + o_idx[i]), (int)q.m, (int)q.n, b.mp,
        b.np};
    widest = std::max<int64_t>(widest, q.m + q.n);
    pos += o;
  }
  if (!h->indices_ready) {
    PCP_CUDA(cudaMemcpyAsync(base + o_seeds, hseeds.data(),
                             sizeof(int32_t) * (size_t)seed_total,
                             cudaMemcpyHostToDevice, st));
    PCP_CUDA(cudaMemcpyAsync(base + o_ctask, ctask,
                             sizeof(ComplementTask) * count,
                             cudaMemcpyHostToDevice, st));
  }
  PCP_CUDA(cudaMemsetAsync(base + o_bad, 0, sizeof(int32_t) * count, st));

  std::vector<GatherTask> gat(count);
  std::vector<SeedTask> seeds(count);
  std::vector<AssembleTask> asmb(count);
  for (int i = 0; i < count; ++i) {
    const pcp_params& q = probs[i].params;
    const pcp_problem& pr = probs[i];
    BatchInstance& b = h->inst[i];
    int32_t* d_idx = reinterpret_cast<int32_t*>(base + o_idx[i]);
    b.d_rows = d_idx;
    b.d_cols = d_idx + b.mp;
    b.d_rbar = d_idx + b.mp + b.np;
    b.d_cbar = d_idx + b.mp + b.np + (q.m - b.mp);
    b.d_work = base + o_work[i];
    b.d_iters = reinterpret_cast<int32_t*>(base + o_it[i]);
    b.d_bad = reinterpret_cast<int32_t*>(base + o_bad) + i;
    double* Ms = reinterpret_cast<double*>(base + o_Ms[i]);
    gat[i] = GatherTask{pr.dM, pr.ldm, b.d_rows, b.d_cols, b.mp, b.np, Ms,
                        b.d_bad};
    SeedTask& t = seeds[i];
    t.D = Ms;
    t.mp = b.mp;
    t.np = b.np;
    t.k0 = b.k0;
    t.kmax = b.kmax;
    t.max_iter = q.seed_max_iter;
    t.r_cap = q.r;
    t.lam = b.lam_seed;
    t.tol = q.seed_tol;
    t.rho = q.seed_rho;
    t.mu_scale = q.seed_mu_scale;
    t.mu_max_ratio = q.seed_mu_max_ratio;
    t.rank_cut = q.rank_cut;
    t.work = b.d_work;
    t.U = reinterpret_cast<double*>(base + o_U[i]);
    t.Sigma = reinterpret_cast<double*>(base + o_Sig[i]);
    t.V = reinterpret_cast<double*>(base + o_V[i]);
    t.timeout_ns = q.wait_timeout_ns > 0 ? (unsigned long long)q.wait_timeout_ns
                                         : 0ull;
    b.d_rank = seed_rank_ptr_cta(b.d_work, b.mp, b.np, b.kmax);
    float* U32 = reinterpret_cast<float*>(base + o_U32[i]);
    float* V32 = reinterpret_cast<float*>(base + o_V32[i]);
    float* isg = reinterpret_cast<float*>(base + o_isg[i]);
    asmb[i] = AssembleTask{t.U, t.Sigma, t.V, b.mp, b.np, b.kmax, q.r,
                           b.d_rank, b.d_rows, b.d_cols, pr.dLu, pr.dLv,
                           q.m, q.n, U32, V32, isg};
    const int64_t ncb = q.n - b.np, nrb = q.m - b.mp;
    sets[2 * i] = FilterSet{pr.dM, b.d_rows, b.mp, 1, b.d_cbar, (int)ncb,
                            pr.ldm, U32, b.mp, q.r, b.d_rank, nullptr, pr.dLv,
                            q.n, b.d_iters, q.filter_tol, q.filter_rho,
                            q.beta0_scale, q.beta_bar_ratio,
                            q.filter_max_iter, q.precision, q.lowp_iters};
    sets[2 * i + 1] = FilterSet{pr.dM, b.d_cols, b.np, pr.ldm, b.d_rbar,
                                (int)nrb, 1, V32, b.np, q.r, b.d_rank, isg,
                                pr.dLu, q.m, b.d_iters + ncb, q.filter_tol,
                                q.filter_rho, q.beta0_scale,
                                q.beta_bar_ratio, q.filter_max_iter,
                                q.precision, q.lowp_iters};
    sets[2 * i].skip = reinterpret_cast<const int32_t*>(base + o_skip) + i;
    sets[2 * i + 1].skip = sets[2 * i].skip;
  }
  // host blocks for the argument copies must outlive the async copies; the
  // handle keeps them
  h->h_gat.resize(sizeof(GatherTask) * count);
  h->h_asm.resize(sizeof(AssembleTask) * count);
  h->h_sargs.resize(seed_batched_args_bytes(count));
  h->h_filt.resize(fbytes);
  h->h_stask.resize(sizeof(SummaryTask) * count);
  SummaryTask* stask = reinterpret_cast<SummaryTask*>(h->h_stask.data());
  for (int i = 0; i < count; ++i) {
    const pcp_params& q = probs[i].params;
    const BatchInstance& b = h->inst[i];
    stask[i] = SummaryTask{seed_ctl_ptr_cta(b.d_work, b.mp, b.np, b.kmax),
                           b.d_iters, (q.m - b.mp) + (q.n - b.np), b.d_bad,
                           reinterpret_cast<int32_t*>(base + o_skip) + i,
                           b.mp, b.np, q.m, q.n, q.s_r, q.s_c,
                           (q.grow_seed && grow_gate && grow_gate[i]) ? 1 : 0};
  }
  h->d_summary = reinterpret_cast<BatchSummary*>(base + o_sum);
  pcp_status s;
  // Every argument block is copied before the first launch: a copy from
  // pageable host memory issued behind a running kernel would hold the
  // calling thread until that kernel ends (the server's scheduler thread
  // among them).  A plan's capture follows its direct run on the same
  // workspace: the blocks there already hold these bytes, so the graph
  // carries no host copies.
  if (!h->indices_ready) {
    if ((s = gather_batched_async(gat.data(), count, h->h_gat.data(),
                                  base + o_gat, st, true, false)) != PCP_OK ||
        (s = seed_pcp_batched_async(seeds.data(), count, h->h_sargs.data(),
                                    base + o_sargs, st, true, false)) !=
            PCP_OK ||
        (s = assemble_batched_async(asmb.data(), count, h->h_asm.data(),
                                    base + o_asm, st, true, false)) !=
            PCP_OK ||
        (s = l1_filter_batched_async(sets.data(), 2 * count,
                                     h->h_filt.data(), base + o_filt, st,
                                     true, false)) != PCP_OK)
      return s;
    PCP_CUDA(cudaMemcpyAsync(base + o_stask, stask,
                             sizeof(SummaryTask) * count,
                             cudaMemcpyHostToDevice, st));
  }
  if (timed) {
    for (cudaEvent_t& e : h->ev) PCP_CUDA(cudaEventCreate(&e));
    PCP_CUDA(cudaEventRecord(h->ev[0], st));
  }
  NvtxStages nvtx("pcp.batch.seed");
  if (!h->indices_ready) {
    const int bx = (int)std::min<int64_t>((widest + 255) / 256, 64);
    complement_batched_kernel<<<dim3(bx, count), 256, 0, st>>>(
        reinterpret_cast<const ComplementTask*>(base + o_ctask));
    PCP_CUDA(cudaGetLastError());
  }
  if ((s = gather_batched_async(gat.data(), count, h->h_gat.data(),
                                base + o_gat, st, false)) != PCP_OK)
    return s;
  if ((s = seed_pcp_batched_async(seeds.data(), count, h->h_sargs.data(),
                                  base + o_sargs, st, false)) != PCP_OK)
    return s;
  if ((s = assemble_batched_async(asmb.data(), count, h->h_asm.data(),
                                  base + o_asm, st, false)) != PCP_OK)
    return s;
  batch_gate_kernel<<<(count + 255) / 256, 256, 0, st>>>(
      reinterpret_cast<const SummaryTask*>(base + o_stask), count);
  PCP_CUDA(cudaGetLastError());
  if (timed) PCP_CUDA(cudaEventRecord(h->ev[1], st));
  nvtx.next("pcp.batch.filter");
  if ((s = l1_filter_batched_async(sets.data(), 2 * count, h->h_filt.data(),
                                   base + o_filt, st, false)) != PCP_OK)
    return s;
  if (timed) PCP_CUDA(cudaEventRecord(h->ev[2], st));
  nvtx.next("pcp.batch.spass");
  batch_summary_kernel<<<count, 256, 0, st>>>(
      reinterpret_cast<const SummaryTask*>(base + o_stask), h->d_summary);
  PCP_CUDA(cudaGetLastError());
  for (int i = 0; i < count; ++i) {
    const pcp_problem& pr = probs[i];
    if (!pr.dS) continue;
    s = pcp_spass(pr.dM, pr.ldm, pr.dLu, pr.params.m, pr.dLv, pr.params.n,
                  pr.params.r, pr.dS, pr.lds, pr.params.m, pr.params.n, st);
    if (s != PCP_OK) return s;
  }
  if (timed) PCP_CUDA(cudaEventRecord(h->ev[3], st));
  return PCP_OK;
}

pcp_status batch_finish(BatchHandle* h, pcp_info* infos, cudaStream_t st,
                        float batch_ms) {
  pcp_status first = PCP_OK;
  if (infos) {
    std::vector<BatchSummary> sum(h->count);
    PCP_CUDA(cudaMemcpyAsync(sum.data(), h->d_summary,
                             sizeof(BatchSummary) * h->count,
                             cudaMemcpyDeviceToHost, st));
    PCP_CUDA(cudaStreamSynchronize(st));
    float stage_ms[3] = {0.0f, 0.0f, 0.0f};
    if (h->ev[0])
      for (int q = 0; q < 3; ++q)
        cudaEventElapsedTime(&stage_ms[q], h->ev[q], h->ev[q + 1]);
    h->status.clear();
    h->skipped.assign(h->count, 0);
    for (int i = 0; i < h->count; ++i) {
      const pcp_params& q = h->probs[i].params;
      const BatchInstance& b = h->inst[i];
      const BatchSummary& u = sum[i];
      pcp_info& inf = infos[i];
      std::memset(&inf, 0, sizeof(inf));
      inf.rank = u.rank;
      inf.seed_iters = u.iters;
      inf.seed_residual = u.residual;
      inf.seed_m = b.mp;
      inf.seed_n = b.np;
      inf.seed_rank_raw = u.rank_raw;
      inf.problems = (q.m - b.mp) + (q.n - b.np);
      inf.lambda = b.lam_full;
      inf.filter_iters_max = u.iters_max;
      inf.problems_unconverged = u.unconverged;
      inf.filter_iters_mean =
          inf.problems > 0 ? (double)u.iters_sum / (double)inf.problems : 0.0;
      inf.rank_ok = (u.rank_raw >= 1 &&
                     (double)b.mp / u.rank_raw >= q.s_r - 1e-9 &&
                     (double)b.np / u.rank_raw >= q.s_c - 1e-9)
                        ? 1
                        : 0;
      inf.t_total_ms = batch_ms;
      inf.t_seed_ms = stage_ms[0];   // stage times of the whole batch
      inf.t_filter_ms = stage_ms[1];
      inf.t_spass_ms = stage_ms[2];
      pcp_status si = PCP_OK;
      if (u.bad) si = PCP_ERR_NONFINITE;
      else if (!u.converged) si = PCP_ERR_SEED_NOCONV;
      else if (!inf.rank_ok) si = PCP_ERR_RANK_TEST;
      else if (u.unconverged) si = PCP_ERR_FILTER_NOCONV;
      inf.status = (int32_t)si;
      h->skipped[i] = u.skipped ? 1 : 0;
      if (si != PCP_OK && first == PCP_OK) {
        first = si;
        set_error("batch instance %d: status %d (rank %d, raw %d, iters %d)",
                  i, (int)si, u.rank, u.rank_raw, u.iters);
      }
      h->status.push_back(si);
    }
  }
  for (cudaEvent_t& e : h->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  if (h->d_base && !h->prealloc) {
    PCP_CUDA(cudaFreeAsync(h->d_base, st));
    h->d_base = nullptr;
  }
  return first;
}

}  // namespace pcp

namespace {

// One round of the batched solve: launch, wait, and fill one pcp_info per
// instance; with gate, instances whose seed fails Eq. rank_test and will
// grow skip their filters (h->skipped marks them).
pcp_status batch_round(int count, const pcp_problem* probs, pcp_info* infos,
                       cudaStream_t st, bool gate, std::vector<char>* skipped,
                       float* total_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (infos) {
    PCP_CUDA(cudaEventCreate(&e0));
    PCP_CUDA(cudaEventCreate(&e1));
    PCP_CUDA(cudaEventRecord(e0, st));
  }
  std::vector<unsigned char> g(gate ? count : 0, 1);
  pcp::BatchHandle h;
  pcp_status s = pcp::batch_launch(count, probs, st, &h, infos != nullptr,
                                   gate ? g.data() : nullptr);
  if (s != PCP_OK) {
    if (h.d_base) cudaFreeAsync(h.d_base, st);
    for (cudaEvent_t e : h.ev)
      if (e) cudaEventDestroy(e);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return s;
  }
  float ms = 0.0f;
  if (infos) {
    PCP_CUDA(cudaEventRecord(e1, st));
    PCP_CUDA(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  s = pcp::batch_finish(&h, infos, st, ms);
  if (skipped) *skipped = h.skipped;
  if (total_ms) *total_ms = ms;
  return s;
}

}  // namespace

extern "C" pcp_status pcp_l1filter_batch(int32_t count,
                                         const pcp_problem* probs,
                                         pcp_info* infos, void* stream) {
  PCP_ARG(count >= 0, "pcp_l1filter_batch: count < 0");
  if (count == 0) return PCP_OK;
  PCP_ARG(probs, "pcp_l1filter_batch: null problems");
  cudaStream_t st = (cudaStream_t)stream;
  // Without infos nothing grows (Section 3.5 needs the seed's rank), so the
  // filters are never gated off.
  if (!infos)
    return batch_round(count, probs, nullptr, st, false, nullptr, nullptr);
  // Section 3.5 for the instances that ask for it: a seed failing Eq.
  // rank_test grows to (s_r r') x (s_c r') along the same orders, and the
  // grown instances run again as one batch, until none is left to grow.
  // Each round gates off the filters of the seeds that are about to grow.
  std::vector<pcp_problem> cur(probs, probs + count);
  std::vector<std::vector<int64_t>> orders(2 * (size_t)count);
  std::vector<int> act(count);
  std::iota(act.begin(), act.end(), 0);
  for (int round = 0; round < 17 && !act.empty(); ++round) {
    std::vector<pcp_problem> g;
    for (int i : act) g.push_back(cur[i]);
    std::vector<pcp_info> gi(g.size());
    std::vector<char> skipped;
    // the last round grows nothing more, so its filters all run
    const bool gate = round < 16;
    pcp_status s = batch_round((int)g.size(), g.data(), gi.data(), st, gate,
                               &skipped, nullptr);
    if (s == PCP_ERR_ARG || s == PCP_ERR_CUDA || s == PCP_ERR_NOMEM ||
        s == PCP_ERR_UNSUPPORTED)
      return s;
    std::vector<int> next, redo;
    for (size_t u = 0; u < act.size(); ++u) {
      const int i = act[u];
      if (round > 0) gi[u].t_total_ms += infos[i].t_total_ms;
      infos[i] = gi[u];
      const pcp_params& q = cur[i].params;
      int gm = 0, gn = 0;
      const bool grows = q.grow_seed &&
                         infos[i].status == PCP_ERR_RANK_TEST &&
                         pcp::grown_seed_size(q, infos[i], &gm, &gn);
      if (!grows) {
        // a skipped instance the host does not grow runs again in full
        if (u < skipped.size() && skipped[u]) redo.push_back(i);
        continue;
      }
      if (orders[2 * i].empty()) {
        orders[2 * i] =
            q.row_order ? std::vector<int64_t>(q.row_order, q.row_order + q.m)
                        : pcp::sample_order(q.m, q.rng_seed);
        orders[2 * i + 1] =
            q.col_order ? std::vector<int64_t>(q.col_order, q.col_order + q.n)
                        : pcp::sample_order(q.n, q.rng_seed ^ 0xC01C01C0ull);
      }
      cur[i].params.seed_m = gm;
      cur[i].params.seed_n = gn;
      cur[i].params.row_order = orders[2 * i].data();
      cur[i].params.col_order = orders[2 * i + 1].data();
      next.push_back(i);
    }
    if (!redo.empty()) {
      std::vector<pcp_problem> rp;
      for (int i : redo) rp.push_back(cur[i]);
      std::vector<pcp_info> ri(rp.size());
      s = batch_round((int)rp.size(), rp.data(), ri.data(), st, false,
                      nullptr, nullptr);
      if (s == PCP_ERR_ARG || s == PCP_ERR_CUDA || s == PCP_ERR_NOMEM ||
          s == PCP_ERR_UNSUPPORTED)
        return s;
      for (size_t u = 0; u < redo.size(); ++u) {
        ri[u].t_total_ms += infos[redo[u]].t_total_ms;
        infos[redo[u]] = ri[u];
      }
    }
    act.swap(next);
  }
  pcp_status s = PCP_OK;
  for (int i = 0; i < count && s == PCP_OK; ++i)
    s = (pcp_status)infos[i].status;
  return s;
}

// ---------------------------------------------------------------------------
// Batch plans: the batched solve with its workspace allocated once and its
// launches captured into a CUDA graph that every run replays.
struct pcp_batch_plan {
  std::vector<pcp_problem> probs;            // the instances, seeds fixed
  std::vector<std::vector<int64_t>> arrays;  // host index arrays they use
  pcp::BatchHandle h;                         // workspace, argument blocks
  cudaStream_t cap_st = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" void pcp_batch_plan_destroy(pcp_batch_plan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->cap_st) cudaStreamDestroy(P->cap_st);
  if (P->h.d_base) cudaFree(P->h.d_base);
  delete P;
}

extern "C" pcp_status pcp_l1filter_batch_plan(int32_t count,
                                              const pcp_problem* probs,
                                              void* stream,
                                              pcp_batch_plan** out) {
  PCP_ARG(out, "pcp_l1filter_batch_plan: null output");
  *out = nullptr;
  PCP_ARG(count >= 1 && count <= 65535 && probs,
          "pcp_l1filter_batch_plan: count %d outside [1, 65535] or null "
          "problems", count);
  cudaStream_t st = (cudaStream_t)stream;
  // one batched solve settles every instance's seed (Section 3.5 growth
  // where asked for); the plan keeps the seed each instance ended with
  std::vector<pcp_info> inf(count);
  pcp_status s = pcp_l1filter_batch(count, probs, inf.data(), stream);
  if (s == PCP_ERR_ARG || s == PCP_ERR_CUDA || s == PCP_ERR_NOMEM ||
      s == PCP_ERR_UNSUPPORTED || s == PCP_ERR_TIMEOUT)
    return s;
  pcp_batch_plan* P = new pcp_batch_plan();
  P->probs.assign(probs, probs + count);
  P->arrays.reserve(4 * (size_t)count);
  auto keep = [&](const int64_t* v, int64_t len) -> const int64_t* {
    if (!v) return nullptr;
    P->arrays.emplace_back(v, v + len);
    return P->arrays.back().data();
  };
  for (int i = 0; i < count; ++i) {
    pcp_params& q = P->probs[i].params;
    const int mp0 = q.seed_m > 0 ? q.seed_m : (int)std::llround(q.s_r * q.r);
    const int np0 = q.seed_n > 0 ? q.seed_n : (int)std::llround(q.s_c * q.r);
    const bool grown = q.grow_seed && (inf[i].seed_m != mp0 ||
                                       inf[i].seed_n != np0);
    if (grown) {
      // the growth took prefixes of these orders (the library's sampling
      // order when none was given)
      if (!q.row_order) {
        P->arrays.push_back(pcp::sample_order(q.m, q.rng_seed));
        q.row_order = P->arrays.back().data();
      } else {
        q.row_order = keep(q.row_order, q.m);
      }
      if (!q.col_order) {
        P->arrays.push_back(pcp::sample_order(q.n, q.rng_seed ^ 0xC01C01C0ull));
        q.col_order = P->arrays.back().data();
      } else {
        q.col_order = keep(q.col_order, q.n);
      }
      q.seed_m = (int32_t)inf[i].seed_m;
      q.seed_n = (int32_t)inf[i].seed_n;
    } else {
      const int mp = mp0, np = np0;
      q.seed_rows = keep(q.seed_rows, mp);
      q.seed_cols = keep(q.seed_cols, np);
      q.row_order = keep(q.row_order, q.m);
      q.col_order = keep(q.col_order, q.n);
    }
    q.grow_seed = 0;
  }
  pcp::BatchHandle& h = P->h;
  h.size_only = true;
  s = pcp::batch_launch(count, P->probs.data(), st, &h, false);
  if (s != PCP_OK) {
    pcp_batch_plan_destroy(P);
    return s;
  }
  h.size_only = false;
  cudaError_t e = cudaMalloc(&h.d_base, h.bytes);
  if (e != cudaSuccess) {
    h.d_base = nullptr;
    pcp_batch_plan_destroy(P);
    return pcp::cuda_fail(e, "cudaMalloc(batch plan workspace)", __FILE__,
                          __LINE__);
  }
  h.prealloc = true;
  // a direct run uploads the index sets and settles one-time set-up, then
  // the same launches are captured (without the index uploads)
  // The direct run must reproduce the settling call instance by instance
  // (same seeds, kernels and reduction orders): a difference means the
  // preallocated workspace is not what the launches expect.
  std::vector<pcp_info> inf2(count);
  s = pcp::batch_launch(count, P->probs.data(), st, &h, false);
  if (s == PCP_OK) {
    const pcp_status s2 = pcp::batch_finish(&h, inf2.data(), st, 0.0f);
    if (s2 == PCP_ERR_ARG || s2 == PCP_ERR_CUDA || s2 == PCP_ERR_TIMEOUT)
      s = s2;
  }
  for (int i = 0; s == PCP_OK && i < count; ++i)
    if (inf2[i].status != inf[i].status ||
        inf2[i].seed_iters != inf[i].seed_iters ||
        inf2[i].rank != inf[i].rank) {
      pcp::set_error(
          "pcp_l1filter_batch_plan: instance %d of the plan's direct run "
          "differs from the batched call (status %d / %d, seed iterations "
          "%d / %d, rank %d / %d)", i, (int)inf2[i].status,
          (int)inf[i].status, (int)inf2[i].seed_iters,
          (int)inf[i].seed_iters, (int)inf2[i].rank, (int)inf[i].rank);
      s = PCP_ERR_CUDA;
    }
  if (s == PCP_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess)
    s = pcp::cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  if (s == PCP_OK &&
      (e = cudaStreamCreateWithFlags(&P->cap_st, cudaStreamNonBlocking)) !=
          cudaSuccess)
    s = pcp::cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
  if (s != PCP_OK) {
    pcp_batch_plan_destroy(P);
    return s;
  }
  h.indices_ready = true;
  if ((e = cudaStreamBeginCapture(P->cap_st,
                                  cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess) {
    pcp_batch_plan_destroy(P);
    return pcp::cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
  }
  s = pcp::batch_launch(count, P->probs.data(), P->cap_st, &h, false);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(P->cap_st, &g);
  if (s == PCP_OK && e == cudaSuccess && g)
    e = cudaGraphInstantiate(&P->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (s != PCP_OK || e != cudaSuccess || !P->exec) {
    if (s == PCP_OK)
      s = pcp::cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown,
                         "batch plan graph capture", __FILE__, __LINE__);
    pcp_batch_plan_destroy(P);
    return s;
  }
  *out = P;
  return PCP_OK;
}

extern "C" pcp_status pcp_l1filter_batch_run(pcp_batch_plan* P,
                                             pcp_info* infos, void* stream) {
  PCP_ARG(P && P->exec, "pcp_l1filter_batch_run: null plan");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (infos) {
    PCP_CUDA(cudaEventCreate(&e0));
    PCP_CUDA(cudaEventCreate(&e1));
    PCP_CUDA(cudaEventRecord(e0, st));
  }
  PCP_CUDA(cudaGraphLaunch(P->exec, st));
  if (!infos) return PCP_OK;
  PCP_CUDA(cudaEventRecord(e1, st));
  PCP_CUDA(cudaEventSynchronize(e1));
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return pcp::batch_finish(&P->h, infos, st, ms);
}
