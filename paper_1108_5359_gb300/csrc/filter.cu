// l1 filtering (Section 3.2): Algorithm 1 on many independent problems.
//
// Problem j solves  min ||e||_1  s.t.  x_j = A z + e  (Eq. l1g, one column),
// A = U^s (column filter, Eq. l1c') or V^s (row filter, Eq. l1r'), with the
// ADM steps of Algorithm 1:
//   e_{k+1} = S_{1/beta_k}(x - A z_k + y_k/beta_k)
//   z_{k+1} = A^T (x - e_{k+1} + y_k/beta_k)
//   y_{k+1} = y_k + beta_k (x - A z_{k+1} - e_{k+1}),
//   beta_{k+1} = min(rho beta_k, beta_bar)
// stopping when ||x - A z_k - e_k||_inf is below eps times ||x - e_k||_inf
// (floored at kStopNormFloor ||x||_inf; the paper divides by ||x||_inf).
// Each problem runs its own instance (own beta_0 = beta0_scale/||x||_inf and
// stop test); the problems are independent (Section 3.2), which is the grid
// decomposition.
//
// FP32 form of the same iteration: the state holds d = x - e instead of e.
// With v = x - A z_k + y_k/beta_k and c = v - S_{1/beta_k}(v) (v clipped to
// +-1/beta_k), e_{k+1} = v - c gives
//   d_{k+1} = A z_k - y_k/beta_k + c,   x - e_{k+1} + y_k/beta_k = A z_k + c,
//   residual x - A z_{k+1} - e_{k+1} = d_{k+1} - A z_{k+1},
// so no step subtracts two copies of a large outlier: x enters only through
// v, which is clipped.  (With e stored, an outlier of size |x_i| leaves an
// FP32 rounding of ~|x_i| 2^-24 in z and in the residual.)
//
// GB300 mapping (FP32 SIMT form):
//   * one CTA = 8 warps = 32 problems; lane l of every warp works on problem
//     l, warp w owns the entries t = w, w+8, w+16, ... of that problem;
//   * x, y, d of the owned entries live in registers for the whole solve,
//     A (p x r) is staged once into shared memory (row-major, zero padded to
//     RMAX columns) and read as warp-broadcast float4;
//   * one pass over the owned rows per iteration fuses A z (for the
//     residual and dual step), the next shrinkage, and the partial products
//     of A^T v for the next z; a cross-warp reduction through shared memory
//     then yields z for every lane (deterministic order);
//   * the infinity-norm stop test is a cross-warp max; a problem that has
//     converged writes its z and is frozen (its lanes keep computing but
//     never write again) so every problem stops exactly at its own test.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace pcp {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;


template <int RMAX>
__device__ __forceinline__ void load_arow(const float* __restrict__ As, int t,
                                          float (&a)[RMAX]) {
  const float4* row = reinterpret_cast<const float4*>(As + t * RMAX);
#pragma unroll
  for (int q = 0; q < RMAX / 4; ++q) {
    float4 v = row[q];
    a[4 * q + 0] = v.x;
    a[4 * q + 1] = v.y;
    a[4 * q + 2] = v.z;
    a[4 * q + 3] = v.w;
  }
}

// Algorithm 1 on the 32 problems of tile `tile` of set `a`.
template <int SPT, int RMAX>
__device__ __forceinline__ void adm_f32_tile(const FilterArgs& a,
                                             const int tile) {
  extern __shared__ __align__(16) float smem[];
  float* As = smem;                                 // [kWarps*SPT][RMAX]
  float* red = As + kWarps * SPT * RMAX;            // [kWarps][RMAX][32]
  float* zsh = red + kWarps * RMAX * 32;            // [RMAX][32]
  float* mxs = zsh + RMAX * 32;                     // [kWarps][32]
  float* mds = mxs + kWarps * 32;                   // [kWarps][32]

  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int j = tile * 32 + lane;
  const bool valid = j < a.N;
  const int p = a.p;
  int reff = a.r;
  if (a.d_rank) reff = min(max(*a.d_rank, 0), a.r);

  // Stage A (p x r, column-major, ld lda) as row-major [t][k], zero padded.
  for (int idx = threadIdx.x; idx < kWarps * SPT * RMAX; idx += kThreads) {
    const int t = idx / RMAX, k = idx - t * RMAX;
    As[idx] = (t < p && k < reff) ? a.A[t + (int64_t)k * a.lda] : 0.0f;
  }

  // Load the owned entries of x_j.
  float x[SPT], y[SPT], d[SPT];  // d = x - e
  const int64_t qoff = valid ? (int64_t)a.qidx[j] * a.sq : 0;
  float xm = 0.0f;
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    const int t = w + kWarps * s;
    float v = 0.0f;
    if (valid && t < p) v = __ldg(a.M + (int64_t)a.pidx[t] * a.sp + qoff);
    x[s] = v;
    y[s] = 0.0f;
    xm = fmaxf(xm, fabsf(v));
  }
  mxs[w * 32 + lane] = xm;
  __syncthreads();
  float xinf = 0.0f;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) xinf = fmaxf(xinf, mxs[q * 32 + lane]);
  // A zero column has the exact solution z = 0 and takes no iteration.
  bool done = !(xinf > 0.0f);
  const float inv_xinf = done ? 0.0f : 1.0f / xinf;
  float beta = done ? 1.0f : a.beta0_scale * inv_xinf;
  const float beta_bar = beta * a.beta_bar_ratio;

  // Iteration 1, step 1 with z_0 = 0, y_0 = 0: e_1 = S_{1/beta_0}(x), so
  // d_1 = x - e_1 = clip(x, 1/beta_0); partial products of z_1 = A^T d_1.
  float acc[RMAX];
#pragma unroll
  for (int k = 0; k < RMAX; ++k) acc[k] = 0.0f;
  {
    const float ib = 1.0f / beta;
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int t = w + kWarps * s;
      if (t < p) {
        d[s] = clip(x[s], ib);
        const float v = d[s];
        float ar[RMAX];
        load_arow<RMAX>(As, t, ar);
#pragma unroll
        for (int k = 0; k < RMAX; ++k) acc[k] = fmaf(ar[k], v, acc[k]);
      } else {
        d[s] = 0.0f;
      }
    }
  }
  if (done && valid && w == 0) {
    for (int k = 0; k < a.r; ++k) a.Z[(int64_t)a.qidx[j] + k * a.ldz] = 0.0f;
    if (a.iters_out) a.iters_out[j] = 0;
  }
  if (!valid) done = true;

  float z[RMAX];
  int iter = 0;
  while (true) {
    // z_{k+1}: reduce the partial products across the 8 warps.
#pragma unroll
    for (int k = 0; k < RMAX; ++k) red[(w * RMAX + k) * 32 + lane] = acc[k];
    __syncthreads();
    for (int k = w; k < RMAX; k += kWarps) {
      float sacc = 0.0f;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) sacc += red[(q * RMAX + k) * 32 + lane];
      zsh[k * 32 + lane] = sacc;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RMAX; ++k) z[k] = zsh[k * 32 + lane];
    ++iter;

    // One pass over the owned rows: A z_{k+1}, residual, dual step, then
    // step 1 and the A^T partial products of the next iteration.
    const float bn = fminf(a.rho * beta, beta_bar);
    const float ibn = 1.0f / bn;
    float rmax = 0.0f, dmax = 0.0f;
#pragma unroll
    for (int k = 0; k < RMAX; ++k) acc[k] = 0.0f;
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int t = w + kWarps * s;
      if (t < p) {
        float ar[RMAX];
        load_arow<RMAX>(As, t, ar);
        float az = 0.0f;
#pragma unroll
        for (int k = 0; k < RMAX; ++k) az = fmaf(ar[k], z[k], az);
        const float res = d[s] - az;
        rmax = fmaxf(rmax, fabsf(res));
        dmax = fmaxf(dmax, fabsf(d[s]));
        y[s] = fmaf(beta, res, y[s]);
        const float yb = y[s] * ibn;
        const float c = clip(x[s] - az + yb, ibn);
        d[s] = az - yb + c;
        const float v = az + c;
#pragma unroll
        for (int k = 0; k < RMAX; ++k) acc[k] = fmaf(ar[k], v, acc[k]);
      }
    }
    beta = bn;
    mxs[w * 32 + lane] = rmax;
    mds[w * 32 + lane] = dmax;
    __syncthreads();
    float rm = 0.0f, dm = 0.0f;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      rm = fmaxf(rm, mxs[q * 32 + lane]);
      dm = fmaxf(dm, mds[q * 32 + lane]);
    }
    const bool conv_now =
        !done && (rm < a.eps * fmaxf(dm, kStopNormFloor * xinf));
    const bool out_now = conv_now || (!done && iter >= a.max_iter);
    if (out_now && w == 0) {
      const int64_t row = a.qidx[j];
#pragma unroll
      for (int k = 0; k < RMAX; ++k) {
        if (k < a.r) {
          const float sc = a.scale ? a.scale[k] : 1.0f;
          a.Z[row + k * a.ldz] = (k < reff) ? z[k] * sc : 0.0f;
        }
      }
      if (a.iters_out) a.iters_out[j] = conv_now ? iter : -iter;
    }
    done = done || out_now;
    if (__syncthreads_and(done)) break;
  }
}

template <int SPT, int RMAX>
__global__ void __launch_bounds__(kThreads, 1)
    adm_f32_kernel(const FilterArgs a) {
  adm_f32_tile<SPT, RMAX>(a, blockIdx.x);
}

// Batched form: CTA b runs tile tiles[2b+1] of set tiles[2b].
template <int SPT, int RMAX>
__global__ void __launch_bounds__(kThreads, 1)
    adm_f32_batched_kernel(const FilterArgs* __restrict__ sets,
                           const int32_t* __restrict__ tiles) {
  const FilterArgs a = sets[tiles[2 * blockIdx.x]];
  if (a.skip != nullptr && *a.skip != 0) return;  // whole CTA, one set
  adm_f32_tile<SPT, RMAX>(a, tiles[2 * blockIdx.x + 1]);
}

template <int SPT, int RMAX>
size_t adm_smem_bytes() {
  return sizeof(float) * ((size_t)kWarps * SPT * RMAX +
                          (size_t)kWarps * RMAX * 32 + (size_t)RMAX * 32 +
                          (size_t)2 * kWarps * 32);
}

template <int SPT, int RMAX>
cudaError_t launch_adm(const FilterArgs& a, cudaStream_t st) {
  const size_t smem = adm_smem_bytes<SPT, RMAX>();
  // per process (the attribute is per function); host threads may race to
  // set it, which is harmless: every setter writes the same value
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(
        adm_f32_kernel<SPT, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)smem);
    if (e != cudaSuccess) return e;
    configured.store(true, std::memory_order_release);
  }
  const int grid = (a.N + 31) / 32;
  adm_f32_kernel<SPT, RMAX><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int SPT>
cudaError_t dispatch_r(const FilterArgs& a, cudaStream_t st) {
  if (a.r <= 8) return launch_adm<SPT, 8>(a, st);
  if (a.r <= 16) return launch_adm<SPT, 16>(a, st);
  if (a.r <= 24) return launch_adm<SPT, 24>(a, st);
  if (a.r <= 32) return launch_adm<SPT, 32>(a, st);
  return cudaErrorInvalidValue;
}

// Batched launches: the shape class of a set is (SPT index, RMAX index).
int shape_class(int p, int r) {
  const int si = p <= 64 ? 0 : (p <= 128 ? 1 : 2);
  return si * 4 + (r - 1) / 8;
}

template <int SPT, int RMAX>
cudaError_t launch_adm_batched(const FilterArgs* d_sets, const int32_t* d_tiles,
                               int ntiles, cudaStream_t st) {
  const size_t smem = adm_smem_bytes<SPT, RMAX>();
  static std::atomic<bool> configured{false};
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(
        adm_f32_batched_kernel<SPT, RMAX>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured.store(true, std::memory_order_release);
  }
  adm_f32_batched_kernel<SPT, RMAX><<<ntiles, kThreads, smem, st>>>(d_sets,
                                                                    d_tiles);
  return cudaGetLastError();
}

template <int SPT>
cudaError_t dispatch_batched_r(int ri, const FilterArgs* d_sets,
                               const int32_t* d_tiles, int ntiles,
                               cudaStream_t st) {
  switch (ri) {
    case 0: return launch_adm_batched<SPT, 8>(d_sets, d_tiles, ntiles, st);
    case 1: return launch_adm_batched<SPT, 16>(d_sets, d_tiles, ntiles, st);
    case 2: return launch_adm_batched<SPT, 24>(d_sets, d_tiles, ntiles, st);
    case 3: return launch_adm_batched<SPT, 32>(d_sets, d_tiles, ntiles, st);
  }
  return cudaErrorInvalidValue;
}

// SIMT classes 0..11, tensor-core classes 12..35 (12 + tc_shape_class)
constexpr int kSimtClasses = 12;
constexpr int kShapeClasses = kSimtClasses + 24;

size_t args_block_bytes(int nsets) {
  return (sizeof(FilterArgs) * (size_t)nsets + 255) / 256 * 256;
}

}  // namespace

// ---- kernel choice for PCP_FP32 ---------------------------------------------
// PCP_FP32 asks for FP32 accuracy without naming a kernel.  For shapes both
// kernels take (p <= 256, r <= 32) the choice is read from a table compiled
// into the library (filter_table.inc, written by a tuning run that timed
// both kernels per class), so it is a function of the shape alone: the same
// input gives the same bits in every process and in the single, batched
// and served forms.
namespace {
#include "filter_table.inc"

int tune_slot_p(int p) { return p <= 64 ? 0 : (p <= 128 ? 1 : 2); }
int tune_slot_r(int r) { return (r - 1) / 8; }
}  // namespace

bool filter_uses_simt(int precision, int p, int r) {
  if (p > 256 || r > 32) return false;
  if (precision == PCP_FP32_SIMT) return true;
  if (precision != PCP_FP32) return false;
  return kFp32KernelTable[tune_slot_p(p)][tune_slot_r(r)] == PCP_KERNEL_SIMT;
}

size_t filter_batch_bytes(const FilterSet* sets, int nsets) {
  size_t tiles = 0;
  for (int i = 0; i < nsets; ++i) tiles += (size_t)(sets[i].N + 15) / 16;
  return args_block_bytes(nsets) + 8 * tiles + 16 * kShapeClasses;
}

pcp_status l1_filter_batched_async(const FilterSet* sets, int nsets,
                                   void* h_buf, void* d_buf,
                                   cudaStream_t st, bool upload,
                                   bool launch) {
  if (nsets <= 0) return PCP_OK;
  char* hb = static_cast<char*>(h_buf);
  FilterArgs* ha = reinterpret_cast<FilterArgs*>(hb);
  std::vector<std::vector<int32_t>> by_class(kShapeClasses);
  for (int i = 0; i < nsets; ++i) {
    const FilterSet& f = sets[i];
    PCP_ARG(f.p >= 1 && f.p <= 512 && f.r >= 1 && f.r <= 64 && f.N >= 0,
            "batched filter: set %d has p=%d r=%d N=%d", i, f.p, f.r, f.N);
    const bool simt = filter_uses_simt(f.precision, f.p, f.r);
    FilterArgs a;
    a.M = f.M;
    a.pidx = f.pidx;
    a.p = f.p;
    a.sp = f.sp;
    a.qidx = f.qidx;
    a.N = f.N;
    a.sq = f.sq;
    a.A = f.A;
    a.lda = f.lda;
    a.r = f.r;
    a.d_rank = f.d_rank;
    a.scale = f.scale;
    a.Z = f.Z;
    a.ldz = f.ldz;
    a.eps = (float)f.eps;
    a.rho = (float)f.rho;
    a.beta0_scale = (float)f.beta0_scale;
    a.beta_bar_ratio = (float)f.beta_bar_ratio;
    a.max_iter = f.max_iter;
    const bool refined = f.precision == PCP_TF32_REFINED ||
                         f.precision == PCP_BF16_REFINED;
    a.lowp_iters = refined ? f.lowp_iters : 0;
    a.lowp_bf16 = f.precision == PCP_BF16_REFINED;
    a.iters_out = f.iters_out;
    a.skip = f.skip;
    std::memcpy(ha + i, &a, sizeof(a));
    const int cls = simt ? shape_class(f.p, f.r)
                         : kSimtClasses + tc_shape_class(f.p, f.r);
    const int per_tile = simt ? 32 : 16;
    std::vector<int32_t>& t = by_class[cls];
    for (int b = 0; b < (f.N + per_tile - 1) / per_tile; ++b) {
      t.push_back(i);
      t.push_back(b);
    }
  }
  size_t off = args_block_bytes(nsets);
  size_t used = off;
  std::vector<size_t> class_off(kShapeClasses, 0);
  for (int c = 0; c < kShapeClasses; ++c) {
    if (by_class[c].empty()) continue;
    class_off[c] = used;
    std::memcpy(hb + used, by_class[c].data(), 4 * by_class[c].size());
    used += (4 * by_class[c].size() + 15) / 16 * 16;
  }
  if (upload)
    PCP_CUDA(cudaMemcpyAsync(d_buf, h_buf, used, cudaMemcpyHostToDevice, st));
  if (!launch) return PCP_OK;
  char* db = static_cast<char*>(d_buf);
  const FilterArgs* d_sets = reinterpret_cast<const FilterArgs*>(db);
  for (int c = 0; c < kShapeClasses; ++c) {
    if (by_class[c].empty()) continue;
    const int ntiles = (int)(by_class[c].size() / 2);
    const int32_t* d_tiles = reinterpret_cast<const int32_t*>(db + class_off[c]);
    cudaError_t e;
    if (c >= kSimtClasses) {
      e = l1_filter_tc_batched_launch(c - kSimtClasses, d_sets, d_tiles,
                                      ntiles, st);
      if (e != cudaSuccess)
        return cuda_fail(e, "adm_tc_batched_kernel launch", __FILE__,
                         __LINE__);
      continue;
    }
    const int si = c / 4, ri = c % 4;
    if (si == 0)
      e = dispatch_batched_r<8>(ri, d_sets, d_tiles, ntiles, st);
    else if (si == 1)
      e = dispatch_batched_r<16>(ri, d_sets, d_tiles, ntiles, st);
    else
      e = dispatch_batched_r<32>(ri, d_sets, d_tiles, ntiles, st);
    if (e != cudaSuccess)
      return cuda_fail(e, "adm_f32_batched_kernel launch", __FILE__, __LINE__);
  }
  return PCP_OK;
}

}  // namespace pcp

extern "C" pcp_status pcp_l1_filter(
    const float* dM, const int32_t* d_pidx, int32_t p, int64_t sp,
    const int32_t* d_qidx, int32_t N, int64_t sq, const float* dA, int32_t lda,
    int32_t r, const int32_t* d_rank, const float* d_scale, float* dZ,
    int64_t ldz, double eps, double rho, double beta0_scale,
    double beta_bar_ratio, int32_t max_iter, int32_t precision,
    int32_t lowp_iters, int32_t* d_iters, void* stream) {
  PCP_ARG(p >= 1 && p <= 512, "pcp_l1_filter: p=%d outside [1, 512]", p);
  PCP_ARG(r >= 1 && r <= 64, "pcp_l1_filter: r=%d outside [1, 64]", r);
  PCP_ARG(N >= 0, "pcp_l1_filter: N=%d < 0", N);
  PCP_ARG(lda >= p, "pcp_l1_filter: lda=%d < p=%d", lda, p);
  PCP_ARG(ldz >= 1, "pcp_l1_filter: ldz < 1");
  PCP_ARG(eps > 0 && rho > 1 && beta0_scale > 0 && beta_bar_ratio >= 1,
          "pcp_l1_filter: need eps > 0, rho > 1, beta0_scale > 0, "
          "beta_bar_ratio >= 1");
  PCP_ARG(max_iter >= 1, "pcp_l1_filter: max_iter < 1");
  PCP_ARG(lowp_iters >= 0, "pcp_l1_filter: lowp_iters < 0");
  PCP_ARG(precision >= PCP_FP32 && precision <= PCP_FP32_SIMT,
          "pcp_l1_filter: unknown precision %d", precision);
  PCP_ARG(precision != PCP_FP32_SIMT || (p <= 256 && r <= 32),
          "pcp_l1_filter: the SIMT form takes p <= 256 and r <= 32 "
          "(p=%d r=%d)", p, r);
  if (precision == PCP_FP64) {
    pcp::set_error("pcp_l1_filter: precision %d not built", precision);
    return PCP_ERR_UNSUPPORTED;
  }
  if (N == 0) return PCP_OK;
  PCP_ARG(dM && d_pidx && d_qidx && dA && dZ, "pcp_l1_filter: null pointer");
  pcp::FilterArgs a;
  a.skip = nullptr;
  a.M = dM;
  a.pidx = d_pidx;
  a.p = p;
  a.sp = sp;
  a.qidx = d_qidx;
  a.N = N;
  a.sq = sq;
  a.A = dA;
  a.lda = lda;
  a.r = r;
  a.d_rank = d_rank;
  a.scale = d_scale;
  a.Z = dZ;
  a.ldz = ldz;
  a.eps = (float)eps;
  a.rho = (float)rho;
  a.beta0_scale = (float)beta0_scale;
  a.beta_bar_ratio = (float)beta_bar_ratio;
  a.max_iter = max_iter;
  const bool refined =
      precision == PCP_TF32_REFINED || precision == PCP_BF16_REFINED;
  a.lowp_iters = refined ? lowp_iters : 0;
  a.lowp_bf16 = precision == PCP_BF16_REFINED;
  a.iters_out = d_iters;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  auto run_simt = [&]() {
    if (p <= 64) return pcp::dispatch_r<8>(a, st);
    if (p <= 128) return pcp::dispatch_r<16>(a, st);
    return pcp::dispatch_r<32>(a, st);
  };
  if (pcp::filter_uses_simt(precision, p, r)) {
    if ((e = run_simt()) != cudaSuccess)
      return pcp::cuda_fail(e, "adm_f32_kernel launch", __FILE__, __LINE__);
  } else {
    e = pcp::l1_filter_tc_launch(a, st);
    if (e != cudaSuccess)
      return pcp::cuda_fail(e, "adm_tc_kernel launch", __FILE__, __LINE__);
  }
  return PCP_OK;
}

extern "C" int32_t pcp_l1_filter_kernel(int32_t p, int32_t r,
                                        int32_t precision) {
  PCP_ARG(p >= 1 && p <= 512 && r >= 1 && r <= 64,
          "pcp_l1_filter_kernel: p=%d r=%d outside [1, 512] x [1, 64]", p, r);
  PCP_ARG(precision >= PCP_FP32 && precision <= PCP_FP32_SIMT &&
              precision != PCP_FP64,
          "pcp_l1_filter_kernel: precision %d not available", precision);
  PCP_ARG(precision != PCP_FP32_SIMT || (p <= 256 && r <= 32),
          "pcp_l1_filter_kernel: the SIMT form takes p <= 256 and r <= 32");
  return pcp::filter_uses_simt(precision, p, r) ? PCP_KERNEL_SIMT
                                                : PCP_KERNEL_TENSOR;
}
