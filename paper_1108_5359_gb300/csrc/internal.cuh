// Internal (not exported) entry points shared between translation units.
#pragma once

#include "common.cuh"

namespace pcp {

// Control block of one seed PCP solve (device memory, start of its
// workspace): barrier state, status and diagnostics.
struct SeedCtl {
  unsigned int bar_count;  // grid barrier arrivals since the launch
  int fin_sweeps;          // Jacobi sweeps of the final FP64 SVD of the core
  int error;
  int iters;
  int rank;
  int converged;
  int k_final;
  int rank_raw;
  int ntrace;
  int jsweeps;     // total Jacobi sweeps (block 0), for tracing
  int jpath[3];    // Rayleigh-Ritz steps by form: first-order, cluster, full
  long long jcyc[4];  // block 0 Jacobi cycles: angles, A, V, end-of-round
  long long sub[8];   // block 0 sub-step cycle counters (tracing)
  double residual;
  double sigma1;
  double pad[4];
};

// One seed PCP instance for the batched (one CTA per seed) solver.
struct SeedTask {
  const double* D;  // mp x np, FP64, ld mp
  int mp, np, k0, kmax, max_iter, r_cap;
  double lam, tol, rho, mu_scale, mu_max_ratio, rank_cut;
  void* work;  // seed_workspace_bytes_cta(mp, np, kmax) bytes
  double *U, *Sigma, *V;  // outputs, ld mp / np, kmax columns
  unsigned long long timeout_ns;  // limit of one barrier wait; 0 = default
};

size_t seed_workspace_bytes_cta(int mp, int np, int kmax);
size_t seed_args_bytes();  // bytes of one packed per-instance argument block
// Bytes of the host / device argument area of a batched seed launch.
size_t seed_batched_args_bytes(int count);
// Pack the tasks into h_args (seed_batched_args_bytes(count) bytes), copy
// them to d_args and launch: a team of CTAs per seed, sized by its work
// (cooperative launch) when every seed gets at least one co-resident CTA,
// else one CTA per seed.  upload = false: d_args already holds the same
// packed bytes (a batch plan's capture after its direct run), nothing is
// copied; launch = false: pack and copy only (the batched solve copies every
// argument block before its first launch, so that no copy from pageable
// host memory waits behind a running kernel).  The same flags on the other
// batched launches below.
pcp_status seed_pcp_batched_async(const SeedTask* tasks, int count,
                                  void* h_args, void* d_args,
                                  cudaStream_t st, bool upload = true,
                                  bool launch = true);
// Device addresses of the control block / the seed rank (int) inside a
// CTA-solver workspace.
SeedCtl* seed_ctl_ptr_cta(void* d_work, int mp, int np, int kmax);
int* seed_rank_ptr_cta(void* d_work, int mp, int np, int kmax);

// Algorithm 1's stop test in FP32: ||x - A z - e||_inf < eps * max(||x -
// e||_inf, kStopNormFloor ||x||_inf).  The paper divides by ||x||_inf; with
// outliers far above the low-rank part that bound is loose on the part that
// matters (the fit of x - e), so the FP32 kernels measure the residual
// against x - e, floored for problems whose low-rank part is (near) zero.
constexpr float kStopNormFloor = 1e-3f;

// Device arguments of one set of Algorithm 1 problems (see pcp_l1_filter).
// lowp_iters: tensor-core kernel only, iterations with one-pass TF32
// products before the split (FP32-accurate) products; 0 = split throughout.
struct FilterArgs {
  const float* M;
  const int32_t* pidx;
  int p;
  int64_t sp;
  const int32_t* qidx;
  int N;
  int64_t sq;
  const float* A;
  int lda;
  int r;
  const int32_t* d_rank;
  const float* scale;
  float* Z;
  int64_t ldz;
  float eps, rho, beta0_scale, beta_bar_ratio;
  int max_iter;
  int lowp_iters;
  int lowp_bf16;  // the low-precision passes use BF16 (else one-pass TF32)
  int32_t* iters_out;
  // batched form only: the set's problems are skipped when *skip != 0 (an
  // instance whose seed failed Eq. rank_test and will grow); nullptr: never
  const int32_t* skip;
};

// Tensor-core form of Algorithm 1 (filter_tc.cu): 16 problems per CTA,
// p <= 512, r <= 64.  Single launch over a.N problems.
bool l1_filter_tc_fits(int p, int r);
cudaError_t l1_filter_tc_launch(const FilterArgs& a, cudaStream_t st);
// Batched: CTA b runs 16-problem tile tiles[2b+1] of set tiles[2b]; every
// set of one launch has the same kernel shape (tc_shape_class).
int tc_shape_class(int p, int r);
cudaError_t l1_filter_tc_batched_launch(int shape, const FilterArgs* d_sets,
                                        const int32_t* d_tiles, int ntiles,
                                        cudaStream_t st);

// One set of Algorithm 1 problems for the batched filter (the arguments of
// pcp_l1_filter, constants included, so that every set keeps its own).
struct FilterSet {
  const float* M;
  const int32_t* pidx;
  int p;
  int64_t sp;
  const int32_t* qidx;
  int N;
  int64_t sq;
  const float* A;
  int lda;
  int r;
  const int32_t* d_rank;
  const float* scale;
  float* Z;
  int64_t ldz;
  int32_t* iters_out;
  double eps, rho, beta0_scale, beta_bar_ratio;
  int max_iter;
  int precision;   // pcp_precision
  int lowp_iters;  // PCP_TF32_REFINED
  const int32_t* skip = nullptr;  // see FilterArgs::skip
};
// The FP32 SIMT kernel serves PCP_FP32_SIMT (p <= 256, r <= 32); every
// other precision runs on the tensor-core kernel.
bool filter_uses_simt(int precision, int p, int r);
// Bytes of the device argument block for these sets (h_buf and d_buf).
size_t filter_batch_bytes(const FilterSet* sets, int nsets);
// All sets, 32 problems per CTA, one launch per kernel shape present (the
// shape is fixed by p and r; sets of equal shape share a launch).
pcp_status l1_filter_batched_async(const FilterSet* sets, int nsets,
                                   void* h_buf, void* d_buf,
                                   cudaStream_t st, bool upload = true,
                                   bool launch = true);

// Batched gather / assembly: one launch for all instances.
struct GatherTask {
  const float* M;
  int64_t ldm;
  const int32_t* rows;
  const int32_t* cols;
  int mp, np;
  double* Ms;
  int32_t* bad;
};
pcp_status gather_batched_async(const GatherTask* tasks, int count,
                                void* h_buf, void* d_buf, cudaStream_t st,
                                bool upload = true, bool launch = true);
struct AssembleTask {
  const double *U, *Sigma, *V;
  int mp, np, ku, r;
  const int32_t* d_rank;
  const int32_t *rows, *cols;
  float *Lu, *Lv;
  int64_t ldu, ldv;
  float *U32, *V32, *inv_sigma32;
};
pcp_status assemble_batched_async(const AssembleTask* tasks, int count,
                                  void* h_buf, void* d_buf, cudaStream_t st,
                                  bool upload = true, bool launch = true);

// Tensor-core S pass (tcgen05 + TMA): applicability, launch, and the device
// count of bounded waits that ran out.
bool spass_tc_fits(const float* dM, int64_t ldm, float* dS, int64_t lds,
                   int r, int64_t m, int64_t n);
pcp_status spass_tc_launch(const float* dM, int64_t ldm, const float* dLu,
                           int64_t ldu, const float* dLv, int64_t ldv, int r,
                           float* dS, int64_t lds, int64_t m, int64_t n,
                           cudaStream_t st);
pcp_status spass_tc_read_timeouts(int* out);

}  // namespace pcp
