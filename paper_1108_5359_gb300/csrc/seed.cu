// Seed matrix recovery (Section 3.1, Eq. SPCP) in FP64 on the device.
//
// min ||L||_* + lam ||S||_1  s.t.  D = L + S  on the m' x n' seed D = M^s,
// solved by the inexact augmented-Lagrangian ADM the paper cites for it
// (pseudo code omitted in the paper):
//   L_{k+1} = SVT_{1/mu_k}(D - S_k + Y_k/mu_k)                  (Eq. SVT)
//   S_{k+1} = shrink_{lam/mu_k}(D - L_{k+1} + Y_k/mu_k)
//   Y_{k+1} = Y_k + mu_k (D - L_{k+1} - S_{k+1}),  mu_{k+1} = min(rho mu_k, mu_max)
// with S_0 = 0, Y_0 = D / max(||D||_2, ||D||_inf/lam), mu_0 = mu_scale/||D||_2,
// stopping at ||D - L - S||_F / ||D||_F <= tol (Section 4.1.1).
//
// The SVT needs only the singular triplets above 1/mu.  They come from a
// warm-started subspace iteration with Rayleigh-Ritz on G = D - S + Y/mu:
//   T = G^T Omega,  Psi = orth(T),  P = G Psi,  C = P^T P ~ V diag(s^2) V^T,
//   Pt = P V,  s_c^2 = ||Pt e_c||^2 (FP64 Rayleigh quotients),
//   SVT(G Psi Psi^T) = Pt diag(max(1 - tau/s, 0)) (Psi V)^T,
//   Omega_next = Pt diag(1/s)  (the left Ritz vectors),
// where orth() is a column-normalised Cholesky QR.  The subspace size k
// starts at k0 and grows while every Ritz value exceeds tau.  At the exit
// the skinny SVD of L^s is read off directly: U^s = Pt diag(1/s),
// Sigma^s = s - tau, V^s = Psi V (Section 3.2 uses exactly these factors).
//
// Precision: D, S, Y, G, every product and the Ritz values are FP64.  The
// k x k rotation V that diagonalises the Rayleigh-Ritz matrix is found by a
// Jacobi eigen-solve in FP32 (the matrix is scaled to unit diagonal maximum
// first); V enters the FP64 products as exact FP64 numbers, so the only
// effect of its FP32 accuracy is a ~1e-7 loss of orthogonality of the
// rotated bases, well below the ALM tolerance.
//
// GB300 form: one cooperative persistent launch (grid = one CTA per SM) runs
// the whole ALM loop.  Phases are separated by a software grid barrier whose
// spin is bounded by %globaltimer (on expiry every CTA sets an error word and
// returns).  The m' x n' state (S, Y, G and G^T) stays in L2.  Small k x k
// factorisations (Cholesky, Jacobi) run redundantly in every CTA so that
// they need no barrier; inputs and code are identical, so every CTA obtains
// bit-identical factors.  Cross-CTA data is read with L2-only loads
// (ld.global.cg) so no CTA sees a stale L1 line.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <queue>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace pcp {

constexpr int kSeedThreads = 256;
constexpr int kSeedKmaxLimit = 64;
constexpr int kSeedTraceCap = 4096;  // (timestamp, phase) records
constexpr int kSeedTeamMax = 64;     // largest team of the batched solver
constexpr int kSeedMaxSide = 512;    // largest m', n'
constexpr int kSeedGemmGroup = 4;    // tasks per pass of the tall products
// The tall and rank-k products of the ALM run in FP32 while its residual is
// above this, FP64 after.  An FP64 emulation of the iteration with FP32
// products (200 x 200 and 50 x 50 seeds) reached the oracle's L^s to
// 1.3e-7 .. 1.9e-7 with the switch anywhere from 1e-4 down to 3e-7, and
// to ~5e-7 with FP32 products throughout; on GB300 1e-6 took the 200 x 200
// seed from 2.96 to 2.89 ms and the 500 x 500 seed from 9.77 to 9.24 ms
// against 1e-4, with the same error against L0.
#ifndef PCP_SEED_LOWP_RES
#define PCP_SEED_LOWP_RES 1e-6
#endif
constexpr double kSeedLowpRes = PCP_SEED_LOWP_RES;
// Power steps on D before the first Rayleigh-Ritz step, whose largest Ritz
// value stands for ||D||_2 in mu_0 and Y_0.  An FP64 emulation needed the
// same ALM iteration count with 2, 1 or 0 steps, but on GB300 (FP32 k x k
// eigen-solve) one step left a 50 x 50 rank-5 seed at 6.5e-4 from the
// oracle's L^s after 31 iterations, against 5.7e-7 after 25 with two.
#ifndef PCP_SEED_POWER_STEPS
#define PCP_SEED_POWER_STEPS 2
#endif
constexpr int kSeedPowerSteps = PCP_SEED_POWER_STEPS;
static_assert(kSeedPowerSteps >= 0 && kSeedPowerSteps <= 2, "0..2 power steps");
// Largest single-cluster team (a non-portable cluster size on this part).
constexpr int kSeedClusterMax = 16;
// limit of one grid-barrier wait when the caller gives none
constexpr unsigned long long kSeedDefaultWaitNs = 2000000000ull;  // 2 s
// Partial-sum slots of the grid solver: fixed, so a solve's result does not
// depend on its CTA count; one per SM of this part (a sweep on the 200 x 200
// seed: 3.34 ms with 512 slots, 3.05 ms with 152, 3.15 ms with 76; on the
// 500 x 500 seed 11.19 / 10.63 / 11.80 ms; every slot costs each CTA a
// k-vector read in the Ritz-value reduction).
constexpr int kSeedGridSlots = 152;
// A seed with fewer rows and columns than slots gets one slot per row (or
// column) instead: a slot holds at least one row, and a small seed's CTAs
// (one per row) each walk one slot per phase instead of several empty ones.
// A function of the seed's size alone, so the result still does not depend
// on the team.
inline int seed_slots(int mp, int np, int cap) {
  return std::max(1, std::min(cap, std::max(mp, np)));
}

struct SeedLayout {
  size_t ctl, part, colsq, S, Y, G, Gt, Om, P, Pt, T, Psi, PsiT, Gam, Gam2,
      Om32, Psi32, trace, total;
};

SeedLayout seed_layout(int mp, int np, int kmax, int nbmax) {
  SeedLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t mn = (size_t)mp * np * sizeof(double);
  L.ctl = take(sizeof(SeedCtl));
  L.part = take((size_t)nbmax * 4 * sizeof(double));
  L.colsq = take((size_t)nbmax * kmax * sizeof(double));
  L.S = take(mn);
  L.Y = take(mn);
  L.G = take(mn);
  L.Gt = take(mn);
  L.Om = take((size_t)mp * kmax * sizeof(double));
  L.P = take((size_t)mp * kmax * sizeof(double));
  L.Pt = take((size_t)mp * kmax * sizeof(double));
  L.T = take((size_t)np * kmax * sizeof(double));
  L.Psi = take((size_t)np * kmax * sizeof(double));
  L.PsiT = take((size_t)np * kmax * sizeof(double));
  L.Gam = take((size_t)kmax * kmax * sizeof(double));
  L.Gam2 = take((size_t)kmax * kmax * sizeof(double));
  L.Om32 = take((size_t)mp * kmax * sizeof(float));
  L.Psi32 = take((size_t)np * kmax * sizeof(float));
  L.trace = take((size_t)kSeedTraceCap * 2 * sizeof(unsigned long long));
  L.total = off;
  return L;
}

// Workspace of the cooperative (one seed over the whole GPU) solver.
size_t seed_workspace_bytes(int mp, int np, int kmax) {
  return seed_layout(mp, np, kmax, kMaxCoopBlocks).total;
}

// Workspace of one instance of the batched solver (a team of at most
// kSeedTeamMax CTAs per seed).
size_t seed_workspace_bytes_cta(int mp, int np, int kmax) {
  return seed_layout(mp, np, kmax, kSeedTeamMax).total;
}

namespace {

// 16-byte aligned: the batched launch packs these back to back with a
// stride of sizeof(SeedArgs), which device code indexes the same way
struct alignas(16) SeedArgs {
  const double* D;
  int mp, np, kmax, k0;
  double lam, tol, rho, mu_scale, mu_max_ratio, rank_cut;
  int max_iter, r_cap;
  // the tall and rank-k products run in FP32 while the ALM residual is
  // above this, FP64 after
  double lowp_res;
  int smem_doubles;  // dynamic shared memory of the launch, in doubles
  // partial-sum slots of the three reductions (norms of D, Ritz values,
  // residual): fixed per solve, so the summation order (and the result)
  // does not depend on how many CTAs the team has
  int nv;
  unsigned long long timeout_ns;
  SeedCtl* ctl;
  double* part;
  double* colsq;           // [block][kmax] partial column sums of Pt^2
  double *S, *Y, *G, *Gt;
  double *Om, *P, *Pt;     // mp x kmax, row-major (row stride kmax)
  double *T, *Psi, *PsiT;  // np x kmax, row-major
  double* Gam;             // kmax x kmax
  double* Gam2;            // kmax x kmax: Psi1^T Psi1
  float *Om32, *Psi32;     // FP32 copies of Om, Psi (early tall products)
  unsigned long long* trace;  // block 0's phase timestamps
  double *U, *Sigma, *V;   // outputs (column-major, ld mp / np)
};

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

// Software grid barrier, bounded by a timeout.
__device__ bool grid_sync(SeedCtl* ctl, unsigned int nblocks,
                          unsigned long long timeout_ns) {
  // Counter barrier on a monotonically increasing arrival count (the control
  // block is zeroed per launch): barrier g completes when the count reaches
  // (g + 1) * nblocks.  bar.sync orders the CTA's writes before thread 0's
  // release-add, and thread 0's acquire-load before the CTA's later reads,
  // so only one thread per CTA synchronises at GPU scope (no per-thread
  // fences).
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* cnt = &ctl->bar_count;
    unsigned int arrived;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;"
                 : "=r"(arrived)
                 : "l"(cnt)
                 : "memory");
    const unsigned int target = (arrived / nblocks + 1) * nblocks;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];"
                   : "=r"(cur)
                   : "l"(cnt)
                   : "memory");
      if ((int)(cur - target) >= 0) break;
      if (*(volatile int*)&ctl->error) break;
      // the clock is read on every spin (each spin is an L2 round trip, far
      // longer than the read), so a wait ends within one spin of its limit
      if (globaltimer_ns() - t0 > timeout_ns) {
        atomicExch(&ctl->error, (int)PCP_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    s_ok = (*(volatile int*)&ctl->error) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block 0 records (globaltimer, phase) after the phase ends.
__device__ __forceinline__ void trace_mark(const SeedArgs& a, int phase) {
  if (a.trace && blockIdx.x == 0 && threadIdx.x == 0) {
    const int i = a.ctl->ntrace;
    if (i < kSeedTraceCap) {
      a.trace[2 * i] = globaltimer_ns();
      a.trace[2 * i + 1] = (unsigned long long)phase;
      a.ctl->ntrace = i + 1;
    }
  }
}

// Deterministic N(0,1) from a counter (splitmix64 + Box-Muller).
__device__ double hash_normal(unsigned long long a, unsigned long long b) {
  auto mix = [](unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const unsigned long long h1 = mix(a * 0x100000001B3ull + b);
  const unsigned long long h2 = mix(h1 ^ 0xD1B54A32D192ED03ull);
  const double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Fixed-order (deterministic) block reduction of v over all threads.
__device__ double block_reduce_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < kSeedThreads / 32; ++q) s += red[q];
  __syncthreads();
  return s;
}

__device__ double block_reduce_max(double v, double* red) {
  v = warp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < kSeedThreads / 32; ++q) s = fmax(s, red[q]);
  __syncthreads();
  return s;
}

// sum over blocks q < nb of src[q * stride + off]; every thread gets it.
__device__ double sum_partials(const double* src, int nb, int stride, int off,
                               double* red) {
  double acc = 0.0;
  for (int q = threadIdx.x; q < nb; q += kSeedThreads)
    acc += ldg_cg(src + (size_t)q * stride + off);
  return block_reduce_sum(acc, red);
}

// out[task*kmax + c] = sum_t X[t + task*ldx] * B[t*kmax + c], c < k.
// A CTA takes its tasks (task = bid + i nblk) kSeedGemmGroup at a time:
// their columns of X are staged in shared memory (xs, kSeedMaxSide each)
// and every row of B a thread loads serves all of them, so the L2 round
// trips for B are shared.  Each thread owns one c and the slice t = part +
// s nparts, with four accumulators per task; a task's partial sums go to
// gred (kSeedThreads each) and are added in a fixed order, so a task's
// result does not depend on how many tasks its CTA holds.
template <int kG, typename TF>
__device__ void tall_gemm_group(const double* X, int ldx, int len, int ntask,
                                const TF* B, int k, int kmax, double* out,
                                double* gred, double* xs_raw, int bid,
                                int nblk) {
  TF* xs = reinterpret_cast<TF*>(xs_raw);
  const int tid = threadIdx.x;
  const int nparts = kSeedThreads / k;
  const int c = tid % k, part = tid / k;
  for (int t0 = bid; t0 < ntask; t0 += kG * nblk) {
    const int ng = min(kG, (ntask - t0 + nblk - 1) / nblk);
    for (int g = 0; g < ng; ++g) {
      const double* x = X + (size_t)(t0 + g * nblk) * ldx;
      for (int t = tid; t < len; t += kSeedThreads)
        xs[g * kSeedMaxSide + t] = (TF)ldg_cg(x + t);
    }
    __syncthreads();
    if (part < nparts) {
      TF acc[kG][4];
#pragma unroll
      for (int g = 0; g < kG; ++g)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[g][i] = TF(0);
      int t = part;
#pragma unroll 2
      for (; t + 3 * nparts < len; t += 4 * nparts) {
        TF bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          bv[i] = __ldcg(B + (size_t)(t + i * nparts) * kmax + c);
#pragma unroll
        for (int g = 0; g < kG; ++g)
          if (g < ng)
#pragma unroll
            for (int i = 0; i < 4; ++i)
              acc[g][i] = fma(xs[g * kSeedMaxSide + t + i * nparts], bv[i],
                              acc[g][i]);
      }
      for (; t < len; t += nparts) {
        const TF bv = __ldcg(B + (size_t)t * kmax + c);
#pragma unroll
        for (int g = 0; g < kG; ++g)
          if (g < ng) acc[g][0] = fma(xs[g * kSeedMaxSide + t], bv, acc[g][0]);
      }
#pragma unroll
      for (int g = 0; g < kG; ++g)
        if (g < ng)
          gred[g * kSeedThreads + part * k + c] =
              (double)((acc[g][0] + acc[g][1]) + (acc[g][2] + acc[g][3]));
    }
    __syncthreads();
    for (int idx = tid; idx < ng * k; idx += kSeedThreads) {
      const int g = idx / k, cc = idx - g * k;
      double s = 0.0;
      for (int q = 0; q < nparts; ++q) s += gred[g * kSeedThreads + q * k + cc];
      __stcg(out + (size_t)(t0 + g * nblk) * kmax + cc, s);
    }
    __syncthreads();
  }
}

// Group size by the tasks per CTA (the group's accumulators cost registers,
// so a CTA with one or two tasks runs the narrower forms).  With B32 (an
// FP32 copy of B) the products run in FP32: the seed uses that while the
// ALM residual is above 1e-4, where their ~1e-7 relative error is far below
// what the inexact ALM leaves, and this part's FP64 pipe (2 FMA/clk/SM)
// made the tall products FP64-throughput bound on the 500 x 500 seed.
__device__ void tall_gemm_t(const double* X, int ldx, int len, int ntask,
                            const double* B, const float* B32, int k, int kmax,
                            double* out, double* gred, double* xs, int bid,
                            int nblk) {
  if (B32) {
    if (ntask <= nblk)
      tall_gemm_group<1>(X, ldx, len, ntask, B32, k, kmax, out, gred, xs, bid,
                         nblk);
    else if (ntask <= 2 * nblk)
      tall_gemm_group<2>(X, ldx, len, ntask, B32, k, kmax, out, gred, xs, bid,
                         nblk);
    else
      tall_gemm_group<kSeedGemmGroup>(X, ldx, len, ntask, B32, k, kmax, out,
                                      gred, xs, bid, nblk);
    return;
  }
  if (ntask <= nblk)
    tall_gemm_group<1>(X, ldx, len, ntask, B, k, kmax, out, gred, xs, bid, nblk);
  else if (ntask <= 2 * nblk)
    tall_gemm_group<2>(X, ldx, len, ntask, B, k, kmax, out, gred, xs, bid, nblk);
  else
    tall_gemm_group<kSeedGemmGroup>(X, ldx, len, ntask, B, k, kmax, out, gred,
                                    xs, bid, nblk);
}

// Gm = X^T X (k x k) for X (nrows x k, row-major stride kmax); one warp per
// entry a <= b, both triangles written.
__device__ void gram(const double* X, int nrows, int k, int kmax,
                     double* Gm, int bid, int nblk) {
  const int lane = threadIdx.x & 31;
  const int gw = bid * (kSeedThreads / 32) + (threadIdx.x >> 5);
  const int nw = nblk * (kSeedThreads / 32);
  const int npairs = k * (k + 1) / 2;
  for (int pq = gw; pq < npairs; pq += nw) {
    // pq -> (a, b) with a <= b, row-major over the upper triangle
    int a = 0, rem = pq;
    while (rem >= k - a) {
      rem -= k - a;
      ++a;
    }
    const int b = a + rem;
    double s0 = 0.0, s1 = 0.0;
    int t = lane;
    for (; t + 32 < nrows; t += 64) {
      const double x0 = ldg_cg(X + (size_t)t * kmax + a);
      const double y0 = ldg_cg(X + (size_t)t * kmax + b);
      const double x1 = ldg_cg(X + (size_t)(t + 32) * kmax + a);
      const double y1 = ldg_cg(X + (size_t)(t + 32) * kmax + b);
      s0 = fma(x0, y0, s0);
      s1 = fma(x1, y1, s1);
    }
    for (; t < nrows; t += 32)
      s0 = fma(ldg_cg(X + (size_t)t * kmax + a),
               ldg_cg(X + (size_t)t * kmax + b), s0);
    const double s = warp_sum(s0 + s1);
    if (lane == 0) {
      __stcg(Gm + a * kmax + b, s);
      __stcg(Gm + b * kmax + a, s);
    }
  }
}

// Right-looking Cholesky of the k x k (k <= K <= 32) scaled Gram in A32 by
// one warp, the matrix held in registers: lane c keeps column c (a[r] =
// A_rc).  Step j takes the pivot from lane j, every lane c > j scales its
// entry of row j (R_jc = A_jc / sqrt(A_jj)), and each later row r gets its
// rank-1 update A_rc -= R_jr R_jc with R_jr broadcast from lane r.  Same
// operations in the same order per entry as the CTA-wide form, without its
// k CTA barriers.  The K x K body is straight-line code (no test on k):
// rows and columns past k hold zeros, so their steps change nothing that
// is kept, and the broadcasts of a step overlap the next step's pivot
// chain.  A non-positive pivot (or a dead column) gives R_jj = 1 and a
// zero row, and marks the column dead.  R (upper triangle and diagonal) is
// written back to A; the lower triangle is left as it was.  A: the block's
// first entry, row stride lda; rs_out (optional): the reciprocal pivots
// rs_j the rows were scaled by.
template <int K, bool kRs>
__device__ __noinline__ void chol_warp(float* A, int lda, int k, int* dead,
                                       float* rs_out) {
  const int lane = threadIdx.x & 31;
  const bool own = lane < k;
  float a[K];
#pragma unroll
  for (int r = 0; r < K; ++r)
    a[r] = (own && r < k) ? A[r * lda + lane] : 0.0f;
  int dl = own ? dead[lane] : 1;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float piv = __shfl_sync(0xffffffffu, a[j], j);
    const int dj = __shfl_sync(0xffffffffu, dl, j);
    const bool bad = !(piv > 1e-6f) || dj;
    const float rs = bad ? 0.0f : rsqrtf(piv);
    float rj = a[j] * rs;  // R_jc for lanes c > j
    if (lane == j) {
      rj = bad ? 1.0f : piv * rs;
      if (bad) dl = 1;
      if (kRs && j < k) rs_out[j] = rs;
    }
    if (lane >= j) a[j] = rj;
    const float rju = lane > j ? rj : 0.0f;  // columns <= j are final
#pragma unroll
    for (int r = j + 1; r < K; ++r) {
      const float rjr = __shfl_sync(0xffffffffu, rj, r);
      a[r] = fmaf(-rjr, rju, a[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < K; ++r)
    if (own && r < k && r <= lane) A[r * lda + lane] = a[r];
  if (own) dead[lane] = dl;
}

// The same factorisation for 32 < k <= 64 in four steps, each entry taking
// the same operations in the same order as the right-looking CTA-wide form
// (so the same bits): one warp factors the leading 32 x 32 block (keeping
// its reciprocal pivots in rs); a thread per column c >= 32 forms rows
// 0..31 of R in turn, R_jc = (A_jc - sum_{i<j} R_ij R_ic) rs_j with the
// terms in i order; the trailing block takes its 32 updates A_rc -=
// R_ir R_ic in i order (upper triangle); one warp factors it.
static_assert(kSeedKmaxLimit <= 64, "the Cholesky forms cover k <= 64");
__device__ __noinline__ void chol_blocked64(float* A32, int k, int* dead,
                                            float* rs) {
  const int tid = threadIdx.x;
  if (tid < 32) chol_warp<32, true>(A32, k, 32, dead, rs);
  __syncthreads();
  {
    // rows 0..31 of columns c >= 32, right-looking in registers: warp w
    // takes columns 32 + w + 8 q (q < 4), lane j holds row j of each; at
    // step i lane i finalises R_ic = a_ic rs_i and broadcasts it, and every
    // lane j > i takes its update a_jc -= R_ij R_ic (four independent
    // chains per warp)
    const int lane = tid & 31, w = tid >> 5;
    constexpr int kQ = 4;
    float v[kQ];
    int cq[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      cq[q] = 32 + w + (kSeedThreads / 32) * q;
      v[q] = cq[q] < k ? A32[lane * k + cq[q]] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float rsi = rs[i];
      const float rij = lane > i ? A32[i * k + lane] : 0.0f;
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        if (lane == i) v[q] *= rsi;
        const float ric = __shfl_sync(0xffffffffu, v[q], i);
        if (lane > i) v[q] = fmaf(-rij, ric, v[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q)
      if (cq[q] < k) A32[lane * k + cq[q]] = v[q];
  }
  __syncthreads();
  const int k2 = k - 32;
  for (int idx = tid; idx < k2 * k2; idx += kSeedThreads) {
    const int r = 32 + idx / k2, c = 32 + idx % k2;
    if (c < r) continue;
    float acc = A32[r * k + c];
#pragma unroll 8
    for (int i = 0; i < 32; ++i)
      acc = fmaf(-A32[i * k + r], A32[i * k + c], acc);
    A32[r * k + c] = acc;
  }
  __syncthreads();
  if (tid < 32)
    chol_warp<32, false>(A32 + 32 * k + 32, k, k2, dead + 32, nullptr);
}

// Column-normalised Cholesky QR: Out = X diag(1/||x_a||) R^{-1} with
// R^T R = diag(1/||x_a||) X^T X diag(1/||x_a||) (unit diagonal, well
// conditioned).  The k x k Cholesky factor and its inverse are computed in
// FP32 (FP64 latency on this part is ~64 cycles per dependent FMA and ~650
// per divide or square root); the row products X R^{-1} run in FP64 with
// those FP32 values.  The result is orthonormal to ~1e-7, which the ALM
// absorbs (tested against the full-SVD FP64 oracle).  Columns whose norm or
// pivot vanishes are dead and come out zero.  A32: k x k shared; Ri32: k.
__device__ void cholqr_apply(const double* X, int nrows, int k, int kmax,
                             const double* Gm, double* Out, float* Out32,
                             float* A32,
                             float* Ri32, double* Rd, double* dsc, int* dead,
                             double* rowb, int bid, int nblk, int row_warps,
                             long long* sub) {
  const int tid = threadIdx.x;
  const bool prof = sub && bid == 0 && tid == 0;
  long long q0 = prof ? clock64() : 0;
  for (int c = tid; c < k; c += kSeedThreads) {
    const double g = ldg_cg(Gm + c * kmax + c);
    dead[c] = !(g > 0.0);
    dsc[c] = (g > 0.0) ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  // scaled Gram in FP32 (redundant per CTA: FP64 here would occupy the
  // chip's narrow FP64 pipe in every CTA at once)
  int coupled = 0;
  for (int a = tid >> 4; a < k; a += kSeedThreads / 16) {
    const float da = (float)dsc[a];
    for (int b = tid & 15; b < k; b += 16) {
      float v = (float)ldg_cg(Gm + a * kmax + b) * da * (float)dsc[b];
      if (dead[a] || dead[b]) {
        v = (a == b) ? 1.0f : 0.0f;
        coupled = 1;
      } else if (a != b && !(fabsf(v) <= 1e-3f)) {
        coupled = 1;
      }
      A32[a * k + b] = v;
    }
  }
  // Nearly orthogonal columns (warm-started iterations): the Cholesky
  // factor of I + F with |F| <= 1e-3 is R = I + triu(F) + O(1e-6); the
  // O(1e-6) non-orthogonality it leaves is removed with E downstream, so
  // the k sequential pivot steps are skipped.
  const bool near_orth = !__syncthreads_or(coupled);
  long long q1 = prof ? clock64() : 0;
  // Right-looking Cholesky, R in the upper triangle (a non-positive pivot
  // marks the column dead: R_jj = 1, rest of the row 0): one warp in
  // registers for k <= 32, the blocked form above it (k <= 64, the
  // subspace limit).
  if (!near_orth) {
    if (k <= 32) {
      if (tid < 32) {
        if (k <= 16)
          chol_warp<16, false>(A32, k, k, dead, nullptr);
        else
          chol_warp<32, false>(A32, k, k, dead, nullptr);
      }
    } else {
      chol_blocked64(A32, k, dead, Ri32);
    }
  }
  __syncthreads();
  // Reciprocal pivots, then one warp per output row solves x R = t~ by
  // forward substitution (lane c owns columns c and c + 32).  The row data
  // and the arithmetic are FP64; R and its reciprocal pivots are the FP32
  // factor's values, widened once into FP64 copies (Rd, with a dead
  // direction's reciprocal pivot 0) so that the k dependent steps of a row
  // carry no conversions.  Keeping t~ in FP64 matters: rounding it to FP32
  // perturbs the directions near the threshold enough to slow the ALM.
  for (int c = tid; c < k; c += kSeedThreads) Ri32[c] = 1.0f / A32[c * k + c];
  __syncthreads();
  double* Rid = rowb;  // kmax doubles
  for (int idx = tid; idx < k * k; idx += kSeedThreads) {
    const int j = idx / k, c = idx - j * k;
    Rd[idx] = c > j ? (double)A32[idx] : 0.0;
  }
  for (int c = tid; c < k; c += kSeedThreads)
    Rid[c] = dead[c] ? 0.0 : (double)Ri32[c];
  __syncthreads();
  long long q2 = prof ? clock64() : 0;
  // row_warps warps per CTA (1 for a grid-wide team: the FP64 pipe is
  // narrow on this part, so rows are spread over as many SMs as possible)
  const int lane = tid & 31, wid = tid >> 5;
  for (int t = (wid < row_warps) ? bid * row_warps + wid : nrows; t < nrows;
       t += nblk * row_warps) {
    const int c0 = lane, c1 = lane + 32;
    const int cc0 = min(c0, k - 1), cc1 = min(c1, k - 1);
    double p0 = c0 < k ? ldg_cg(X + (size_t)t * kmax + c0) * dsc[c0] : 0.0;
    double p1 = c1 < k ? ldg_cg(X + (size_t)t * kmax + c1) * dsc[c1] : 0.0;
    double o0 = 0.0, o1 = 0.0;
    for (int j = 0; j < k; ++j) {
      const int owner = j & 31;
      const double mine = ((j < 32) ? p0 : p1) * Rid[j];
      const double xj = __shfl_sync(0xffffffffu, mine, owner);
      if (lane == owner) {
        if (j < 32) o0 = xj; else o1 = xj;
      }
      // Rd holds zeros on and below the diagonal, so columns <= j are
      // left as they are
      p0 = fma(-xj, Rd[j * k + cc0], p0);
      p1 = fma(-xj, Rd[j * k + cc1], p1);
    }
    if (c0 < k) {
      __stcg(Out + (size_t)t * kmax + c0, o0);
      Out32[(size_t)t * kmax + c0] = (float)o0;
    }
    if (c1 < k) {
      __stcg(Out + (size_t)t * kmax + c1, o1);
      Out32[(size_t)t * kmax + c1] = (float)o1;
    }
  }
  if (prof) {
    const long long q3 = clock64();
    sub[0] += q1 - q0;
    sub[1] += q2 - q1;
    sub[2] += q3 - q2;
  }
}

// Rotation (c, s) that zeroes a_pq of the symmetric 2 x 2 block
// [[app, apq], [apq, aqq]] (A' = J^T A J with J = [[c, s], [-s, c]]); the
// identity when a_pq is at the FP32 noise floor (2 ulp of the unit largest
// diagonal) or negligible against its own diagonal.
// Branch-free, built from the fast reciprocal / reciprocal-square-root
// units: the angle only has to be accurate to a few ulp (an inexact
// rotation is still orthogonal to FP32 precision and the next sweep removes
// what it leaves).
__device__ __forceinline__ bool jacobi_angle(float app, float aqq, float apq,
                                             float& c, float& s) {
  const float mag = fabsf(apq);
  const bool rot = (mag * mag > 1e-14f * fabsf(app * aqq)) && (mag > 2.4e-7f);
  const float den = rot ? 2.0f * apq : 1.0f;
  const float theta = __fdividef(aqq - app, den);
  const float u = fmaf(theta, theta, 1.0f);
  const float t = __fdividef(copysignf(1.0f, theta),
                             fabsf(theta) + u * rsqrtf(u));
  const float cc = rsqrtf(fmaf(t, t, 1.0f));
  c = rot ? cc : 1.0f;
  s = rot ? t * cc : 0.0f;
  return rot;
}

// Cyclic Jacobi eigen-decomposition (FP32) of the symmetric k x k matrix in
// A0 (k even, entries scaled to at most 1), parallel round-robin ordering.
// One barrier per round: every thread owns 2 x 2 blocks (rows of pair i,
// columns of pair j) and recomputes the two rotations it needs from the
// current A; it writes the rotated block of A into the other buffer and
// rotates its block of V (columns of pair j) in place.  Returns the buffer
// holding the final A (diagonal = eigenvalues); V's columns are the
// eigenvectors.
__device__ float* block_jacobi32(float* A0, float* A1, float* V, int k,
                                 unsigned char* tab, int max_sweeps,
                                 int* sweeps_out, long long* cyc) {
  const int tid = threadIdx.x;
  // round-robin schedule: tab[round*k + x] = position of slot x (slot 0
  // fixed, the others rotate); pair i is (slot i, slot k-1-i)
  for (int e = tid; e < (k - 1) * k; e += kSeedThreads) {
    const int round = e / k, x = e - round * k;
    tab[e] = (unsigned char)(x == 0 ? 0 : 1 + (x - 1 + round) % (k - 1));
  }
  __shared__ int s_rot[2];
  __shared__ float s_cs[kSeedKmaxLimit];  // (c, s) of each pair
  const bool prof = cyc && blockIdx.x == 0 && tid == 0;
  long long c0 = 0;
  for (int idx = tid; idx < k * k; idx += kSeedThreads)
    V[idx] = (idx / k == idx % k) ? 1.0f : 0.0f;
  const int half = k / 2;
  float* A = A0;
  float* An = A1;
  int flip = 0;
  if (tid == 0) s_rot[0] = s_rot[1] = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0 && sweeps_out && blockIdx.x == 0) *sweeps_out += 1;
    for (int round = 0; round < k - 1; ++round) {
      const long long t0 = prof ? clock64() : 0;
      __syncthreads();
      if (prof) c0 += clock64() - t0;
      // Wide matrices (more than 16 pairs): the pair angles are computed
      // once each and shared (one more barrier per round); narrow ones
      // recompute them per block (independent, so they overlap) and keep
      // one barrier per round.
      const bool shared_angles = half > 16;
      if (shared_angles) {
        const unsigned char* tr = tab + round * k;
        for (int i = tid; i < half; i += kSeedThreads) {
          int pi = tr[i], qi = tr[k - 1 - i];
          if (pi > qi) { const int t = pi; pi = qi; qi = t; }
          float ci, si;
          if (jacobi_angle(A[pi * k + pi], A[qi * k + qi], A[pi * k + qi],
                           ci, si))
            s_rot[flip] = 1;
          s_cs[2 * i] = ci;
          s_cs[2 * i + 1] = si;
        }
        __syncthreads();
      }
      // 2-D thread map without integer division: 16 x 16 for half <= 16,
      // 8 x 32 otherwise
      const int jsh = half <= 16 ? 4 : 5;
      for (int w = tid; w < (half << jsh); w += kSeedThreads) {
        const int i = w >> jsh, j = w & ((1 << jsh) - 1);
        if (j >= half) continue;
        const unsigned char* tr = tab + round * k;
        int pi = tr[i], qi = tr[k - 1 - i];
        int pj = tr[j], qj = tr[k - 1 - j];
        if (pi > qi) { const int t = pi; pi = qi; qi = t; }
        if (pj > qj) { const int t = pj; pj = qj; qj = t; }
        float ci, si, cj, sj;
        bool rj;
        if (shared_angles) {
          ci = s_cs[2 * i];
          si = s_cs[2 * i + 1];
          cj = s_cs[2 * j];
          sj = s_cs[2 * j + 1];
          rj = sj != 0.0f;
        } else {
          const bool ri = jacobi_angle(A[pi * k + pi], A[qi * k + qi],
                                       A[pi * k + qi], ci, si);
          rj = jacobi_angle(A[pj * k + pj], A[qj * k + qj], A[pj * k + qj],
                            cj, sj);
          if (ri && i == j) s_rot[flip] = 1;
        }
        const float b00 = A[pi * k + pj], b01 = A[pi * k + qj];
        const float b10 = A[qi * k + pj], b11 = A[qi * k + qj];
        const float r00 = ci * b00 - si * b10, r01 = ci * b01 - si * b11;
        const float r10 = si * b00 + ci * b10, r11 = si * b01 + ci * b11;
        An[pi * k + pj] = r00 * cj - r01 * sj;
        An[pi * k + qj] = r00 * sj + r01 * cj;
        An[qi * k + pj] = r10 * cj - r11 * sj;
        An[qi * k + qj] = r10 * sj + r11 * cj;
        if (rj) {
          const float v0 = V[pi * k + pj], v1 = V[pi * k + qj];
          const float v2 = V[qi * k + pj], v3 = V[qi * k + qj];
          V[pi * k + pj] = cj * v0 - sj * v1;
          V[pi * k + qj] = sj * v0 + cj * v1;
          V[qi * k + pj] = cj * v2 - sj * v3;
          V[qi * k + qj] = sj * v2 + cj * v3;
        }
      }
      float* t = A;
      A = An;
      An = t;
    }
    __syncthreads();
    const int any = s_rot[flip];
    __syncthreads();
    if (tid == 0) s_rot[flip] = 0;
    flip ^= 1;
    if (!any) break;
  }
  __syncthreads();
  (void)c0;
  return A;
}

// ---- FP64 finalisation helpers (the skinny SVD of the converged iterate) ---

// Gm[a*kmax + b] = sc_a sc_b sum_t X[t*kmax + sel_a] X[t*kmax + sel_b] for
// a, b < nk (sc = 1 when null); one warp per entry a <= b with a fixed
// summation order, both triangles written.
__device__ void gram_sel(const double* X, int nrows, int kmax, const int* sel,
                         const double* sc, int nk, double* Gm, int bid,
                         int nblk) {
  const int lane = threadIdx.x & 31;
  const int gw = bid * (kSeedThreads / 32) + (threadIdx.x >> 5);
  const int nw = nblk * (kSeedThreads / 32);
  const int npairs = nk * (nk + 1) / 2;
  for (int pq = gw; pq < npairs; pq += nw) {
    int a = 0, rem = pq;
    while (rem >= nk - a) {
      rem -= nk - a;
      ++a;
    }
    const int b = a + rem;
    const int ca = sel[a], cb = sel[b];
    double s0 = 0.0, s1 = 0.0;
    int t = lane;
    for (; t + 32 < nrows; t += 64) {
      s0 = fma(ldg_cg(X + (size_t)t * kmax + ca),
               ldg_cg(X + (size_t)t * kmax + cb), s0);
      s1 = fma(ldg_cg(X + (size_t)(t + 32) * kmax + ca),
               ldg_cg(X + (size_t)(t + 32) * kmax + cb), s1);
    }
    for (; t < nrows; t += 32)
      s0 = fma(ldg_cg(X + (size_t)t * kmax + ca),
               ldg_cg(X + (size_t)t * kmax + cb), s0);
    double v = warp_sum(s0 + s1);
    if (sc) v = v * sc[a] * sc[b];
    if (lane == 0) {
      __stcg(Gm + a * kmax + b, v);
      __stcg(Gm + b * kmax + a, v);
    }
  }
}

// 1/sqrt(x) to FP64 accuracy without the FP64 divide / square-root
// sequences (hundreds of cycles on this part): an FP32 estimate refined by
// two Newton steps y <- y (3/2 - x y^2 / 2), each doubling the correct bits
// (~2^-23 -> 2^-46 -> full).  0 for x <= 0 (a dead direction).
__device__ __forceinline__ double rsqrt_f64(double x) {
  if (!(x > 0.0)) return 0.0;
  float xf = (float)x;
  double y;
  if (xf > 0.0f && xf < 3.0e38f) {
    y = (double)rsqrtf(xf);
  } else {
    y = 1.0 / sqrt(x);  // outside the FP32 range (not met in practice)
  }
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

// Cholesky A = R^T R (R upper) of two nk x nk SPD matrices in FP64, in
// place (row-major, stride nk), side by side.  Step j: threads 0 and 32
// form y_j = 1/sqrt(a_jj) of their matrix; then every trailing entry
// a_ab -= (a_ja a_jb) y_j^2 (a <= b, both > j) with row j left unscaled; at
// the end row j is scaled by y_j (R_jj = sqrt(a_jj), R_jb = a_jb / R_jj) and
// the strict lower triangle zeroed.  y0 / y1 keep the reciprocal pivots
// 1 / R_jj.  A non-positive pivot gives y = 0: that row of R is zero.
__device__ void chol2_f64(double* A0, double* A1, int nk, double* y0,
                          double* y1) {
  const int tid = threadIdx.x;
  for (int j = 0; j < nk; ++j) {
    if (tid == 0) y0[j] = rsqrt_f64(A0[j * nk + j]);
    if (tid == 32) y1[j] = rsqrt_f64(A1[j * nk + j]);
    __syncthreads();
    const int w = nk - j - 1;
    const double yy0 = y0[j] * y0[j], yy1 = y1[j] * y1[j];
    for (int idx = tid; idx < 2 * w * w; idx += kSeedThreads) {
      const int m = idx >= w * w;
      const int e = idx - m * w * w;
      const int ra = j + 1 + e / w, rb = j + 1 + e % w;
      if (rb < ra) continue;
      double* A = m ? A1 : A0;
      const double yy = m ? yy1 : yy0;
      A[ra * nk + rb] =
          fma(-(A[j * nk + ra] * yy), A[j * nk + rb], A[ra * nk + rb]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < 2 * nk * nk; idx += kSeedThreads) {
    const int m = idx >= nk * nk;
    const int e = idx - m * nk * nk;
    const int ra = e / nk, rb = e - ra * nk;
    double* A = m ? A1 : A0;
    const double* y = m ? y1 : y0;
    A[e] = rb >= ra ? A[e] * y[ra] : 0.0;
  }
  __syncthreads();
}

// Solve R X = B in place for two upper-triangular systems (R0 X0 = B0,
// R1 X1 = B1; nk x nk, row-major, reciprocal pivots y0 / y1), all columns at
// once: row a from the last up, x_a = b_a / R_aa, then b_c -= R_ca x_a for
// the rows c above it.
__device__ void backsub2_f64(const double* R0, const double* R1, double* B0,
                             double* B1, int nk, const double* y0,
                             const double* y1) {
  const int tid = threadIdx.x;
  for (int ra = nk - 1; ra >= 0; --ra) {
    for (int idx = tid; idx < 2 * nk; idx += kSeedThreads) {
      const int m = idx >= nk, q = idx - m * nk;
      double* B = m ? B1 : B0;
      B[ra * nk + q] *= (m ? y1 : y0)[ra];
    }
    __syncthreads();
    for (int idx = tid; idx < 2 * ra * nk; idx += kSeedThreads) {
      const int m = idx >= ra * nk;
      const int e = idx - m * ra * nk;
      const int rc = e / nk, q = e - rc * nk;
      double* B = m ? B1 : B0;
      const double* R = m ? R1 : R0;
      B[rc * nk + q] = fma(-R[rc * nk + ra], B[ra * nk + q], B[rc * nk + q]);
    }
    __syncthreads();
  }
}

// One-sided (Hestenes) Jacobi in FP64 on the columns of the nk x nk matrix
// C (row-major), accumulating the rotations in W (set to I here): on
// return C's columns are orthogonal (C_in W = C_out) and W is orthogonal.
// Parallel round-robin ordering (every pair of columns meets once per
// sweep), one warp per pair, lanes over rows.  The pair (p, q), p < q, is
// rotated when (x.y)^2 > 1e-28 (x.x)(y.y): t = tan of the angle from the
// FP32 quadratic formula (the next sweep corrects its FP32 error), c =
// (1 + t^2)^-1/2 by rsqrt_f64, s = t c, so every rotation is orthogonal to
// FP64 rounding.  Sweeps until one rotates nothing (at most 16).  Returns
// the number of sweeps.
__device__ int hestenes_f64(double* C, double* W, int nk) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  for (int idx = tid; idx < nk * nk; idx += kSeedThreads)
    W[idx] = (idx / nk == idx % nk) ? 1.0 : 0.0;
  __syncthreads();
  if (nk < 2) return 0;
  const int nkp = (nk + 1) & ~1;
  const int half = nkp / 2;
  int sweep = 0;
  while (sweep < 16) {
    ++sweep;
    int rot = 0;
    for (int rd = 0; rd < nkp - 1; ++rd) {
      for (int i = wid; i < half; i += kSeedThreads / 32) {
        const int s0 = i, s1 = nkp - 1 - i;  // slots of the pair
        const int x0 = s0 == 0 ? 0 : 1 + (s0 - 1 + rd) % (nkp - 1);
        const int x1 = 1 + (s1 - 1 + rd) % (nkp - 1);
        const int p = min(x0, x1), q = max(x0, x1);
        if (q >= nk) continue;  // padding column (odd nk)
        const int r0 = lane, r1 = lane + 32;
        const double xp0 = r0 < nk ? C[r0 * nk + p] : 0.0;
        const double xq0 = r0 < nk ? C[r0 * nk + q] : 0.0;
        const double xp1 = r1 < nk ? C[r1 * nk + p] : 0.0;
        const double xq1 = r1 < nk ? C[r1 * nk + q] : 0.0;
        const double al = warp_sum(fma(xp0, xp0, xp1 * xp1));
        const double be = warp_sum(fma(xq0, xq0, xq1 * xq1));
        const double ga = warp_sum(fma(xp0, xq0, xp1 * xq1));
        if (!(al > 0.0 && be > 0.0 && ga * ga > 1e-28 * al * be)) continue;
        const float z = (float)(be - al) / (2.0f * (float)ga);
        const float tf = copysignf(1.0f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.0f)));
        if (tf == 0.0f) continue;
        rot = 1;
        const double t = (double)tf;
        const double c = rsqrt_f64(fma(t, t, 1.0));
        const double sn = t * c;
        if (r0 < nk) {
          C[r0 * nk + p] = fma(c, xp0, -sn * xq0);
          C[r0 * nk + q] = fma(sn, xp0, c * xq0);
          const double wp = W[r0 * nk + p], wq = W[r0 * nk + q];
          W[r0 * nk + p] = fma(c, wp, -sn * wq);
          W[r0 * nk + q] = fma(sn, wp, c * wq);
        }
        if (r1 < nk) {
          C[r1 * nk + p] = fma(c, xp1, -sn * xq1);
          C[r1 * nk + q] = fma(sn, xp1, c * xq1);
          const double wp = W[r1 * nk + p], wq = W[r1 * nk + q];
          W[r1 * nk + p] = fma(c, wp, -sn * wq);
          W[r1 * nk + q] = fma(sn, wp, c * wq);
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rot)) break;
  }
  return sweep;
}

// Fast form of the final FP64 SVD, for the usual case of nearly orthonormal
// bases (F = G - I with |F| <= 1e-4, G the Gram of Ut or Vt) and a core
// whose singular values are well separated against its off-diagonal part.
// On entry D0 = F_u, D1 = F_v (FP64, nk x nk, row-major), sg = sigma_K.
//   Löwdin orthonormalisation to second order: Q = Ut X, X = (I + F)^-1/2
//     = I - F/2 + 3/8 F^2 + O(F^3);  Ut = Q S, S = I + F/2 - F^2/8 + O(F^3);
//   core C = S_u diag(sigma) S_v = diag(sigma) + E, with
//     E = (F_u Sigma + Sigma F_v)/2 + F_u Sigma F_v / 4 - F_u^2 Sigma / 8
//         - Sigma F_v^2 / 8;
//   first-order SVD of C = diag(d) + offdiag(E), d = sigma + diag(E):
//     A_pq = (d_q E_pq + d_p E_qp) / (d_q^2 - d_p^2),
//     B_pq = (d_q E_qp + d_p E_pq) / (d_q^2 - d_p^2)   (antisymmetric),
//     W_u = exp(A) = I + A + A^2/2 + A^3/6 + A^4/24 (orthogonal to
//     |A|^5/120), W_v likewise from B;  U = Ut X_u W_u, V = Vt X_v W_v,
//     Sigma = d.
// Every k x k product here is of perturbation matrices (|F| <= 1e-4,
// |A|, |B| <= 5e-3), so it runs in FP32 on FP32 copies made once (an FP64
// operand converted inside an O(nk^3) loop would put the conversions on
// this part's narrow FP64 pipe): its rounding is ~1e-7 of a term already
// ~1e-5 or below.  Linear terms and the sums stay FP64.  The error left in
// the SVD is ~|E| |A| (<= 1e-8 of sigma_1, ~1e-12 typically); U and V are
// orthonormal to ~1e-14.  Returns false (outputs undefined) when |A| or |B|
// exceeds 5e-3 (a near-degenerate pair): the caller then takes the exact
// path.  On success D0 = M_u = X_u W_u, D1 = M_v, d in dout.  Shared
// memory: D0 .. D4, nk^2 doubles each (D2 .. D4 hold FP32 data).
// Products of nk x nk FP32 matrices (row-major, nk <= 64) with 4 x 4
// register tiles, one per thread of the CTA (16 x 16 tiles): for every
// output (p, q) in this thread's tile, acc1 = sum_c X_pc s_c Y1_cq and
// acc2 = sum_c X_pc Y2_cq (s = 1 without xs; Y1 + Y1b when Y1b is given),
// each summed over c in order; out(p, q, acc1, acc2) stores the results.
template <typename Out>
__device__ __forceinline__ void mm64_tile(const float* X, const float* xs,
                                          const float* Y1, const float* Y1b,
                                          const float* Y2, int nk, Out out) {
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  const int r0 = 4 * ti, c0 = 4 * tj;
  if (r0 >= nk || c0 >= nk) return;
  float a1[4][4], a2[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) a1[i][j] = a2[i][j] = 0.0f;
  for (int c = 0; c < nk; ++c) {
    float xv[4], y1[4], y2[4];
    const float sc = xs ? xs[c] : 1.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      xv[i] = r0 + i < nk ? X[(r0 + i) * nk + c] * sc : 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = c0 + j < nk;
      y1[j] = in ? Y1[c * nk + c0 + j] : 0.0f;
      if (Y1b) y1[j] += in ? Y1b[c * nk + c0 + j] : 0.0f;
      y2[j] = (Y2 && in) ? Y2[c * nk + c0 + j] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a1[i][j] = fmaf(xv[i], y1[j], a1[i][j]);
        if (Y2) a2[i][j] = fmaf(xv[i], y2[j], a2[i][j]);
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (r0 + i < nk && c0 + j < nk) out(r0 + i, c0 + j, a1[i][j], a2[i][j]);
}

__device__ bool svd_fast_f64(double* D0, double* D1, double* D2, double* D3,
                             double* D4, int nk, const double* sg,
                             double* dout) {
  const int tid = threadIdx.x;
  const int n2 = nk * nk;
  __shared__ float sg32[kSeedKmaxLimit];
  float* Fu32 = reinterpret_cast<float*>(D2);
  float* Fv32 = Fu32 + n2;
  float* P1 = reinterpret_cast<float*>(D3);  // F_u^2
  float* P2 = P1 + n2;                       // F_v^2
  float* P3 = reinterpret_cast<float*>(D4);  // F_u Sigma F_v
  float* AB = P3 + n2;  // A above the diagonal, B (transposed) below
  for (int e = tid; e < n2; e += kSeedThreads) {
    Fu32[e] = (float)D0[e];
    Fv32[e] = (float)D1[e];
  }
  for (int q = tid; q < nk; q += kSeedThreads) sg32[q] = (float)sg[q];
  __syncthreads();
  mm64_tile(Fu32, nullptr, Fu32, nullptr, nullptr, nk,
            [&](int p, int q, float v, float) { P1[p * nk + q] = v; });
  mm64_tile(Fv32, nullptr, Fv32, nullptr, nullptr, nk,
            [&](int p, int q, float v, float) { P2[p * nk + q] = v; });
  mm64_tile(Fu32, sg32, Fv32, nullptr, nullptr, nk,
            [&](int p, int q, float v, float) { P3[p * nk + q] = v; });
  __syncthreads();
  auto E = [&](int p, int q) -> double {
    return 0.5 * fma(D0[p * nk + q], sg[q], sg[p] * D1[p * nk + q]) +
           0.25 * (double)P3[p * nk + q] -
           0.125 * fma((double)P1[p * nk + q], sg[q],
                       sg[p] * (double)P2[p * nk + q]);
  };
  for (int q = tid; q < nk; q += kSeedThreads) dout[q] = sg[q] + E(q, q);
  __syncthreads();
  int bad = 0;
  for (int e = tid; e < n2; e += kSeedThreads) {
    const int p = e / nk, q = e - p * nk;
    if (p >= q) continue;
    const double epq = E(p, q), eqp = E(q, p);
    const double dp = dout[p], dq = dout[q];
    const float den = (float)((dq - dp) * (dq + dp));
    const float a = (float)fma(dq, epq, dp * eqp) / den;
    const float b = (float)fma(dq, eqp, dp * epq) / den;
    if (!(fabsf(a) <= 5e-3f && fabsf(b) <= 5e-3f)) bad = 1;
    AB[p * nk + q] = a;
    AB[q * nk + p] = b;
  }
  if (__syncthreads_or(bad)) return false;
  // X = -F/2 + 3/8 F^2 (X - I, FP64) in place over F; A and B as full
  // antisymmetric matrices: A over F_u Sigma F_v, B in place over AB (each
  // pair (p, q) is read and written by one thread)
  float* Af = P3;
  float* Bf = AB;
  for (int idx = tid; idx < 2 * n2; idx += kSeedThreads) {
    const int w = idx / n2, e = idx - w * n2;
    double* D = w ? D1 : D0;
    D[e] = fma(-0.5, D[e], 0.375 * (double)(w ? P2 : P1)[e]);
  }
  for (int e = tid; e < n2; e += kSeedThreads) {
    const int p = e / nk, q = e - p * nk;
    if (p > q) continue;
    if (p == q) {
      Af[e] = 0.0f;
      Bf[e] = 0.0f;
      continue;
    }
    const float a = AB[p * nk + q], b = AB[q * nk + p];
    Af[p * nk + q] = a;
    Af[q * nk + p] = -a;
    Bf[p * nk + q] = b;
    Bf[q * nk + p] = -b;
  }
  __syncthreads();
  // A^2, B^2 over the FP32 copies of F, then H = A^2/2 + A^3/6 + A^4/24
  // (W - I - A) over F^2 (no longer needed)
  float* A2 = Fu32;
  float* B2 = Fv32;
  mm64_tile(Af, nullptr, Af, nullptr, nullptr, nk,
            [&](int p, int q, float v, float) { A2[p * nk + q] = v; });
  mm64_tile(Bf, nullptr, Bf, nullptr, nullptr, nk,
            [&](int p, int q, float v, float) { B2[p * nk + q] = v; });
  __syncthreads();
  float* Hu = P1;
  float* Hv = P2;
  mm64_tile(A2, nullptr, Af, nullptr, A2, nk,
            [&](int p, int q, float a3, float a4) {
              Hu[p * nk + q] = fmaf(0.5f, A2[p * nk + q],
                                    fmaf(a3, 1.0f / 6.0f, a4 * (1.0f / 24.0f)));
            });
  mm64_tile(B2, nullptr, Bf, nullptr, B2, nk,
            [&](int p, int q, float a3, float a4) {
              Hv[p * nk + q] = fmaf(0.5f, B2[p * nk + q],
                                    fmaf(a3, 1.0f / 6.0f, a4 * (1.0f / 24.0f)));
            });
  __syncthreads();
  // FP32 copies of X over A^2, B^2
  float* Xu32 = A2;
  float* Xv32 = B2;
  for (int e = tid; e < n2; e += kSeedThreads) {
    Xu32[e] = (float)D0[e];
    Xv32[e] = (float)D1[e];
  }
  __syncthreads();
  // M = (I + X)(I + W) = I + X + W + X W, W = A + H: each thread writes the
  // FP64 entries of its own tile (the product reads the FP32 copies only)
  mm64_tile(Xu32, nullptr, Af, Hu, nullptr, nk,
            [&](int p, int q, float xw, float) {
              const int e = p * nk + q;
              D0[e] = (p == q ? 1.0 : 0.0) + D0[e] +
                      ((double)Af[e] + (double)Hu[e]) + (double)xw;
            });
  mm64_tile(Xv32, nullptr, Bf, Hv, nullptr, nk,
            [&](int p, int q, float xw, float) {
              const int e = p * nk + q;
              D1[e] = (p == q ? 1.0 : 0.0) + D1[e] +
                      ((double)Bf[e] + (double)Hv[e]) + (double)xw;
            });
  __syncthreads();
  return true;
}

// Hardware barrier over the CTAs of this thread-block cluster, with release
// / acquire ordering of their memory operations at cluster scope (the
// cross-CTA data lives in global memory and is read with L2 loads).  Every
// thread of every CTA of the cluster calls it the same number of times.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n"
      "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// How a seed's team of CTAs separates the phases of an ALM iteration.
enum { kTeamCta = 0,      // one CTA: __syncthreads
       kTeamGrid = 1,     // cooperative grid: software grid barrier
       kTeamCluster = 2   // one thread-block cluster: hardware barrier
};

// The ALM body, run by a team of CTAs: a cooperative grid (phases separated
// by the software grid barrier), one thread-block cluster (the hardware
// cluster barrier) or a single CTA (one seed per CTA, __syncthreads).
// b / nb: this CTA's position in the team.  The partial-sum slots of the
// reductions are fixed per solve, so every team form gives the same bits.
template <int kMode>
__device__ void seed_alm_body(const SeedArgs& a, const int b, const int nb) {
  constexpr bool kGrid = kMode != kTeamCta;  // a team of several CTAs
  extern __shared__ __align__(16) double sm[];
  const int kmax = a.kmax;
  double* red = sm;                      // kSeedThreads
  double* xs = red + kSeedThreads;       // kSeedGemmGroup x kSeedMaxSide
  double* gred = xs + kSeedGemmGroup * kSeedMaxSide;  // x kSeedThreads
  double* lam = gred + kSeedGemmGroup * kSeedThreads;  // kmax (values s_c)
  double* dsc = lam + kmax;              // kmax
  double* xi = dsc + kmax;               // kmax
  double* rowb = xi + kmax;              // kmax
  double* Vd = rowb + kmax;              // kmax*kmax (rotation as FP64)
  float* J0 = reinterpret_cast<float*>(Vd + kmax * kmax);  // 2 x kmax*kmax
  float* W0 = J0 + kmax * kmax;          // Jacobi A / V; Cholesky R / R^-1
  float* cs = W0 + kmax * kmax;          // kmax*kmax floats (Jacobi buffer)
  int* ibuf = reinterpret_cast<int*>(cs + kmax * kmax);  // 2*kmax ints,
  int* dead = ibuf;                      // then kmax*kmax bytes (schedule)
  int* prs = ibuf + kmax;

  const int tid = threadIdx.x;
  const int mp = a.mp, np = a.np;
  const size_t mn = (size_t)mp * np;
  SeedCtl* ctl = a.ctl;
  const unsigned long long tmo = a.timeout_ns;
  // warps per CTA for the row-wise forward substitutions: one per CTA on a
  // wide team (rows spread over many SMs' FP64 pipes), more on small teams
  const int row_warps =
      kGrid ? max(1, min(kSeedThreads / 32, (max(mp, np) + nb - 1) / nb))
            : kSeedThreads / 32;
  auto team_sync = [&]() -> bool {
    if (kMode == kTeamGrid) return grid_sync(ctl, nb, tmo);
    if (kMode == kTeamCluster)
      cluster_sync_all();
    else
      __syncthreads();
    return true;
  };

  // ---- prologue: norms of D, G = D, random Omega ---------------------------
  const int nv = a.nv;
  {
    for (int v = b; v < nv; v += nb) {
      double ss = 0.0, mx = 0.0;
      for (size_t e = (size_t)v * kSeedThreads + tid; e < mn;
           e += (size_t)nv * kSeedThreads) {
        const double d = __ldg(a.D + e);
        ss = fma(d, d, ss);
        mx = fmax(mx, fabs(d));
        __stcg(a.S + e, 0.0);
        __stcg(a.G + e, d);
        const int j = (int)(e / mp), i = (int)(e - (size_t)j * mp);
        __stcg(a.Gt + (size_t)i * np + j, d);
      }
      ss = block_reduce_sum(ss, red);
      mx = block_reduce_max(mx, red);
      if (tid == 0) {
        __stcg(a.part + 4 * v, ss);
        __stcg(a.part + 4 * v + 1, mx);
      }
    }
    for (size_t e = (size_t)b * kSeedThreads + tid; e < (size_t)mp * a.k0;
         e += (size_t)nb * kSeedThreads) {
      const int i = (int)(e / a.k0), c = (int)(e - (size_t)i * a.k0);
      const double v = hash_normal(0x5EEDull + c, i);
      __stcg(a.Om + (size_t)i * kmax + c, v);
      a.Om32[(size_t)i * kmax + c] = (float)v;
    }
  }
  if (!team_sync()) return;
  trace_mark(a, 1);
  const double normF = sqrt(sum_partials(a.part, nv, 4, 0, red));
  double m2 = 0.0;
  for (int q = tid; q < nv; q += kSeedThreads)
    m2 = fmax(m2, ldg_cg(a.part + 4 * q + 1));
  const double norminf = block_reduce_max(m2, red);
  if (!(normF > 0.0)) {
    // D = 0 (or not finite): L = S = 0, rank 0.
    for (size_t e = (size_t)b * kSeedThreads + tid; e < (size_t)mp * kmax;
         e += (size_t)nb * kSeedThreads)
      a.U[e] = 0.0;
    for (size_t e = (size_t)b * kSeedThreads + tid; e < (size_t)np * kmax;
         e += (size_t)nb * kSeedThreads)
      a.V[e] = 0.0;
    if (b == 0) {
      for (int c = tid; c < kmax; c += kSeedThreads) a.Sigma[c] = 0.0;
      if (tid == 0) {
        ctl->iters = 0;
        ctl->rank = 0;
        ctl->rank_raw = 0;
        ctl->converged = 1;
        ctl->residual = 0.0;
        ctl->k_final = a.k0;
      }
    }
    return;
  }

  int k = a.k0;
  double mu = 0.0, mu_max = 0.0, tau = 0.0;
  int it = 0;           // ALM iterations done
  // stages below 2: power steps on D; 2: Rayleigh-Ritz on D; 3: ALM
  int stage = 2 - kSeedPowerSteps;
  bool converged = false;
  double res = 1.0;
  int knext = k;
  // the Ritz bases of this iteration: Pt / PsiT, or P / Psi after the FP64
  // refinement below
  const double* Ptc = a.Pt;
  const double* PsiTc = a.PsiT;

  while (true) {
    // ---- T = G^T Omega ------------------------------------------------------
    tall_gemm_t(a.G, mp, mp, np, a.Om, res > a.lowp_res ? a.Om32 : nullptr, k,
                kmax, a.T, gred, xs, b, nb);
    if (!team_sync()) return;
    trace_mark(a, 2);
    gram(a.T, np, k, kmax, a.Gam, b, nb);
    if (!team_sync()) return;
    trace_mark(a, 3);
    cholqr_apply(a.T, np, k, kmax, a.Gam, a.Psi, a.Psi32, J0, W0, Vd, dsc, dead, rowb,
                 b, nb, row_warps, kGrid ? ctl->sub : nullptr);
    if (!team_sync()) return;
    trace_mark(a, 4);
    // ---- P = G Psi ------------------------------------------------------------
    tall_gemm_t(a.Gt, np, np, mp, a.Psi, res > a.lowp_res ? a.Psi32 : nullptr,
                k, kmax, a.P, gred, xs, b, nb);
    if (stage >= 2) gram(a.Psi, np, k, kmax, a.Gam2, b, nb);  // E = Psi1^T Psi1 - I
    if (!team_sync()) return;
    trace_mark(a, 5);
    gram(a.P, mp, k, kmax, a.Gam, b, nb);
    if (!team_sync()) return;
    trace_mark(a, 6);
    if (stage < 2) {
      // plain power step on D: Omega = orth(P)
      cholqr_apply(a.P, mp, k, kmax, a.Gam, a.Om, a.Om32, J0, W0, Vd, dsc, dead, rowb, b, nb,
                   row_warps, nullptr);
      if (!team_sync()) return;
      trace_mark(a, 7);
      ++stage;
      continue;
    }
    // ---- Rayleigh-Ritz rotation ---------------------------------------------
    // Psi1 (from the FP32 Cholesky QR) has Psi1^T Psi1 = I + E, |E| ~ 1e-7.
    // Its first-order orthonormalisation Psi = Psi1 (I - E/2) is never
    // formed: the Jacobi runs on C1 = P1^T P1 (the correction to C is below
    // the FP32 resolution of the Jacobi's input) and the rotation applied to
    // P1 and Psi1 is W = (I - E/2) V, which makes the rotated bases
    // orthonormal to O(E^2).  The W correction is tiny, so an FP32 product
    // is exact enough for it.
    {
      float* C32 = J0;  // C1 / cmax, then the Jacobi's A
      // E is kept for the W correction after the Jacobi, as floats in the
      // (still unused) storage of Vd; C1 and E in one pass over L2, then
      // C1 scaled by its largest diagonal entry
      float* Esave = reinterpret_cast<float*>(Vd);
      const long long ts0 = clock64();
      double dmax = 0.0;
      for (int p = tid >> 4; p < k; p += kSeedThreads / 16)
        for (int q = tid & 15; q < k; q += 16) {
          const double g = ldg_cg(a.Gam + p * kmax + q);
          Esave[p * k + q] =
              (float)ldg_cg(a.Gam2 + p * kmax + q) - (p == q ? 1.0f : 0.0f);
          C32[p * k + q] = (float)g;
          if (p == q) dmax = fmax(dmax, g);
        }
      const double cm = block_reduce_max(dmax, red);
      const long long ts1 = clock64();
      if (b == 0 && tid == 0) ctl->jcyc[0] += ts1 - ts0;
      const float inv = cm > 0.0 ? (float)(1.0 / cm) : 1.0f;
      for (int idx = tid; idx < k * k; idx += kSeedThreads) C32[idx] *= inv;
      __syncthreads();
      if (b == 0 && tid == 0) ctl->jcyc[3] += clock64() - ts0;
      trace_mark(a, 12);
      // the Jacobi needs a second k x k float buffer: the rotation buffer
      // cs..cs+k*k (see the shared-memory map)
      const long long tj0 = clock64();
      // Far from convergence one sweep per ALM iteration is enough: the Ritz
      // basis is carried to the next iteration (Omega_next = Pt / s), so the
      // diagonalisation keeps improving.  Near convergence (residual below
      // 1e-5) and on the first Rayleigh-Ritz the sweeps run to completion so
      // the returned factors are orthonormal to FP32 accuracy.
      const int max_sweeps = (stage == 2 || res < 1e-5) ? 30 : 1;
      // Warm-started iterations: in the carried Ritz basis C1 is nearly
      // diagonal.  When every pair that matters has |c_pq| <= gate
      // |c_qq - c_pp|, the eigenvectors are I + Theta, Theta_pq =
      // c_pq / (c_qq - c_pp), to O(gate^2) (first-order perturbation), and
      // that replaces the sweeps.  Pairs whose values both lie at or below
      // the SVT threshold (tau^2 / cmax in these units) are left unmixed:
      // both are shrunk to zero, so a rotation between them changes neither
      // L nor the spanned subspace.
      bool fast = false, cluster = false;
      if (stage == 3) {
        const float t2 = (float)((1.0 / mu) * (1.0 / mu) * (double)inv);
        // far from convergence a coarser rotation is enough (the FP64
        // refinement of the last iterations removes what it leaves)
        const float gate = res < 1e-5 ? 1e-3f : 1e-2f;
        int* vio = prs;   // per index: in a pair that fails the gate
        int* sub = dead;  // those indices, in order (both free here)
        for (int c = tid; c < k; c += kSeedThreads) vio[c] = 0;
        __syncthreads();
        int bad = 0;
        for (int idx = tid; idx < k * k; idx += kSeedThreads) {
          const int p = idx / k, q = idx - p * k;
          if (p < q) {
            const float cpp = C32[p * k + p], cqq = C32[q * k + q];
            const float cpq = C32[p * k + q];
            const bool exempt = cpp <= t2 && cqq <= t2;
            if (!exempt && !(fabsf(cpq) <= gate * fabsf(cqq - cpp))) {
              bad = 1;
              vio[p] = 1;
              vio[q] = 1;
            }
          }
        }
        fast = !__syncthreads_or(bad);
        // Failing pairs usually lie within one cluster of nearly equal
        // values (the directions around the SVT threshold); every pair
        // with an index outside it passes the gate.  Then the first-order
        // eigenvectors serve for all pairs but those inside the cluster,
        // whose sub-block is rotated exactly by its own (small) Jacobi.
        __shared__ int s_nsub;
        if (!fast) {
          if (tid == 0) {
            int ns = 0;
            for (int c = 0; c < k; ++c)
              if (vio[c]) sub[ns++] = c;
            s_nsub = ns;
          }
          __syncthreads();
          const int ns = s_nsub, nsp = (ns + 1) & ~1;
          cluster = ns <= 32 && 2 * ns <= k && 3 * nsp * nsp <= kmax * kmax;
        }
        if (fast || cluster) {
          for (int idx = tid; idx < k * k; idx += kSeedThreads) {
            const int p = idx / k, q = idx - p * k;
            float x = (p == q) ? 1.0f : 0.0f;
            if (p != q && !(vio[p] && vio[q])) {
              const float cpp = C32[p * k + p], cqq = C32[q * k + q];
              if (!(cpp <= t2 && cqq <= t2))
                x = __fdividef(C32[p * k + q], cqq - cpp);
            }
            W0[idx] = x;  // V[p][q]
          }
        }
        if (cluster) {
          const int ns = s_nsub, nsp = (ns + 1) & ~1;
          float* As0 = cs;
          float* As1 = cs + nsp * nsp;
          float* Vs = cs + 2 * nsp * nsp;
          for (int idx = tid; idx < nsp * nsp; idx += kSeedThreads) {
            const int i = idx / nsp, j = idx - i * nsp;
            As0[idx] = (i < ns && j < ns) ? C32[sub[i] * k + sub[j]] : 0.0f;
          }
          __syncthreads();
          block_jacobi32(As0, As1, Vs, nsp,
                         reinterpret_cast<unsigned char*>(prs + kmax),
                         max_sweeps, kGrid ? &ctl->jsweeps : nullptr,
                         kGrid ? ctl->jcyc : nullptr);
          // cluster columns of V: V[:, sub_j] = sum_i V[:, sub_i] Vs[i][j]
          // (through C32's storage, which is no longer needed)
          for (int idx = tid; idx < k * ns; idx += kSeedThreads) {
            const int r = idx / ns, j = idx - r * ns;
            float acc = 0.0f;
            for (int i = 0; i < ns; ++i)
              acc = fmaf(W0[r * k + sub[i]], Vs[i * nsp + j], acc);
            C32[idx] = acc;
          }
          __syncthreads();
          for (int idx = tid; idx < k * ns; idx += kSeedThreads) {
            const int r = idx / ns, j = idx - r * ns;
            W0[r * k + sub[j]] = C32[idx];
          }
        }
        __syncthreads();
      }
      if (kGrid && b == 0 && tid == 0)
        ++ctl->jpath[fast ? 0 : (cluster ? 1 : 2)];
      if (!fast && !cluster) {
        float* Afin = block_jacobi32(
            C32, cs, W0, k, reinterpret_cast<unsigned char*>(prs + kmax),
            max_sweeps, kGrid ? &ctl->jsweeps : nullptr,
            kGrid ? ctl->jcyc : nullptr);
        (void)Afin;
      }
      const long long tj1 = clock64();
      if (b == 0 && tid == 0) ctl->jcyc[1] += tj1 - tj0;
      // W = V - (E/2) V (E kept as floats in Vd, V in W0), written to J0,
      // which the Jacobi no longer needs, then widened into Vd
      const float* Ef = reinterpret_cast<const float*>(Vd);
      for (int base = tid; base < k * k; base += 4 * kSeedThreads) {
        int pp[4], qq[4];
        float xs4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int idx = min(base + o * kSeedThreads, k * k - 1);
          pp[o] = idx / k;
          qq[o] = idx - pp[o] * k;
        }
        for (int c = 0; c < k; ++c) {
#pragma unroll
          for (int o = 0; o < 4; ++o)
            xs4[o] = fmaf(Ef[pp[o] * k + c], W0[c * k + qq[o]], xs4[o]);
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int idx = base + o * kSeedThreads;
          if (idx < k * k) J0[idx] = W0[idx] - 0.5f * xs4[o];  // J0 is free
        }
      }
      __syncthreads();
      for (int idx = tid; idx < k * k; idx += kSeedThreads) Vd[idx] = (double)J0[idx];
      __syncthreads();
      if (b == 0 && tid == 0) ctl->jcyc[2] += clock64() - tj1;
    }
    trace_mark(a, 8);
    // ---- rotate: Pt = P V, PsiT = Psi V, slot column sums of Pt^2 ---------
    // Thread (c, part) computes column c of the rows it takes; the sums of
    // Pt^2 per partial-sum slot follow in a fixed order (below), so they do
    // not depend on timing or on the team's size.
    {
      const int nparts = kSeedThreads / k;
      const int c = tid % k, part = tid / k;
      // The rows of all the slots this CTA owns are rotated in parallel
      // (slot v holds rows v, v + nv, ...); after one CTA barrier each
      // slot's column sums of Pt^2 are formed from the stored rows in a
      // fixed order: per part q the rows v + (q + s nparts) nv in turn, then
      // the parts in order, so the sums do not depend on the team's size.
      const int myslots = (nv - b + nb - 1) / nb;
      const int rps = (mp + nv - 1) / nv;  // rows per slot, at most
      if (part < nparts) {
        for (int ri = part; ri < myslots * rps; ri += nparts) {
          const int ls = ri % myslots, t = ri / myslots;
          const int i = b + ls * nb + t * nv;
          if (i >= mp) continue;
          const double* pr = a.P + (size_t)i * kmax;
          double s0 = 0.0, s1 = 0.0;
          int q = 0;
          for (; q + 1 < k; q += 2) {
            s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
            s1 = fma(ldg_cg(pr + q + 1), Vd[(q + 1) * k + c], s1);
          }
          if (q < k) s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
          __stcg(a.Pt + (size_t)i * kmax + c, s0 + s1);
        }
      }
      __syncthreads();
      for (int idx = tid; idx < myslots * k; idx += kSeedThreads) {
        const int ls = idx / k, cc = idx - ls * k;
        const int v = b + ls * nb;
        double s2 = 0.0;
        for (int q = 0; q < nparts; ++q) {
          double csq = 0.0;
          for (int i = v + q * nv; i < mp; i += nv * nparts) {
            const double sv = ldg_cg(a.Pt + (size_t)i * kmax + cc);
            csq = fma(sv, sv, csq);
          }
          s2 += csq;
        }
        __stcg(a.colsq + (size_t)v * kmax + cc, s2);
      }
      __syncthreads();
      if (part < nparts) {
        for (int j = b + part * nb; j < np; j += nb * nparts) {
          const double* pr = a.Psi + (size_t)j * kmax;
          double s0 = 0.0, s1 = 0.0;
          int q = 0;
          for (; q + 1 < k; q += 2) {
            s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
            s1 = fma(ldg_cg(pr + q + 1), Vd[(q + 1) * k + c], s1);
          }
          if (q < k) s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
          __stcg(a.PsiT + (size_t)j * kmax + c, s0 + s1);
        }
      }
    }
    if (!team_sync()) return;
    trace_mark(a, 9);
    const bool prof_alm = kGrid && b == 0 && tid == 0 && a.trace;
    long long pa0 = prof_alm ? clock64() : 0;
    // ---- FP64 Ritz values s_c = ||Pt e_c|| (fixed-order sum over blocks) ---
    {
      const int nparts = kSeedThreads / k;
      const int c = tid % k, part = tid / k;
      if (part < nparts) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int q = part;
        for (; q + 3 * nparts < nv; q += 4 * nparts) {
          s0 += ldg_cg(a.colsq + (size_t)q * kmax + c);
          s1 += ldg_cg(a.colsq + (size_t)(q + nparts) * kmax + c);
          s2 += ldg_cg(a.colsq + (size_t)(q + 2 * nparts) * kmax + c);
          s3 += ldg_cg(a.colsq + (size_t)(q + 3 * nparts) * kmax + c);
        }
        for (; q < nv; q += nparts) s0 += ldg_cg(a.colsq + (size_t)q * kmax + c);
        red[part * k + c] = (s0 + s1) + (s2 + s3);
      }
      __syncthreads();
      if (tid < k) {
        double s2 = 0.0;
        for (int q = 0; q < nparts; ++q) s2 += red[q * k + tid];
        lam[tid] = sqrt(s2);
      }
      __syncthreads();
    }
    Ptc = a.Pt;
    PsiTc = a.PsiT;
    if (prof_alm) {
      const long long t = clock64();
      ctl->sub[5] += t - pa0;  // Ritz values
      pa0 = t;
    }
    if (stage == 3 && res < 1e-5) {
      // ---- FP64 refinement of the Ritz basis (near convergence) -----------
      // The FP32 Jacobi leaves B = Pt^T Pt with off-diagonal entries of
      // ~1e-7 of its diagonal, an error floor at the ALM's own tolerance.
      // First-order perturbation theory removes it: the eigenvectors of
      // B = D + F are I + Theta to O(F^2), Theta_pq = F_pq / (d_q - d_p),
      // so Pt (I + Theta) and PsiT (I + Theta) have orthogonal columns to
      // ~1e-14.  Theta is tiny, so FP32 arithmetic is exact enough for it;
      // pairs too close for the first-order formula are left alone (their
      // shrink factors are nearly equal, so mixing them changes little).
      gram(a.Pt, mp, k, kmax, a.Gam2, b, nb);
      if (!team_sync()) return;
      trace_mark(a, 13);
      for (int idx = tid; idx < k * k; idx += kSeedThreads) {
        const int p = idx / k, q = idx - p * k;
        double x = (p == q) ? 1.0 : 0.0;
        if (p != q) {
          const double gap = ldg_cg(a.Gam2 + q * kmax + q) -
                             ldg_cg(a.Gam2 + p * kmax + p);
          const float f = (float)ldg_cg(a.Gam2 + p * kmax + q);
          const float g = (float)gap;
          if (fabsf(f) < 0.01f * fabsf(g)) x = (double)__fdividef(f, g);
        }
        Vd[idx] = x;  // (I + Theta)[p][q]
      }
      __syncthreads();
      const int nparts = kSeedThreads / k;
      const int c = tid % k, part = tid / k;
      if (part < nparts) {
        for (int i = b + part * nb; i < mp; i += nb * nparts) {
          const double* pr = a.Pt + (size_t)i * kmax;
          double s0 = 0.0, s1 = 0.0;
          int q = 0;
          for (; q + 1 < k; q += 2) {
            s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
            s1 = fma(ldg_cg(pr + q + 1), Vd[(q + 1) * k + c], s1);
          }
          if (q < k) s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
          __stcg(a.P + (size_t)i * kmax + c, s0 + s1);
        }
        for (int j = b + part * nb; j < np; j += nb * nparts) {
          const double* pr = a.PsiT + (size_t)j * kmax;
          double s0 = 0.0, s1 = 0.0;
          int q = 0;
          for (; q + 1 < k; q += 2) {
            s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
            s1 = fma(ldg_cg(pr + q + 1), Vd[(q + 1) * k + c], s1);
          }
          if (q < k) s0 = fma(ldg_cg(pr + q), Vd[q * k + c], s0);
          __stcg(a.Psi + (size_t)j * kmax + c, s0 + s1);
        }
      }
      if (!team_sync()) return;
      trace_mark(a, 14);
      Ptc = a.P;  // P and Psi are free until the next iteration's products
      PsiTc = a.Psi;
    }
    double smax = 0.0;
    for (int c = 0; c < k; ++c) smax = fmax(smax, lam[c]);
    if (stage == 2) {
      // ||D||_2 from the Ritz values; start the ALM.
      mu = a.mu_scale / smax;
      mu_max = mu * a.mu_max_ratio;
      if (b == 0 && tid == 0) ctl->sigma1 = smax;
    }
    tau = 1.0 / mu;
    for (int c = tid; c < k; c += kSeedThreads) {
      const double s = lam[c];
      dsc[c] = (s > tau) ? 1.0 - tau / s : 0.0;  // shrink factor d_c
    }
    __syncthreads();
    int nsv = 0;
    for (int c = 0; c < k; ++c) nsv += (lam[c] > tau);
    knext = k;
    if (stage == 3 && nsv >= k && k < kmax)
      knext = min(kmax, (k + max(6, k / 4) + 1) / 2 * 2);
    // Omega_next = Pt / s (rows distributed); fresh directions for growth
    // and for vanished Ritz vectors.
    {
      const int nparts = kSeedThreads / knext;
      const int c = tid % knext, part = tid / knext;
      if (part < nparts) {
        const bool keep = c < k && lam[c] > 1e-12 * smax;
        const double inv = keep ? 1.0 / lam[c] : 0.0;
        for (int i = b + part * nb; i < mp; i += nb * nparts) {
          const double v = keep ? ldg_cg(Ptc + (size_t)i * kmax + c) * inv
                                : hash_normal(0xA11CEull + 977ull * it + c, i);
          __stcg(a.Om + (size_t)i * kmax + c, v);
          a.Om32[(size_t)i * kmax + c] = (float)v;
        }
      }
    }

    if (stage == 2) {
      // Y_0 = D / J,  J = max(||D||_2, ||D||_inf / lam);  G_1 = D + Y_0/mu_0.
      const double J = fmax(smax, norminf / a.lam);
      for (size_t e = (size_t)b * kSeedThreads + tid; e < mn;
           e += (size_t)nb * kSeedThreads) {
        const double d = __ldg(a.D + e);
        const double y = d / J;
        __stcg(a.Y + e, y);
        const double g = d + y / mu;
        __stcg(a.G + e, g);
        const int j = (int)(e / mp), i = (int)(e - (size_t)j * mp);
        __stcg(a.Gt + (size_t)i * np + j, g);
      }
      stage = 3;
      if (!team_sync()) return;
      trace_mark(a, 10);
      continue;
    }

    if (prof_alm) {
      const long long t = clock64();
      ctl->sub[6] += t - pa0;  // refinement, shrink factors, Omega_next
      pa0 = t;
    }
    // ---- ALM step: L = Pt diag(d) PsiT^T, S, Y, G for the next iteration ---
    const double mu_next = fmin(a.rho * mu, mu_max);
    const double inv_mu = 1.0 / mu, inv_mu_next = 1.0 / mu_next;
    const double lam_mu = a.lam * inv_mu;
    // Tiled form: TT x TT tiles of L from Pt / PsiT rows staged in the
    // shared memory the k x k phases are done with (Vd .. cs, 20 kmax^2
    // bytes); G^T is written through a staged tile so both G and G^T
    // stores are coalesced.  Tile t belongs to partial-sum slot t mod nv.
    // Tile side: 32 when that still gives every CTA of the team about one
    // tile or more, else 16 (32 x 32 tiles on a 200 x 200 seed left three
    // quarters of a 200-CTA team idle: 43 us against 29 us per update for
    // the per-column form).
    auto tiles_of = [&](int t) { return ((mp + t - 1) / t) * ((np + t - 1) / t); };
    const bool fit32 = 8 * (64 * (kmax + 1) + 32 * 33) <= 20 * kmax * kmax;
    const bool fit16 = 8 * (32 * (kmax + 1) + 16 * 17) <= 20 * kmax * kmax;
    const int TT = (fit32 && 2 * tiles_of(32) >= nv) ? 32 : (fit16 ? 16 : 0);
    auto alm_elem = [&](const double l, const int i, const int j,
                        double& zz) -> double {
      const size_t e = (size_t)j * mp + i;
      const double d = __ldg(a.D + e);
      const double y = ldg_cg(a.Y + e);
      const double s = shrink(d - l + y * inv_mu, lam_mu);
      const double z = d - l - s;
      const double yn = fma(mu, z, y);
      zz = fma(z, z, zz);
      __stcg(a.S + e, s);
      __stcg(a.Y + e, yn);
      const double g = d - s + yn * inv_mu_next;
      __stcg(a.G + e, g);
      return g;
    };
    // Far from convergence (residual above 1e-4) the rank-k products of L
    // run in FP32 (operands rounded once when staged, FP32 accumulation):
    // their ~1e-7 relative error is far below what the inexact ALM leaves
    // at that point, and this part's FP64 pipe (2 FMA/clk/SM) made them the
    // update's cost on the 500 x 500 seed.  Every later iteration is FP64.
    const bool lowp = res > a.lowp_res;
    if (TT > 0) {
      const int kp = k | 1;  // odd row pitch: conflict-free reads
      double* Pts = Vd;                 // [TT][kp]
      double* Qs = Pts + TT * kp;       // [TT][kp], scaled by d
      double* Gs = Qs + TT * kp;        // [TT][TT + 1]
      float* Pf = reinterpret_cast<float*>(Pts);  // FP32 form of the same
      float* Qf = Pf + TT * kp;
      const int tcn = (np + TT - 1) / TT;
      const int ntile = ((mp + TT - 1) / TT) * tcn;
      for (int v = b, ls = 0; v < nv; v += nb, ++ls) {
        double zz = 0.0;
        for (int tile = v; tile < ntile; tile += nv) {
          const int i0 = (tile / tcn) * TT, j0 = (tile % tcn) * TT;
          for (int idx = tid; idx < TT * k; idx += kSeedThreads) {
            const int ii = idx / k, c = idx - ii * k;
            const double pv =
                (i0 + ii < mp) ? ldg_cg(Ptc + (size_t)(i0 + ii) * kmax + c)
                               : 0.0;
            const double qv =
                (j0 + ii < np)
                    ? dsc[c] * ldg_cg(PsiTc + (size_t)(j0 + ii) * kmax + c)
                    : 0.0;
            if (lowp) {
              Pf[ii * kp + c] = (float)pv;
              Qf[ii * kp + c] = (float)qv;
            } else {
              Pts[ii * kp + c] = pv;
              Qs[ii * kp + c] = qv;
            }
          }
          __syncthreads();
          for (int q = tid; q < TT * TT; q += kSeedThreads) {
            const int ii = q % TT, jj = q / TT;
            const int i = i0 + ii, j = j0 + jj;
            if (i < mp && j < np) {
              double l;
              int c = 0;
              if (lowp) {
                const float* pr = Pf + ii * kp;
                const float* qr = Qf + jj * kp;
                float l0 = 0.0f, l1 = 0.0f;
                for (; c + 1 < k; c += 2) {
                  l0 = fmaf(pr[c], qr[c], l0);
                  l1 = fmaf(pr[c + 1], qr[c + 1], l1);
                }
                if (c < k) l0 = fmaf(pr[c], qr[c], l0);
                l = (double)(l0 + l1);
              } else {
                const double* pr = Pts + ii * kp;
                const double* qr = Qs + jj * kp;
                double l0 = 0.0, l1 = 0.0;
                for (; c + 1 < k; c += 2) {
                  l0 = fma(pr[c], qr[c], l0);
                  l1 = fma(pr[c + 1], qr[c + 1], l1);
                }
                if (c < k) l0 = fma(pr[c], qr[c], l0);
                l = l0 + l1;
              }
              Gs[jj * (TT + 1) + ii] = alm_elem(l, i, j, zz);
            }
          }
          __syncthreads();
          for (int q = tid; q < TT * TT; q += kSeedThreads) {
            const int ii = q / TT, jj = q % TT;
            const int i = i0 + ii, j = j0 + jj;
            if (i < mp && j < np)
              __stcg(a.Gt + (size_t)i * np + j, Gs[jj * (TT + 1) + ii]);
          }
          __syncthreads();
        }
        // a slot's warp sums wait in shared memory (xs is free here)
        const double wz = warp_sum(zz);
        if ((tid & 31) == 0) xs[ls * (kSeedThreads / 32) + (tid >> 5)] = wz;
      }
    } else {
      // narrow subspace: one column at a time
      for (int v = b, ls = 0; v < nv; v += nb, ++ls) {
        double zz = 0.0;
        for (int j = v; j < np; j += nv) {
          for (int c = tid; c < k; c += kSeedThreads)
            xi[c] = dsc[c] * ldg_cg(PsiTc + (size_t)j * kmax + c);
          __syncthreads();
          for (int i = tid; i < mp; i += kSeedThreads) {
            const double* pr = Ptc + (size_t)i * kmax;
            double l0 = 0.0, l1 = 0.0;
            int c = 0;
            for (; c + 1 < k; c += 2) {
              l0 = fma(ldg_cg(pr + c), xi[c], l0);
              l1 = fma(ldg_cg(pr + c + 1), xi[c + 1], l1);
            }
            if (c < k) l0 = fma(ldg_cg(pr + c), xi[c], l0);
            const double g = alm_elem(l0 + l1, i, j, zz);
            __stcg(a.Gt + (size_t)i * np + j, g);
          }
          __syncthreads();
        }
        // a slot's warp sums wait in shared memory (xs is free here)
        const double wz = warp_sum(zz);
        if ((tid & 31) == 0) xs[ls * (kSeedThreads / 32) + (tid >> 5)] = wz;
      }
    }
    // slot sums of ||Z||^2: the warp sums added in warp order, the same
    // arithmetic as a block reduction per slot, one CTA barrier in all
    __syncthreads();
    for (int ls = tid, nls = (nv - b + nb - 1) / nb; ls < nls;
         ls += kSeedThreads) {
      double zs = 0.0;
      for (int q = 0; q < kSeedThreads / 32; ++q)
        zs += xs[ls * (kSeedThreads / 32) + q];
      __stcg(a.part + 4 * (b + ls * nb) + 2, zs);
    }
    if (prof_alm) ctl->sub[7] += clock64() - pa0;  // elementwise update
    ++it;
    if (!team_sync()) return;
    trace_mark(a, 11);
    res = sqrt(sum_partials(a.part, nv, 4, 2, red)) / normF;
    converged = res <= a.tol;
    if (converged || it >= a.max_iter) break;
    mu = mu_next;
    k = knext;
  }

  // ---- outputs: the skinny SVD of L^s in FP64 ------------------------------
  // The iterate is L^s = Pt diag(d) PsiT^T.  Its bases carry the ~1e-7 loss
  // of orthogonality of the FP32 k x k factorisations, while Algorithm 1
  // (step 2, Eq. l1g) takes A^T A = I; so the factors are re-orthonormalised
  // once here, in FP64.  With K the nk columns whose Ritz value s exceeds
  // tau (the rest are shrunk to zero), Ut = Pt_K diag(1/s_K) and
  // Vt = PsiT_K (nearly orthonormal), L^s = Ut diag(s_K - tau) Vt^T, and
  // the FP64 Grams of Ut and Vt (distributed over the team) give either
  //   fast path (svd_fast_f64): second-order Löwdin orthonormalisation of
  //     Ut, Vt and a first-order (exponential-map) SVD of the nearly
  //     diagonal core, O(nk^2) FP64 work plus FP32 products of
  //     perturbation matrices; taken when the bases are orthonormal to
  //     1e-4 and the singular values are well separated; or
  //   exact path: Ut = Qu Ru, Vt = Qv Rv (Cholesky QR), C = Ru diag(s_K -
  //     tau) Rv^T, one-sided Jacobi C Wv = Wu diag(sigma), U^s = Ut Ru^-1
  //     Wu, V^s = Vt Rv^-1 Wv.
  // Either way U^s Sigma^s V^sT is the iterate's L^s (to ~1e-12 relative,
  // FP64 rounding on the exact path) and U^s, V^s are orthonormal to FP64
  // rounding.  rank = #{sigma > rank_cut sigma_1}, capped at r_cap.
  __shared__ double f_is[kSeedKmaxLimit];   // 1 / s_K
  __shared__ double f_sig[kSeedKmaxLimit];  // sigma_K (scaled), then sigma
  __shared__ double f_y[2][kSeedKmaxLimit]; // reciprocal pivots of Ru, Rv
  __shared__ int f_sel[kSeedKmaxLimit];     // K
  __shared__ int f_ord[kSeedKmaxLimit];     // output order (decreasing sigma)
  __shared__ int f_n[3];                    // nk, rank, rank before the cap
  __shared__ double f_p2;                   // power-of-two scale of C
  if (tid == 0) {
    int nk = 0;
    double smx = 0.0;
    for (int c = 0; c < k; ++c)
      if (lam[c] > tau) {
        f_sel[nk++] = c;
        smx = fmax(smx, lam[c] - tau);
      }
    f_n[0] = nk;
    int e = 0;
    frexp(smx, &e);
    f_p2 = nk > 0 ? ldexp(1.0, -e) : 1.0;
  }
  __syncthreads();
  const int nk = f_n[0];
  for (int q = tid; q < nk; q += kSeedThreads) {
    const double sq = lam[f_sel[q]];
    f_is[q] = 1.0 / sq;
    f_sig[q] = (sq - tau) * f_p2;
  }
  __syncthreads();
  // Grams of Ut and Vt (distributed over the team, fixed summation order)
  gram_sel(Ptc, mp, kmax, f_sel, f_is, nk, a.Gam, b, nb);
  gram_sel(PsiTc, np, kmax, f_sel, nullptr, nk, a.Gam2, b, nb);
  if (!team_sync()) return;
  // every CTA: the same nk x nk factorisations on the same data (identical
  // results), in the dynamic shared memory the iteration is done with
  double* D0 = sm;
  double* D1 = D0 + nk * nk;
  double* D2 = D1 + nk * nk;
  double* D3 = D2 + nk * nk;
  double* D4 = D3 + nk * nk;
  __shared__ double f_d[kSeedKmaxLimit];
  int far = 0;
  for (int idx = tid; idx < nk * nk; idx += kSeedThreads) {
    const int p = idx / nk, q = idx - p * nk;
    const double id = p == q ? 1.0 : 0.0;
    D0[idx] = ldg_cg(a.Gam + p * kmax + q) - id;
    D1[idx] = ldg_cg(a.Gam2 + p * kmax + q) - id;
    if (!(fabs(D0[idx]) <= 1e-4 && fabs(D1[idx]) <= 1e-4)) far = 1;
  }
  // the fast form needs 5 nk^2 doubles of shared memory, the exact one 4
  bool fast = !__syncthreads_or(far) && 5 * nk * nk <= a.smem_doubles;
  if (fast) fast = svd_fast_f64(D0, D1, D2, D3, D4, nk, f_sig, f_d);
  double* Mu = D0;  // diag(1/s_K) Ru^-1 Wu (exact) or X_u W_u (fast)
  double* Mv = D1;
  int fsweeps = 0;
  if (fast) {
    for (int q = tid; q < nk; q += kSeedThreads) f_sig[q] = f_d[q];
  } else {
    // exact path: Cholesky QR and a one-sided Jacobi SVD of the core
    double* Ru = D0;
    double* Rv = D1;
    double* Cm = D2;
    double* Wv = D3;
    for (int idx = tid; idx < nk * nk; idx += kSeedThreads) {
      const int p = idx / nk, q = idx - p * nk;
      Ru[idx] = ldg_cg(a.Gam + p * kmax + q);
      Rv[idx] = ldg_cg(a.Gam2 + p * kmax + q);
    }
    __syncthreads();
    chol2_f64(Ru, Rv, nk, f_y[0], f_y[1]);
    for (int idx = tid; idx < nk * nk; idx += kSeedThreads) {
      const int p = idx / nk, q = idx - p * nk;
      double acc = 0.0;
      for (int c = max(p, q); c < nk; ++c)
        acc = fma(Ru[p * nk + c] * f_sig[c], Rv[q * nk + c], acc);
      Cm[idx] = acc;
    }
    __syncthreads();
    fsweeps = hestenes_f64(Cm, Wv, nk);
    // sigma_q = ||C e_q||, Wu = C diag(1/sigma)
    for (int q = tid; q < nk; q += kSeedThreads) {
      double ss = 0.0;
      for (int p = 0; p < nk; ++p) ss = fma(Cm[p * nk + q], Cm[p * nk + q], ss);
      f_sig[q] = sqrt(ss);
    }
    __syncthreads();
    for (int idx = tid; idx < nk * nk; idx += kSeedThreads) {
      const int q = idx - (idx / nk) * nk;
      Cm[idx] = f_sig[q] > 0.0 ? Cm[idx] / f_sig[q] : 0.0;
    }
    __syncthreads();
    // Ru^-1 Wu (in Cm), Rv^-1 Wv (in Wv)
    backsub2_f64(Ru, Rv, Cm, Wv, nk, f_y[0], f_y[1]);
    Mu = Cm;
    Mv = Wv;
  }
  // U = Pt_K diag(1/s_K) M_u: fold 1/s_K into the rows of M_u
  for (int idx = tid; idx < nk * nk; idx += kSeedThreads)
    Mu[idx] *= f_is[idx / nk];
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < nk; ++q) f_ord[q] = q;
    for (int x = 1; x < nk; ++x) {  // insertion sort, decreasing sigma
      const int v = f_ord[x];
      int y = x - 1;
      while (y >= 0 && f_sig[f_ord[y]] < f_sig[v]) {
        f_ord[y + 1] = f_ord[y];
        --y;
      }
      f_ord[y + 1] = v;
    }
    int cnt = 0;
    const double top = nk > 0 ? f_sig[f_ord[0]] : 0.0;
    for (int q = 0; q < nk; ++q) {
      const double sv = f_sig[f_ord[q]];
      if (sv > 0.0 && sv > a.rank_cut * top) ++cnt;
    }
    f_n[2] = cnt;
    f_n[1] = a.r_cap > 0 ? min(cnt, a.r_cap) : cnt;
  }
  __syncthreads();
  const int rank = f_n[1];
  // U^s = Pt_K M_u and V^s = PsiT_K M_v row by row: one warp per row loads
  // the row's nk entries at once (two per lane), then every lane forms its
  // output columns (c = lane, lane + 32) from shuffles, summing over q in
  // order
  {
    const int lane = tid & 31, wid = tid >> 5;
    constexpr int kW = kSeedThreads / 32;
    const int c0 = lane, c1 = lane + 32;
    const int oc0 = c0 < rank ? f_ord[c0] : 0;
    const int oc1 = c1 < rank ? f_ord[c1] : 0;
    for (int t = b * kW + wid; t < mp + np; t += nb * kW) {
      const bool isu = t < mp;
      const int i = isu ? t : t - mp;
      const double* pr = (isu ? Ptc : PsiTc) + (size_t)i * kmax;
      const double* Mx = isu ? Mu : Mv;
      const double v0 = lane < nk ? ldg_cg(pr + f_sel[lane]) : 0.0;
      const double v1 = lane + 32 < nk ? ldg_cg(pr + f_sel[lane + 32]) : 0.0;
      double o0 = 0.0, o1 = 0.0;
      for (int q = 0; q < nk; ++q) {
        const double vq = __shfl_sync(0xffffffffu, q < 32 ? v0 : v1, q & 31);
        o0 = fma(vq, Mx[q * nk + oc0], o0);
        o1 = fma(vq, Mx[q * nk + oc1], o1);
      }
      double* out = isu ? a.U + i : a.V + i;
      const size_t ld = isu ? (size_t)mp : (size_t)np;
      if (c0 < kmax) out[(size_t)c0 * ld] = c0 < rank ? o0 : 0.0;
      if (c1 < kmax) out[(size_t)c1 * ld] = c1 < rank ? o1 : 0.0;
    }
  }
  trace_mark(a, 15);
  if (b == 0) {
    for (int c = tid; c < kmax; c += kSeedThreads)
      a.Sigma[c] = (c < rank) ? f_sig[f_ord[c]] / f_p2 : 0.0;
    if (tid == 0) {
      ctl->iters = it;
      ctl->rank = rank;
      ctl->rank_raw = f_n[2];
      ctl->fin_sweeps = fast ? -1 : fsweeps;
      ctl->converged = converged ? 1 : 0;
      ctl->residual = res;
      ctl->k_final = k;
    }
    if (tid == 0 && a.trace) {
      // closing records: Jacobi cycle split (phases 95..98) and total
      // Jacobi sweeps (phase 99)
      for (int q = 0; q < 5; ++q) {
        const int i = ctl->ntrace;
        if (i < kSeedTraceCap) {
          a.trace[2 * i] = q < 4 ? (unsigned long long)ctl->jcyc[q]
                                 : (unsigned long long)ctl->jsweeps;
          a.trace[2 * i + 1] = 95ull + q;
          ctl->ntrace = i + 1;
        }
      }
      {  // final SVD: phase 91, value 0 = fast path, else 1 + Jacobi sweeps
        const int i = ctl->ntrace;
        if (i < kSeedTraceCap) {
          a.trace[2 * i] = (unsigned long long)(fast ? 0 : 1 + fsweeps);
          a.trace[2 * i + 1] = 91ull;
          ctl->ntrace = i + 1;
        }
      }
      for (int q = 0; q < 3; ++q) {  // Rayleigh-Ritz forms, phases 88..90
        const int i = ctl->ntrace;
        if (i < kSeedTraceCap) {
          a.trace[2 * i] = (unsigned long long)ctl->jpath[q];
          a.trace[2 * i + 1] = 88ull + q;
          ctl->ntrace = i + 1;
        }
      }
      for (int q = 0; q < 8; ++q) {  // sub-step counters, phases 80..87
        const int i = ctl->ntrace;
        if (i < kSeedTraceCap) {
          a.trace[2 * i] = (unsigned long long)ctl->sub[q];
          a.trace[2 * i + 1] = 80ull + q;
          ctl->ntrace = i + 1;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kSeedThreads, 2)
    seed_alm_kernel(const SeedArgs a) {
  seed_alm_body<kTeamGrid>(a, blockIdx.x, gridDim.x);
}

// The same solve on one thread-block cluster (the whole grid is a single
// cluster of up to kSeedClusterMax CTAs): phases separated by the hardware
// cluster barrier instead of the software grid barrier.
__global__ void __launch_bounds__(kSeedThreads, 1)
    seed_alm_cluster_kernel(const SeedArgs a) {
  seed_alm_body<kTeamCluster>(a, blockIdx.x, gridDim.x);
}

// Batched form: CTA x belongs to the team of seed team[x].x, at position
// team[x].y of team[x].z CTAs.  A team of one CTA separates its phases with
// __syncthreads; a larger team uses the grid barrier on its own seed's
// control block (the launch is cooperative, so every team is co-resident).
__global__ void __launch_bounds__(kSeedThreads, 2)
    seed_alm_team_kernel(const SeedArgs* __restrict__ args,
                         const int4* __restrict__ team,
                         int* __restrict__ lists) {
  const int4 t = team[blockIdx.x];
  if (t.z == 1) {
    // the CTAs without a team take seeds one at a time, each alone, from
    // one queue in decreasing order of predicted cost (lists[0]: the next
    // entry, lists[1]: the length, then the seeds): a seed that runs longer
    // than predicted holds one CTA while the others take the rest
    __shared__ int s_q;
    for (int round = 0;; ++round) {
      if (round > 0) __syncthreads();  // the previous seed is done
      if (threadIdx.x == 0) s_q = atomicAdd(lists, 1);
      __syncthreads();
      const int q = s_q;
      if (q >= lists[1]) break;
      seed_alm_body<kTeamCta>(args[lists[2 + q]], 0, 1);
    }
  } else {
    seed_alm_body<kTeamGrid>(args[t.x], t.y, t.z);
  }
}

// Control blocks start at zero (barrier counters included) before any team
// member runs; so does the list queue's next-entry counter.
__global__ void seed_ctl_zero_kernel(const SeedArgs* __restrict__ args,
                                     int count, int* queue) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *queue = 0;
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    int* c = reinterpret_cast<int*>(args[i].ctl);
    for (int w = threadIdx.x; w < (int)(sizeof(SeedCtl) / 4); w += blockDim.x)
      c[w] = 0;
  }
}

size_t seed_smem_bytes(int kmax) {
  const size_t iter = sizeof(double) * ((size_t)kmax * kmax + kSeedThreads +
                                        kSeedGemmGroup *
                                            (kSeedMaxSide + kSeedThreads) +
                                        4 * kmax) +
                      sizeof(float) * ((size_t)3 * kmax * kmax) +
                      sizeof(int) * 2 * kmax + (size_t)kmax * kmax;
  // the final FP64 SVD: Ru, Rv, C, Wv (nk x nk each, nk <= kmax)
  const size_t fin = sizeof(double) * 4 * (size_t)kmax * kmax;
  return std::max(iter, fin);
}

}  // namespace

// Enqueue the seed solve; results stay on the device (ctl, U, Sigma, V).
namespace {
void fill_seed_args(SeedArgs& a, const SeedLayout& L, char* w,
                    const double* dD, int mp, int np, double lam, double tol,
                    double rho, double mu_scale, double mu_max_ratio,
                    int max_iter, int k0, int kmax, double rank_cut,
                    int r_cap, double* dU, double* dSigma, double* dV,
                    bool trace, unsigned long long timeout_ns) {
  a.D = dD;
  a.mp = mp;
  a.np = np;
  a.kmax = kmax;
  a.k0 = k0;
  a.lam = lam;
  a.tol = tol;
  a.rho = rho;
  a.mu_scale = mu_scale;
  a.mu_max_ratio = mu_max_ratio;
  a.rank_cut = rank_cut;
  a.max_iter = max_iter;
  a.r_cap = r_cap;
  a.timeout_ns = timeout_ns > 0 ? timeout_ns : kSeedDefaultWaitNs;
  a.lowp_res = kSeedLowpRes;
  a.nv = seed_slots(mp, np, kSeedTeamMax);
  a.ctl = reinterpret_cast<SeedCtl*>(w + L.ctl);
  a.part = reinterpret_cast<double*>(w + L.part);
  a.colsq = reinterpret_cast<double*>(w + L.colsq);
  a.S = reinterpret_cast<double*>(w + L.S);
  a.Y = reinterpret_cast<double*>(w + L.Y);
  a.G = reinterpret_cast<double*>(w + L.G);
  a.Gt = reinterpret_cast<double*>(w + L.Gt);
  a.Om = reinterpret_cast<double*>(w + L.Om);
  a.P = reinterpret_cast<double*>(w + L.P);
  a.Pt = reinterpret_cast<double*>(w + L.Pt);
  a.T = reinterpret_cast<double*>(w + L.T);
  a.Psi = reinterpret_cast<double*>(w + L.Psi);
  a.Om32 = reinterpret_cast<float*>(w + L.Om32);
  a.Psi32 = reinterpret_cast<float*>(w + L.Psi32);
  a.PsiT = reinterpret_cast<double*>(w + L.PsiT);
  a.Gam = reinterpret_cast<double*>(w + L.Gam);
  a.Gam2 = reinterpret_cast<double*>(w + L.Gam2);
  a.trace =
      trace ? reinterpret_cast<unsigned long long*>(w + L.trace) : nullptr;
  a.U = dU;
  a.Sigma = dSigma;
  a.V = dV;
}
}  // namespace

static_assert(sizeof(SeedArgs) % 16 == 0, "SeedArgs stride");
size_t seed_args_bytes() { return sizeof(SeedArgs); }

size_t seed_batched_args_bytes(int count) {
  return seed_args_bytes() * (size_t)count +
         sizeof(int4) * ((size_t)count + kMaxCoopBlocks) +
         sizeof(int) * ((size_t)count + 2);
}

SeedCtl* seed_ctl_ptr_cta(void* d_work, int mp, int np, int kmax) {
  const SeedLayout L = seed_layout(mp, np, kmax, kSeedTeamMax);
  return reinterpret_cast<SeedCtl*>(static_cast<char*>(d_work) + L.ctl);
}

int* seed_rank_ptr_cta(void* d_work, int mp, int np, int kmax) {
  const SeedLayout L = seed_layout(mp, np, kmax, kSeedTeamMax);
  return &reinterpret_cast<SeedCtl*>(static_cast<char*>(d_work) + L.ctl)->rank;
}

pcp_status seed_pcp_batched_async(const SeedTask* tasks, int count,
                                  void* h_args, void* d_args,
                                  cudaStream_t st, bool upload, bool launch) {
  if (count <= 0) return PCP_OK;
  char* hb = static_cast<char*>(h_args);
  int kmax_all = 2;
  for (int i = 0; i < count; ++i) {
    const SeedTask& t = tasks[i];
    const SeedLayout L = seed_layout(t.mp, t.np, t.kmax, kSeedTeamMax);
    char* w = static_cast<char*>(t.work);
    SeedArgs a;
    fill_seed_args(a, L, w, t.D, t.mp, t.np, t.lam, t.tol, t.rho, t.mu_scale,
                   t.mu_max_ratio, t.max_iter, t.k0, t.kmax, t.rank_cut,
                   t.r_cap, t.U, t.Sigma, t.V, false, t.timeout_ns);
    std::memcpy(hb + (size_t)i * seed_args_bytes(), &a, sizeof(a));
    kmax_all = std::max(kmax_all, t.kmax);
  }
  const size_t smem = seed_smem_bytes(kmax_all);
  for (int i = 0; i < count; ++i)
    reinterpret_cast<SeedArgs*>(hb + (size_t)i * seed_args_bytes())
        ->smem_doubles = (int)(smem / sizeof(double));
  PCP_CUDA(cudaFuncSetAttribute(seed_alm_team_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  PCP_CUDA(cudaGetDevice(&dev));
  PCP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PCP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  PCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, seed_alm_team_kernel, kSeedThreads, smem));
  const int slots = std::min(per_sm * sms, kMaxCoopBlocks);
  // Schedule (host, deterministic).  Cost of one ALM pass on one CTA,
  // fitted on GB300 to single-seed runs (60 x 60 .. 300 x 300 seeds, one
  // CTA: 0.38 .. 3.7 ms per pass): c(w) = 300 + 0.076 w^0.72 us with
  // w = m' n' k; a team of nb CTAs (grid barrier) runs about nb^0.87 times
  // faster (measured 1.9 / 3.6 / 6.6 / 11.1 at 2 / 4 / 8 / 16 CTAs on the
  // 300 x 300 seed).  With a cooperative launch of `slots` CTAs: seeds whose
  // one-CTA cost is above a target T get the smallest team that brings
  // them under T (at most kSeedTeamMax CTAs, and a quarter of the shorter
  // side), and the other seeds are packed, largest first, onto the
  // remaining CTAs as lists (the packing sizes the number of list CTAs; on
  // the device those CTAs share one queue of the list seeds); T is taken
  // from a geometric grid between the balanced load and the largest seed,
  // minimising the longest CTA.  A seed's result does not depend on its
  // team or CTA (fixed reduction slots), so the schedule changes no bits.
  const int n = count;
  std::vector<double> c1(n);
  std::vector<int> cap(n);
  double csum = 0.0, cmax = 0.0;
  for (int i = 0; i < n; ++i) {
    const double w = (double)tasks[i].mp * tasks[i].np * tasks[i].k0;
    c1[i] = 300.0 + 0.076 * std::pow(w, 0.72);
    // a quarter of the shorter side, or more when the batch leaves CTAs
    // idle: a small seed's phases are latency bound, and each CTA of a
    // larger team takes fewer of the rows, entries and tasks in turn
    // (one 20 x 20 seed: 1.79 ms on 5 CTAs, 1.31 ms on the 152-CTA grid)
    cap[i] = std::max(1, std::min(kSeedTeamMax,
                                  std::max(std::min(tasks[i].mp, tasks[i].np) / 4,
                                           slots / std::max(1, count))));
    csum += c1[i];
    cmax = std::max(cmax, c1[i]);
  }
  constexpr double kTeamExp = 0.87;
  std::vector<int> by_c(n);
  for (int i = 0; i < n; ++i) by_c[i] = i;
  std::stable_sort(by_c.begin(), by_c.end(),
                   [&](int x, int y) { return c1[x] > c1[y]; });
  std::vector<int> nb(n, 1), bin(n, -1);
  int nlist = 0;  // CTAs that run lists
  auto plan_for = [&](double T, std::vector<int>& nbv, std::vector<int>& binv,
                      int& nl) -> double {
    int used = 0;
    double worst = 0.0;
    for (int i : by_c) {
      nbv[i] = 1;
      if (c1[i] > T && cap[i] > 1) {
        const int want =
            (int)std::ceil(std::pow(c1[i] / T, 1.0 / kTeamExp) - 1e-9);
        nbv[i] = std::min(cap[i], std::max(2, want));
        used += nbv[i];
        worst = std::max(worst, c1[i] / std::pow((double)nbv[i], kTeamExp));
      }
    }
    nl = slots - used;
    if (nl < 1) return 1e300;
    // LPT over the list CTAs (a min-heap of loads)
    using Bin = std::pair<double, int>;
    std::priority_queue<Bin, std::vector<Bin>, std::greater<Bin>> heap;
    for (int b = 0; b < nl; ++b) heap.push({0.0, b});
    for (int i : by_c) {
      if (nbv[i] > 1) continue;
      Bin top = heap.top();
      heap.pop();
      binv[i] = top.second;
      top.first += c1[i];
      worst = std::max(worst, top.first);
      heap.push(top);
    }
    return worst;
  };
  if (coop && slots >= 1) {
    double best = 1e301;
    std::vector<int> nbv(n), binv(n);
    const double lo = std::max(1.0, 0.5 * csum / slots);
    const double hi = std::max(lo, cmax);
    for (int g = 0; g <= 40; ++g) {
      const double T = lo * std::pow(hi / lo, g / 40.0);
      int nl = 0;
      const double m = plan_for(T, nbv, binv, nl);
      if (m < best) {
        best = m;
        nb = nbv;
        bin = binv;
        nlist = nl;
      }
    }
  }
  const bool coop_launch = coop && nlist >= 1;
  if (!coop_launch) {
    // no cooperative launch: one CTA per seed, largest first, scheduled
    // by the hardware as CTAs finish
    std::fill(nb.begin(), nb.end(), 1);
    for (int q = 0; q < n; ++q) bin[by_c[q]] = q;
    nlist = n;
  }
  // block table after the argument blocks: team CTAs {seed, rank, size, 0},
  // then one entry {0, 0, 1, 0} per list CTA; the list queue follows the
  // table: the next-entry counter (zeroed before each launch), the number
  // of list seeds, and the list seeds, largest predicted cost first.  The
  // plan above sizes the lists; on the device the list CTAs share them.
  int4* tab = reinterpret_cast<int4*>(hb + seed_args_bytes() * (size_t)count);
  int nblocks = 0;
  for (int i : by_c)
    if (nb[i] > 1)
      for (int b = 0; b < nb[i]; ++b) tab[nblocks++] = make_int4(i, b, nb[i], 0);
  std::vector<std::vector<int>> lists(nlist);
  for (int i : by_c)
    if (nb[i] == 1) lists[bin[i]].push_back(i);
  // only lists that hold a seed get a CTA: a small group (one served
  // request) then occupies only the CTAs it uses, and the cooperative
  // launch of another stream's group can be resident beside it
  int nused = 0;
  for (const auto& l : lists) nused += !l.empty();
  int* lst = reinterpret_cast<int*>(tab + nblocks + nused);
  int off = 0;
  for (int b = 0; b < nused; ++b) tab[nblocks++] = make_int4(0, 0, 1, 0);
  lst[0] = 0;
  for (int i : by_c)
    if (nb[i] == 1) lst[2 + off++] = i;
  lst[1] = off;
  const size_t used_bytes = seed_args_bytes() * (size_t)count +
                            sizeof(int4) * (size_t)nblocks +
                            sizeof(int) * (size_t)(off + 2);
  if (used_bytes > seed_batched_args_bytes(count)) {
    set_error("batched seed: schedule of %d CTAs does not fit its block",
              nblocks);
    return PCP_ERR_ARG;
  }
  if (upload)
    PCP_CUDA(cudaMemcpyAsync(d_args, h_args, used_bytes,
                             cudaMemcpyHostToDevice, st));
  if (!launch) return PCP_OK;
  const SeedArgs* d_a = static_cast<const SeedArgs*>(d_args);
  const int4* d_tab = reinterpret_cast<const int4*>(
      static_cast<char*>(d_args) + seed_args_bytes() * (size_t)count);
  int* d_lst = const_cast<int*>(reinterpret_cast<const int*>(d_tab + nblocks));
  seed_ctl_zero_kernel<<<std::min(count, 1024), 64, 0, st>>>(d_a, count,
                                                              d_lst);
  PCP_CUDA(cudaGetLastError());
  if (coop_launch) {
    void* kargs[] = {(void*)&d_a, (void*)&d_tab, (void*)&d_lst};
    PCP_CUDA(cudaLaunchCooperativeKernel((void*)seed_alm_team_kernel,
                                         dim3(nblocks), dim3(kSeedThreads),
                                         kargs, smem, st));
  } else {
    seed_alm_team_kernel<<<nblocks, kSeedThreads, smem, st>>>(d_a, d_tab,
                                                               d_lst);
    PCP_CUDA(cudaGetLastError());
  }
  return PCP_OK;
}

// Launch the solve as one cluster of nc CTAs.  PCP_ERR_UNSUPPORTED (nothing
// launched) when the device cannot schedule such a cluster.
static pcp_status seed_cluster_launch(const SeedArgs& a, int nc, size_t smem,
                                      cudaStream_t st) {
  PCP_CUDA(cudaFuncSetAttribute(seed_alm_cluster_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  if (nc > 8)
    PCP_CUDA(cudaFuncSetAttribute(
        seed_alm_cluster_kernel,
        cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kSeedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int fit = 0;
  if (cudaOccupancyMaxActiveClusters(&fit, seed_alm_cluster_kernel, &cfg) !=
          cudaSuccess ||
      fit < 1) {
    cudaGetLastError();
    return PCP_ERR_UNSUPPORTED;
  }
  PCP_CUDA(cudaLaunchKernelEx(&cfg, seed_alm_cluster_kernel, a));
  return PCP_OK;
}

pcp_status seed_pcp_async(const double* dD, int mp, int np, double lam,
                          double tol, double rho, double mu_scale,
                          double mu_max_ratio, int max_iter, int k0, int kmax,
                          double rank_cut, int r_cap, void* d_work,
                          double* dU, double* dSigma, double* dV,
                          cudaStream_t st, int** d_rank_out, int ctas,
                          unsigned long long timeout_ns, int* launches,
                          int* team_out) {
  const SeedLayout L = seed_layout(mp, np, kmax, kMaxCoopBlocks);
  char* w = static_cast<char*>(d_work);
  SeedArgs a;
  fill_seed_args(a, L, w, dD, mp, np, lam, tol, rho, mu_scale, mu_max_ratio,
                 max_iter, k0, kmax, rank_cut, r_cap, dU, dSigma, dV, true,
                 timeout_ns);
  if (d_rank_out) *d_rank_out = &a.ctl->rank;

  const size_t smem = seed_smem_bytes(kmax);
  a.smem_doubles = (int)(smem / sizeof(double));
  PCP_CUDA(cudaFuncSetAttribute(seed_alm_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  PCP_CUDA(cudaGetDevice(&dev));
  PCP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PCP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) {
    set_error("seed PCP: device lacks cooperative launch");
    return PCP_ERR_UNSUPPORTED;
  }
  PCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, seed_alm_kernel, kSeedThreads, smem));
  if (per_sm < 1) {
    set_error("seed PCP: kernel does not fit on an SM (smem %zu)", smem);
    return PCP_ERR_UNSUPPORTED;
  }
  a.nv = seed_slots(mp, np, kSeedGridSlots);
  PCP_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(SeedCtl), st));
  // The library's choice for a seed of at most 64 rows and columns is one
  // cluster of 16 CTAs: its phases are barrier-latency bound, and the
  // hardware cluster barrier beats the grid's (20 x 20: 1.38 against 1.50
  // ms on its grid of 20 CTAs, 30 x 30: 1.92 / 2.05, 50 x 50: 1.69 / 1.75,
  // 60 x 60: 1.56 / 1.58); larger seeds need the FP64 pipes of every SM.
  if (ctas == 0 && std::max(mp, np) <= 64) ctas = kSeedClusterMax;
  // One thread-block cluster of `ctas` CTAs (1 .. kSeedClusterMax) when
  // asked for and the device can hold it; the same slots, so the same bits.
  if (ctas >= 1 && ctas <= kSeedClusterMax) {
    pcp_status cs = seed_cluster_launch(a, ctas, smem, st);
    if (cs == PCP_OK) {
      if (launches) ++*launches;
      if (team_out) *team_out = ctas;
      return PCP_OK;
    }
    if (cs != PCP_ERR_UNSUPPORTED) return cs;
    ctas = 0;  // no room for the cluster: the grid form below
  }
  // One CTA per SM, or one per column/row task (max(m', n')) when there are
  // fewer: a sweep on the 200 x 200 seed measured 3.58 ms at 152 CTAs
  // against 3.92 ms at 200 (48 SMs doubled up) and 3.9 ms at 304, and the
  // 500 x 500 seed 11.0 ms at 152 against 11.1 ms at 304; with the current
  // phases, 2.60 ms at 152 against 2.66-2.73 ms at 76-144 (200 x 200) and
  // 7.24 ms against 7.58-9.55 ms (500 x 500).  `ctas` > 0 asks
  // for that many instead (within the co-resident limit of a cooperative
  // launch).  The partial-sum slots are fixed (kSeedGridSlots), so the
  // result does not depend on the grid size.
  const int cap = std::min(sms * per_sm, kMaxCoopBlocks);
  const int grid = ctas > 0 ? std::min(ctas, cap)
                            : std::min(std::min(cap, sms), std::max(mp, np));
  void* args[] = {&a};
  PCP_CUDA(cudaLaunchCooperativeKernel((const void*)seed_alm_kernel, grid,
                                       kSeedThreads, args, smem, st));
  if (launches) ++*launches;
  if (team_out) *team_out = -grid;
  return PCP_OK;
}

pcp_status seed_read_ctl(void* d_work, int mp, int np, int kmax,
                         cudaStream_t st, int* rank, int* iters,
                         double* residual, int* converged, int* error,
                         int* rank_raw) {
  const SeedLayout L = seed_layout(mp, np, kmax, kMaxCoopBlocks);
  SeedCtl h;
  PCP_CUDA(cudaMemcpyAsync(&h, static_cast<char*>(d_work) + L.ctl,
                           sizeof(SeedCtl), cudaMemcpyDeviceToHost, st));
  PCP_CUDA(cudaStreamSynchronize(st));
  if (rank) *rank = h.rank;
  if (iters) *iters = h.iters;
  if (residual) *residual = h.residual;
  if (converged) *converged = h.converged;
  if (error) *error = h.error;
  if (rank_raw) *rank_raw = h.rank_raw;
  return PCP_OK;
}

}  // namespace pcp

extern "C" size_t pcp_seed_workspace_bytes(int32_t mp, int32_t np,
                                           int32_t kmax) {
  if (mp < 1 || np < 1 || kmax < 2) return 0;
  return pcp::seed_workspace_bytes(mp, np, kmax);
}

extern "C" pcp_status pcp_seed_pcp(const double* dD, int32_t mp, int32_t np,
                                   double lambda, double tol, double rho,
                                   double mu_scale, double mu_max_ratio,
                                   int32_t max_iter, int32_t k0, int32_t kmax,
                                   double rank_cut, int32_t r_cap, void* d_work,
                                   double* dU, double* dSigma, double* dV,
                                   int32_t* h_rank, int32_t* h_iters,
                                   double* h_residual, void* stream) {
  PCP_ARG(mp >= 2 && np >= 2 && mp <= pcp::kSeedMaxSide &&
              np <= pcp::kSeedMaxSide,
          "pcp_seed_pcp: seed %dx%d outside [2, %d]", mp, np,
          pcp::kSeedMaxSide);
  // a subspace wider than the short side would hold a direction the seed
  // does not have: its Cholesky pivot is FP32 rounding noise, not zero, and
  // the noise column breaks the bases' orthogonality
  PCP_ARG(kmax >= 2 && kmax <= pcp::kSeedKmaxLimit && kmax % 2 == 0 &&
              kmax <= std::min(mp, np),
          "pcp_seed_pcp: kmax=%d must be even, <= %d and <= min(mp,np)", kmax,
          pcp::kSeedKmaxLimit);
  PCP_ARG(k0 >= 2 && k0 % 2 == 0 && k0 <= kmax,
          "pcp_seed_pcp: k0=%d must be even and in [2, kmax]", k0);
  PCP_ARG(tol > 0 && rho > 1 && mu_scale > 0 && mu_max_ratio >= 1 &&
              max_iter >= 1 && rank_cut >= 0,
          "pcp_seed_pcp: bad tolerances");
  PCP_ARG(dD && d_work && dU && dSigma && dV, "pcp_seed_pcp: null pointer");
  if (!(lambda > 0)) lambda = 1.0 / std::sqrt((double)std::max(mp, np));
  cudaStream_t st = (cudaStream_t)stream;
  pcp_status s = pcp::seed_pcp_async(dD, mp, np, lambda, tol, rho, mu_scale,
                                     mu_max_ratio, max_iter, k0, kmax,
                                     rank_cut, r_cap, d_work, dU, dSigma, dV,
                                     st, nullptr, 0, 0, nullptr, nullptr);
  if (s != PCP_OK) return s;
  int rank = 0, iters = 0, conv = 0, err = 0;
  double resid = 0;
  s = pcp::seed_read_ctl(d_work, mp, np, kmax, st, &rank, &iters, &resid,
                         &conv, &err, nullptr);
  if (s != PCP_OK) return s;
  if (h_rank) *h_rank = rank;
  if (h_iters) *h_iters = iters;
  if (h_residual) *h_residual = resid;
  if (err) {
    pcp::set_error("pcp_seed_pcp: device barrier wait timed out");
    return PCP_ERR_TIMEOUT;
  }
  if (!conv) {
    pcp::set_error("pcp_seed_pcp: no convergence in %d iterations", iters);
    return PCP_ERR_SEED_NOCONV;
  }
  return PCP_OK;
}

extern "C" int32_t pcp_seed_trace(const void* d_work, int32_t mp, int32_t np,
                                  int32_t kmax, uint64_t* h_out, int32_t cap,
                                  void* stream) {
  if (!d_work || mp < 1 || np < 1 || kmax < 2 || cap < 0) return -1;
  const pcp::SeedLayout L = pcp::seed_layout(mp, np, kmax, pcp::kMaxCoopBlocks);
  const char* w = static_cast<const char*>(d_work);
  pcp::SeedCtl h;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, w + L.ctl, sizeof(h), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -1;
  const int n = std::min(std::min(h.ntrace, pcp::kSeedTraceCap), cap);
  if (n > 0 && h_out) {
    if (cudaMemcpyAsync(h_out, w + L.trace, sizeof(uint64_t) * 2 * n,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return -1;
  }
  return n;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of pcp_seed_pcp.
//
// Some callers cannot call cudaMalloc: host frameworks that hand out every
// byte of device memory from their own pool and do not let extensions
// allocate, latency-bound loops where cudaMalloc's implicit device
// synchronisation would stall other streams, and processes whose device
// memory budget is committed up front.  For them the seed workspace lives
// in a fixed file-scope device array instead of a caller buffer.  Its host
// symbol is only a stand-in: the device address is looked up once per
// device with cudaGetSymbolAddress (on that device's first call) and passed
// to the kernel.  Every GPU that loads the library holds the array until the
// process exits.
namespace pcp {
namespace {

constexpr size_t kSeedStaticScratchBytes = (size_t)3 << 20;  // 3 MiB
constexpr int kMaxScratchDevices = 64;

static __device__ __align__(256) unsigned char
    g_seed_static_scratch[kSeedStaticScratchBytes];

std::mutex g_seed_scratch_mu;
void* g_seed_scratch_addr[kMaxScratchDevices] = {};

// Device address of the static scratch on the current device (set up on
// the first call per device, under a lock).
pcp_status seed_static_scratch(void** out) {
  int dev = 0;
  PCP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxScratchDevices) {
    set_error("pcp_seed_pcp_static: device ordinal %d >= %d", dev,
              kMaxScratchDevices);
    return PCP_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_seed_scratch_mu);
  if (!g_seed_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_seed_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                       "cudaGetSymbolAddress(seed scratch)", __FILE__,
                       __LINE__);
    g_seed_scratch_addr[dev] = p;
  }
  *out = g_seed_scratch_addr[dev];
  return PCP_OK;
}

}  // namespace
}  // namespace pcp

extern "C" pcp_status pcp_seed_pcp_static(
    const double* dD, int32_t mp, int32_t np, double lambda, double tol,
    double rho, double mu_scale, double mu_max_ratio, int32_t max_iter,
    int32_t k0, int32_t kmax, double rank_cut, int32_t r_cap, double* dU,
    double* dSigma, double* dV, int32_t* h_rank, int32_t* h_iters,
    double* h_residual, void* stream) {
  PCP_ARG(mp >= 2 && np >= 2 && kmax >= 2,
          "pcp_seed_pcp_static: seed %dx%d, kmax=%d too small", mp, np, kmax);
  const size_t need = pcp::seed_workspace_bytes(mp, np, kmax);
  PCP_ARG(need <= pcp::kSeedStaticScratchBytes,
          "pcp_seed_pcp_static: a %dx%d seed with kmax=%d needs %zu bytes of "
          "scratch, more than the fixed %zu",
          mp, np, kmax, need, pcp::kSeedStaticScratchBytes);
  void* w = nullptr;
  const pcp_status s = pcp::seed_static_scratch(&w);
  if (s != PCP_OK) return s;
  return pcp_seed_pcp(dD, mp, np, lambda, tol, rho, mu_scale, mu_max_ratio,
                      max_iter, k0, kmax, rank_cut, r_cap, w, dU, dSigma, dV,
                      h_rank, h_iters, h_residual, stream);
}
