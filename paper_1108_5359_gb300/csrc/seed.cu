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
//   T = G^T Omega,  Psi = orth(T),  P = G Psi,  C = P^T P = Vb diag(s^2) Vb^T,
//   SVT(G Psi Psi^T) = (P Vb) diag(max(1 - tau/s, 0)) (Psi Vb)^T,
//   Omega_next = P Vb diag(1/s)  (the left Ritz vectors),
// where orth() is a column-normalised Cholesky QR.  The subspace size k
// starts at k0 and grows while every Ritz value exceeds tau.  At the exit
// the skinny SVD of L^s is read off directly: U^s = P Vb diag(1/s),
// Sigma^s = s - tau, V^s = Psi Vb (Section 3.2 uses exactly these factors).
//
// GB300 form: one cooperative persistent launch (grid = one CTA per SM) runs
// the whole ALM loop.  Phases are separated by a software grid barrier whose
// spin is bounded by %globaltimer (on expiry every CTA sets an error word and
// returns).  The m' x n' state (S, Y, G and G^T) stays in L2.  Small k x k
// factorisations (Cholesky, Jacobi eigen-solve) run redundantly in every CTA
// so that they need no barrier; their inputs and code are identical, so
// every CTA obtains bit-identical factors.  All cross-CTA data is read with
// L2-only loads (ld.global.cg) so no CTA sees a stale L1 line.
#include <algorithm>

#include "common.cuh"

namespace pcp {

constexpr int kSeedThreads = 256;
constexpr int kSeedKmaxLimit = 96;

struct SeedCtl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int error;
  int iters;
  int rank;
  int converged;
  int k_final;
  int rank_raw;
  double residual;
  double sigma1;
  double pad[4];
};

struct SeedLayout {
  size_t ctl, part, S, Y, G, Gt, Om, P, Pt, T, Psi, PsiT, Gam, total;
};

static SeedLayout seed_layout(int mp, int np, int kmax) {
  SeedLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t mn = (size_t)mp * np * sizeof(double);
  L.ctl = take(sizeof(SeedCtl));
  L.part = take((size_t)kMaxCoopBlocks * 4 * sizeof(double));
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
  L.total = off;
  return L;
}

size_t seed_workspace_bytes(int mp, int np, int kmax) {
  return seed_layout(mp, np, kmax).total;
}

namespace {

struct SeedArgs {
  const double* D;
  int mp, np, kmax, k0;
  double lam, tol, rho, mu_scale, mu_max_ratio, rank_cut;
  int max_iter, r_cap;
  unsigned long long timeout_ns;
  SeedCtl* ctl;
  double* part;
  double *S, *Y, *G, *Gt;
  double *Om, *P, *Pt;  // mp x kmax, row-major (row stride kmax)
  double *T, *Psi, *PsiT;  // np x kmax, row-major
  double* Gam;             // kmax x kmax
  double *U, *Sigma, *V;   // outputs (column-major, ld mp / np)
};

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

// Software grid barrier (sense by generation), bounded by a timeout.
__device__ bool grid_sync(SeedCtl* ctl, unsigned int nblocks,
                          unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* genp = &ctl->bar_gen;
    const unsigned int gen = *genp;
    __threadfence();
    const unsigned int arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      unsigned int spins = 0;
      while (*genp == gen) {
        if (*(volatile int*)&ctl->error) break;
        if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
          atomicExch(&ctl->error, (int)PCP_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = (*(volatile int*)&ctl->error) == 0;
  }
  __syncthreads();
  return s_ok != 0;
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

// out[task*kmax + c] = sum_t X[t + task*ldx] * B[t*kmax + c], c < k.
__device__ void tall_gemm_t(const double* X, int ldx, int len, int ntask,
                            const double* B, int k, int kmax, double* out,
                            double* red) {
  const int tid = threadIdx.x;
  const int nparts = kSeedThreads / k;
  const int c = tid % k, part = tid / k;
  for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
    const double* x = X + (size_t)task * ldx;
    double acc = 0.0;
    if (part < nparts) {
      for (int t = part; t < len; t += nparts)
        acc = fma(ldg_cg(x + t), ldg_cg(B + (size_t)t * kmax + c), acc);
      red[part * k + c] = acc;
    }
    __syncthreads();
    if (tid < k) {
      double s = 0.0;
      for (int q = 0; q < nparts; ++q) s += red[q * k + tid];
      __stcg(out + (size_t)task * kmax + tid, s);
    }
    __syncthreads();
  }
}

// Gm = X^T X (k x k) for X (nrows x k, row-major stride kmax); one warp per
// entry a <= b, both triangles written.
__device__ void gram(const double* X, int nrows, int k, int kmax,
                     double* Gm) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (kSeedThreads / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (kSeedThreads / 32);
  for (int pq = gw; pq < k * k; pq += nw) {
    const int a = pq / k, b = pq - a * k;
    if (a > b) continue;
    double s = 0.0;
    for (int t = lane; t < nrows; t += 32)
      s = fma(ldg_cg(X + (size_t)t * kmax + a), ldg_cg(X + (size_t)t * kmax + b),
              s);
    s = warp_sum(s);
    if (lane == 0) {
      __stcg(Gm + a * kmax + b, s);
      __stcg(Gm + b * kmax + a, s);
    }
  }
}

// Column-normalised Cholesky QR: Out = X diag(1/||x_a||) R^{-1} with
// R^T R = diag(1/||x_a||) X^T X diag(1/||x_a||).  Columns whose norm or
// pivot vanishes are dead and come out zero.  A, Ri: k x k shared buffers.
__device__ void cholqr_apply(const double* X, int nrows, int k, int kmax,
                             const double* Gm, double* Out, double* A,
                             double* Ri, double* dsc, int* dead) {
  const int tid = threadIdx.x;
  for (int c = tid; c < k; c += kSeedThreads) {
    const double g = ldg_cg(Gm + c * kmax + c);
    dead[c] = !(g > 0.0);
    dsc[c] = (g > 0.0) ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += kSeedThreads) {
    const int a = idx / k, b = idx - a * k;
    double v = ldg_cg(Gm + a * kmax + b) * dsc[a] * dsc[b];
    if (dead[a] || dead[b]) v = (a == b) ? 1.0 : 0.0;
    A[idx] = v;
    Ri[idx] = 0.0;
  }
  __syncthreads();
  // right-looking Cholesky, R stored in the upper triangle of A
  for (int j = 0; j < k; ++j) {
    __shared__ double s_piv;
    if (tid == 0) {
      double piv = A[j * k + j];
      if (!(piv > 1e-13) || dead[j]) {
        dead[j] = 1;
        piv = 1.0;
      } else {
        piv = sqrt(piv);
      }
      s_piv = piv;
    }
    __syncthreads();
    const double piv = s_piv;
    const bool dj = dead[j];
    for (int c = j + 1 + tid; c < k; c += kSeedThreads)
      A[j * k + c] = dj ? 0.0 : A[j * k + c] / piv;
    if (tid == 0) A[j * k + j] = piv;
    __syncthreads();
    const int rem = k - j - 1;
    for (int idx = tid; idx < rem * rem; idx += kSeedThreads) {
      const int a = j + 1 + idx / rem, b = j + 1 + idx % rem;
      if (a <= b) A[a * k + b] -= A[j * k + a] * A[j * k + b];
    }
    __syncthreads();
  }
  // Ri = R^{-1} (upper triangular), one column per thread
  for (int c = tid; c < k; c += kSeedThreads) {
    Ri[c * k + c] = 1.0 / A[c * k + c];
    for (int a = c - 1; a >= 0; --a) {
      double s = 0.0;
      for (int b = a + 1; b <= c; ++b) s = fma(A[a * k + b], Ri[b * k + c], s);
      Ri[a * k + c] = -s / A[a * k + a];
    }
  }
  __syncthreads();
  // rows of the output, distributed over the grid
  for (int t = blockIdx.x; t < nrows; t += gridDim.x) {
    for (int c = tid; c < k; c += kSeedThreads) {
      double s = 0.0;
      if (!dead[c])
        for (int a = 0; a <= c; ++a)
          s = fma(ldg_cg(X + (size_t)t * kmax + a) * dsc[a], Ri[a * k + c], s);
      __stcg(Out + (size_t)t * kmax + c, s);
    }
  }
}

// Cyclic Jacobi eigen-decomposition of the symmetric k x k matrix in A
// (k even), parallel (round-robin) ordering.  On return A's diagonal holds
// the eigenvalues and V the eigenvectors (columns).  Every CTA runs it on
// the same data and gets the same bits.
__device__ void block_jacobi(double* A, double* V, int k, double* cs,
                             int* prs) {
  const int tid = threadIdx.x;
  __shared__ int s_rot;
  __shared__ double s_thr;
  for (int idx = tid; idx < k * k; idx += kSeedThreads)
    V[idx] = (idx / k == idx % k) ? 1.0 : 0.0;
  if (tid == 0) {
    double dmax = 0.0;
    for (int i = 0; i < k; ++i) dmax = fmax(dmax, fabs(A[i * k + i]));
    s_thr = 1e-15 * dmax;
  }
  __syncthreads();
  const double thr = s_thr;
  const int half = k / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int round = 0; round < k - 1; ++round) {
      __syncthreads();
      if (tid < half) {
        auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + round) % (k - 1); };
        int p = pos(tid), q = pos(k - 1 - tid);
        if (p > q) { const int t = p; p = q; q = t; }
        const double apq = A[p * k + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > thr) {
          const double theta = (A[q * k + q] - A[p * k + p]) / (2.0 * apq);
          const double t = (theta >= 0.0 ? 1.0 : -1.0) /
                           (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
          s_rot = 1;
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
        prs[2 * tid] = p;
        prs[2 * tid + 1] = q;
      }
      __syncthreads();
      for (int idx = tid; idx < half * k; idx += kSeedThreads) {
        const int i = idx / k, x = idx - i * k;
        const double s = cs[2 * i + 1];
        if (s != 0.0) {
          const double c = cs[2 * i];
          const int p = prs[2 * i], q = prs[2 * i + 1];
          const double ap = A[p * k + x], aq = A[q * k + x];
          A[p * k + x] = c * ap - s * aq;
          A[q * k + x] = s * ap + c * aq;
        }
      }
      __syncthreads();
      for (int idx = tid; idx < half * k; idx += kSeedThreads) {
        const int i = idx / k, x = idx - i * k;
        const double s = cs[2 * i + 1];
        if (s != 0.0) {
          const double c = cs[2 * i];
          const int p = prs[2 * i], q = prs[2 * i + 1];
          const double ap = A[x * k + p], aq = A[x * k + q];
          A[x * k + p] = c * ap - s * aq;
          A[x * k + q] = s * ap + c * aq;
          const double vp = V[x * k + p], vq = V[x * k + q];
          V[x * k + p] = c * vp - s * vq;
          V[x * k + q] = s * vp + c * vq;
        }
      }
    }
    __syncthreads();
    if (s_rot == 0) break;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSeedThreads, 1)
    seed_alm_kernel(const SeedArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int kmax = a.kmax;
  double* A = sm;                       // kmax*kmax
  double* Vb = A + kmax * kmax;         // kmax*kmax
  double* red = Vb + kmax * kmax;       // kSeedThreads
  double* lam = red + kSeedThreads;     // kmax
  double* dsc = lam + kmax;             // kmax
  double* xi = dsc + kmax;              // kmax
  double* cs = xi + kmax;               // kmax (pairs of c,s)
  int* ibuf = reinterpret_cast<int*>(cs + kmax);  // 2*kmax ints
  int* dead = ibuf;
  int* prs = ibuf + kmax;
  __shared__ double s_scalar[8];

  const int tid = threadIdx.x;
  const int nb = gridDim.x, b = blockIdx.x;
  const int mp = a.mp, np = a.np;
  const size_t mn = (size_t)mp * np;
  SeedCtl* ctl = a.ctl;
  const unsigned long long tmo = a.timeout_ns;

  // ---- prologue: norms of D, G = D, random Omega ---------------------------
  {
    double ss = 0.0, mx = 0.0;
    for (size_t e = (size_t)b * kSeedThreads + tid; e < mn;
         e += (size_t)nb * kSeedThreads) {
      const double d = __ldg(a.D + e);
      ss = fma(d, d, ss);
      mx = fmax(mx, fabs(d));
      __stcg(a.S + e, 0.0);
      __stcg(a.G + e, d);
      const int j = (int)(e / mp), i = (int)(e - (size_t)j * mp);
      __stcg(a.Gt + (size_t)i * np + j, d);
    }
    ss = warp_sum(ss);
    mx = warp_max(mx);
    if ((tid & 31) == 0) {
      red[tid >> 5] = ss;
      red[8 + (tid >> 5)] = mx;
    }
    __syncthreads();
    if (tid == 0) {
      double s2 = 0.0, m2 = 0.0;
      for (int q = 0; q < kSeedThreads / 32; ++q) {
        s2 += red[q];
        m2 = fmax(m2, red[8 + q]);
      }
      __stcg(a.part + 4 * b, s2);
      __stcg(a.part + 4 * b + 1, m2);
    }
    for (size_t e = (size_t)b * kSeedThreads + tid; e < (size_t)mp * a.k0;
         e += (size_t)nb * kSeedThreads) {
      const int i = (int)(e / a.k0), c = (int)(e - (size_t)i * a.k0);
      __stcg(a.Om + (size_t)i * kmax + c, hash_normal(0x5EEDull + c, i));
    }
  }
  if (!grid_sync(ctl, nb, tmo)) return;
  if (tid == 0) {
    double s2 = 0.0, m2 = 0.0;
    for (int q = 0; q < nb; ++q) {
      s2 += ldg_cg(a.part + 4 * q);
      m2 = fmax(m2, ldg_cg(a.part + 4 * q + 1));
    }
    s_scalar[0] = sqrt(s2);
    s_scalar[1] = m2;
  }
  __syncthreads();
  const double normF = s_scalar[0];
  const double norminf = s_scalar[1];
  if (!(normF > 0.0)) {
    // D = 0: L = S = 0, rank 0.
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
  int stage = 0;        // 0,1: power steps on D; 2: Rayleigh-Ritz on D; 3: ALM
  bool converged = false;
  double res = 1.0;

  while (true) {
    // ---- T = G^T Omega ------------------------------------------------------
    tall_gemm_t(a.G, mp, mp, np, a.Om, k, kmax, a.T, red);
    if (!grid_sync(ctl, nb, tmo)) return;
    gram(a.T, np, k, kmax, a.Gam);
    if (!grid_sync(ctl, nb, tmo)) return;
    cholqr_apply(a.T, np, k, kmax, a.Gam, a.Psi, A, Vb, dsc, dead);
    if (!grid_sync(ctl, nb, tmo)) return;
    // ---- P = G Psi ------------------------------------------------------------
    tall_gemm_t(a.Gt, np, np, mp, a.Psi, k, kmax, a.P, red);
    if (!grid_sync(ctl, nb, tmo)) return;
    gram(a.P, mp, k, kmax, a.Gam);
    if (!grid_sync(ctl, nb, tmo)) return;
    if (stage < 2) {
      // plain power step on D: Omega = orth(P)
      cholqr_apply(a.P, mp, k, kmax, a.Gam, a.Om, A, Vb, dsc, dead);
      if (!grid_sync(ctl, nb, tmo)) return;
      ++stage;
      continue;
    }
    // ---- Rayleigh-Ritz: C = P^T P = Vb diag(lam) Vb^T -----------------------
    for (int idx = tid; idx < k * k; idx += kSeedThreads) {
      const int p = idx / k, q = idx - p * k;
      A[idx] = ldg_cg(a.Gam + p * kmax + q);
    }
    __syncthreads();
    block_jacobi(A, Vb, k, cs, prs);
    __syncthreads();
    double smax = 0.0;
    for (int c = 0; c < k; ++c) smax = fmax(smax, sqrt(fmax(A[c * k + c], 0.0)));
    if (stage == 2) {
      // ||D||_2 from the Ritz values; start the ALM.
      mu = a.mu_scale / smax;
      mu_max = mu * a.mu_max_ratio;
      if (b == 0 && tid == 0) ctl->sigma1 = smax;
    }
    tau = 1.0 / mu;
    int nsv = 0;
    for (int c = tid; c < k; c += kSeedThreads) {
      const double s = sqrt(fmax(A[c * k + c], 0.0));
      lam[c] = s;
      dsc[c] = (s > tau) ? 1.0 - tau / s : 0.0;  // shrink factor d_c
    }
    __syncthreads();
    for (int c = 0; c < k; ++c) nsv += (lam[c] > tau);
    // ---- rotate: Pt = P Vb, Omega_next = Pt / s, PsiT = Psi Vb --------------
    int knext = k;
    if (stage == 3 && nsv >= k && k < kmax)
      knext = min(kmax, (k + max(6, k / 4) + 1) / 2 * 2);
    for (int i = b; i < mp; i += nb) {
      for (int c = tid; c < knext; c += kSeedThreads) {
        if (c < k) {
          double s = 0.0;
          for (int q = 0; q < k; ++q)
            s = fma(ldg_cg(a.P + (size_t)i * kmax + q), Vb[q * k + c], s);
          __stcg(a.Pt + (size_t)i * kmax + c, s);
          const double sc = lam[c];
          __stcg(a.Om + (size_t)i * kmax + c,
                 (sc > 1e-12 * smax) ? s / sc
                                     : hash_normal(0xA11CEull + 977ull * it + c, i));
        } else {
          __stcg(a.Om + (size_t)i * kmax + c,
                 hash_normal(0xB0B0ull + 977ull * it + c, i));
        }
      }
    }
    for (int j = b; j < np; j += nb) {
      for (int c = tid; c < k; c += kSeedThreads) {
        double s = 0.0;
        for (int q = 0; q < k; ++q)
          s = fma(ldg_cg(a.Psi + (size_t)j * kmax + q), Vb[q * k + c], s);
        __stcg(a.PsiT + (size_t)j * kmax + c, s);
      }
    }
    if (!grid_sync(ctl, nb, tmo)) return;

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
      if (!grid_sync(ctl, nb, tmo)) return;
      continue;
    }

    // ---- ALM step: L = Pt diag(d) PsiT^T, S, Y, G for the next iteration ---
    const double mu_next = fmin(a.rho * mu, mu_max);
    const double lam_mu = a.lam / mu;
    double zz = 0.0;
    for (int j = b; j < np; j += nb) {
      for (int c = tid; c < k; c += kSeedThreads)
        xi[c] = dsc[c] * ldg_cg(a.PsiT + (size_t)j * kmax + c);
      __syncthreads();
      for (int i = tid; i < mp; i += kSeedThreads) {
        double l = 0.0;
        for (int c = 0; c < k; ++c)
          l = fma(ldg_cg(a.Pt + (size_t)i * kmax + c), xi[c], l);
        const size_t e = (size_t)j * mp + i;
        const double d = __ldg(a.D + e);
        const double y = ldg_cg(a.Y + e);
        const double s = shrink(d - l + y / mu, lam_mu);
        const double z = d - l - s;
        const double yn = fma(mu, z, y);
        zz = fma(z, z, zz);
        __stcg(a.S + e, s);
        __stcg(a.Y + e, yn);
        const double g = d - s + yn / mu_next;
        __stcg(a.G + e, g);
        __stcg(a.Gt + (size_t)i * np + j, g);
      }
      __syncthreads();
    }
    zz = warp_sum(zz);
    if ((tid & 31) == 0) red[tid >> 5] = zz;
    __syncthreads();
    if (tid == 0) {
      double s2 = 0.0;
      for (int q = 0; q < kSeedThreads / 32; ++q) s2 += red[q];
      __stcg(a.part + 4 * b + 2, s2);
    }
    ++it;
    if (!grid_sync(ctl, nb, tmo)) return;
    if (tid == 0) {
      double s2 = 0.0;
      for (int q = 0; q < nb; ++q) s2 += ldg_cg(a.part + 4 * q + 2);
      s_scalar[2] = sqrt(s2) / normF;
    }
    __syncthreads();
    res = s_scalar[2];
    converged = res <= a.tol;
    if (converged || it >= a.max_iter) break;
    mu = mu_next;
    k = knext;
  }

  // ---- outputs: skinny SVD of L^s sorted by decreasing singular value -------
  // this iteration's factors: U = Omega_next (= Pt / s), Sigma = s - tau,
  // V = PsiT; rank = #{s - tau > rank_cut * max(s - tau)}, capped at r_cap.
  if (tid == 0) {
    int* order = prs;
    int cnt = 0;
    for (int c = 0; c < k; ++c) order[c] = c;
    // insertion sort by decreasing s (k <= 96)
    for (int x = 1; x < k; ++x) {
      const int v = order[x];
      int y = x - 1;
      while (y >= 0 && lam[order[y]] < lam[v]) {
        order[y + 1] = order[y];
        --y;
      }
      order[y + 1] = v;
    }
    const double top = lam[order[0]] - tau;
    for (int c = 0; c < k; ++c) {
      const double sv = lam[order[c]] - tau;
      if (sv > 0.0 && sv > a.rank_cut * top) ++cnt;
    }
    dead[1] = cnt;
    if (a.r_cap > 0) cnt = min(cnt, a.r_cap);
    dead[0] = cnt;
  }
  __syncthreads();
  const int rank = dead[0];
  const int* order = prs;
  for (int i = b; i < mp; i += nb)
    for (int c = tid; c < kmax; c += kSeedThreads)
      a.U[i + (size_t)c * mp] =
          (c < rank) ? ldg_cg(a.Om + (size_t)i * kmax + order[c]) : 0.0;
  for (int j = b; j < np; j += nb)
    for (int c = tid; c < kmax; c += kSeedThreads)
      a.V[j + (size_t)c * np] =
          (c < rank) ? ldg_cg(a.PsiT + (size_t)j * kmax + order[c]) : 0.0;
  if (b == 0) {
    for (int c = tid; c < kmax; c += kSeedThreads)
      a.Sigma[c] = (c < rank) ? lam[order[c]] - tau : 0.0;
    if (tid == 0) {
      ctl->iters = it;
      ctl->rank = rank;
      ctl->rank_raw = dead[1];
      ctl->converged = converged ? 1 : 0;
      ctl->residual = res;
      ctl->k_final = k;
    }
  }
}

size_t seed_smem_bytes(int kmax) {
  return sizeof(double) * ((size_t)2 * kmax * kmax + kSeedThreads + 4 * kmax) +
         sizeof(int) * 2 * kmax;
}

}  // namespace

// Enqueue the seed solve; results stay on the device (ctl, U, Sigma, V).
pcp_status seed_pcp_async(const double* dD, int mp, int np, double lam,
                          double tol, double rho, double mu_scale,
                          double mu_max_ratio, int max_iter, int k0, int kmax,
                          double rank_cut, int r_cap, void* d_work,
                          double* dU, double* dSigma, double* dV,
                          cudaStream_t st, int** d_rank_out) {
  const SeedLayout L = seed_layout(mp, np, kmax);
  char* w = static_cast<char*>(d_work);
  SeedArgs a;
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
  a.timeout_ns = 2000000000ull;  // 2 s per barrier wait
  a.ctl = reinterpret_cast<SeedCtl*>(w + L.ctl);
  a.part = reinterpret_cast<double*>(w + L.part);
  a.S = reinterpret_cast<double*>(w + L.S);
  a.Y = reinterpret_cast<double*>(w + L.Y);
  a.G = reinterpret_cast<double*>(w + L.G);
  a.Gt = reinterpret_cast<double*>(w + L.Gt);
  a.Om = reinterpret_cast<double*>(w + L.Om);
  a.P = reinterpret_cast<double*>(w + L.P);
  a.Pt = reinterpret_cast<double*>(w + L.Pt);
  a.T = reinterpret_cast<double*>(w + L.T);
  a.Psi = reinterpret_cast<double*>(w + L.Psi);
  a.PsiT = reinterpret_cast<double*>(w + L.PsiT);
  a.Gam = reinterpret_cast<double*>(w + L.Gam);
  a.U = dU;
  a.Sigma = dSigma;
  a.V = dV;
  if (d_rank_out) *d_rank_out = &a.ctl->rank;

  const size_t smem = seed_smem_bytes(kmax);
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
  const int grid = std::min(sms, kMaxCoopBlocks);
  PCP_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(SeedCtl), st));
  void* args[] = {&a};
  PCP_CUDA(cudaLaunchCooperativeKernel((const void*)seed_alm_kernel, grid,
                                       kSeedThreads, args, smem, st));
  return PCP_OK;
}

pcp_status seed_read_ctl(void* d_work, int mp, int np, int kmax,
                         cudaStream_t st, int* rank, int* iters,
                         double* residual, int* converged, int* error,
                         int* rank_raw) {
  const SeedLayout L = seed_layout(mp, np, kmax);
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
  PCP_ARG(mp >= 2 && np >= 2, "pcp_seed_pcp: seed %dx%d too small", mp, np);
  PCP_ARG(kmax >= 2 && kmax <= pcp::kSeedKmaxLimit && kmax % 2 == 0 &&
              kmax <= std::min(mp, np) + (std::min(mp, np) & 1),
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
                                     st, nullptr);
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
