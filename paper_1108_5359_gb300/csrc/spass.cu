// Streaming stages of Algorithm 2: the seed gather (Eq. partition), the
// factor assembly of the generalized Nystrom representation (Eq. l1s'), and
// the S pass S = M - L with L = Lu Lv^T (Algorithm 2 output).
//
// S pass on GB300: HBM bound for r up to ~40 (8 bytes moved per entry, 2r
// flops).  A CTA owns a 128 x 64 tile of M; each thread owns 4 consecutive
// rows (one float4 per column) of 8 columns.  All eight float4 loads of M are
// issued before the rank-r products (memory-level parallelism), Lu / Lv
// tiles sit in shared memory laid out k-major so a thread reads its 4 Lu
// entries as one float4 and the warp-shared 8 Lv entries as two broadcast
// float4 per k.  M is read with an evict-first (streaming) hint and S is
// written with a streaming store so neither pollutes L2.
#include <algorithm>

#include "common.cuh"

namespace pcp {
namespace {

constexpr int kTileM = 128;   // rows per CTA (32 lanes x 4)
constexpr int kTileN = 64;    // columns per CTA (8 warps x 8)
constexpr int kColsPerWarp = 8;
constexpr int kSpassThreads = 256;
constexpr int kSpassMaxR = 64;

__global__ void __launch_bounds__(kSpassThreads)
    spass_kernel(const float* __restrict__ M, int64_t ldm,
                 const float* __restrict__ Lu, int64_t ldu,
                 const float* __restrict__ Lv, int64_t ldv, int r,
                 float* __restrict__ S, int64_t lds, int64_t m, int64_t n,
                 int vec_ok) {
  extern __shared__ __align__(16) float sp_smem[];
  float* su = sp_smem;                 // [k][row], r x kTileM
  float* sv = sp_smem + r * kTileM;    // [k][col], r x kTileN
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kTileM;
  const int64_t j0 = (int64_t)blockIdx.y * kTileN;

  // Stage the Lu and Lv tiles (coalesced along rows of each column).
  for (int idx = threadIdx.x; idx < r * kTileM; idx += kSpassThreads) {
    const int k = idx / kTileM, ii = idx - k * kTileM;
    const int64_t i = i0 + ii;
    su[idx] = (i < m) ? __ldg(Lu + i + (int64_t)k * ldu) : 0.0f;
  }
  for (int idx = threadIdx.x; idx < r * kTileN; idx += kSpassThreads) {
    const int k = idx / kTileN, jj = idx - k * kTileN;
    const int64_t jc = j0 + jj;
    sv[idx] = (jc < n) ? __ldg(Lv + jc + (int64_t)k * ldv) : 0.0f;
  }

  const int64_t ib = i0 + 4 * lane;             // first of my 4 rows
  const int cb = w * kColsPerWarp;              // first of my 8 columns
  const bool full_rows = vec_ok && (ib + 3 < m);

  // Issue the loads of M early.
  float4 mv[kColsPerWarp];
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) {
    const int64_t jc = j0 + cb + c;
    if (jc < n && full_rows) {
      mv[c] = __ldcs(reinterpret_cast<const float4*>(M + ib + jc * ldm));
    } else {
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      if (jc < n)
        for (int q = 0; q < 4; ++q)
          if (ib + q < m) t[q] = __ldcs(M + ib + q + jc * ldm);
      mv[c] = make_float4(t[0], t[1], t[2], t[3]);
    }
  }
  __syncthreads();

  float acc[kColsPerWarp][4];
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[c][q] = 0.0f;

#pragma unroll 4
  for (int k = 0; k < r; ++k) {
    const float4 u = *reinterpret_cast<const float4*>(su + k * kTileM + 4 * lane);
    const float4 va = *reinterpret_cast<const float4*>(sv + k * kTileN + cb);
    const float4 vb =
        *reinterpret_cast<const float4*>(sv + k * kTileN + cb + 4);
    const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
    const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int c = 0; c < kColsPerWarp; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[c][q] = fmaf(uu[q], vv[c], acc[c][q]);
  }

#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) {
    const int64_t jc = j0 + cb + c;
    if (jc >= n) continue;
    const float4 o = make_float4(mv[c].x - acc[c][0], mv[c].y - acc[c][1],
                                 mv[c].z - acc[c][2], mv[c].w - acc[c][3]);
    if (full_rows) {
      __stcs(reinterpret_cast<float4*>(S + ib + jc * lds), o);
    } else {
      const float t[4] = {o.x, o.y, o.z, o.w};
      for (int q = 0; q < 4; ++q)
        if (ib + q < m) __stcs(S + ib + q + jc * lds, t[q]);
    }
  }
}

// M^s = M[I_s, J_s] in FP64; counts non-finite entries into *bad.
__global__ void gather_seed_kernel(const float* __restrict__ M, int64_t ldm,
                                   const int32_t* __restrict__ rows, int mp,
                                   const int32_t* __restrict__ cols, int np,
                                   double* __restrict__ Ms,
                                   int32_t* __restrict__ bad) {
  const int64_t total = (int64_t)mp * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / mp), i = (int)(e - (int64_t)j * mp);
    const float v = __ldg(M + rows[i] + (int64_t)cols[j] * ldm);
    if (bad && !isfinite(v)) atomicAdd(bad, 1);
    Ms[e] = (double)v;
  }
}

// Factor assembly (Eq. l1s'): seed rows of Lu / Lv, FP32 copies of U^s and
// V^s for the filters, and 1/sigma for the row-filter output scale.
__global__ void assemble_kernel(const double* __restrict__ U,
                                const double* __restrict__ sigma,
                                const double* __restrict__ V, int mp, int np,
                                const int32_t* __restrict__ d_rank, int r,
                                const int32_t* __restrict__ rows,
                                const int32_t* __restrict__ cols,
                                float* __restrict__ Lu, int64_t ldu,
                                float* __restrict__ Lv, int64_t ldv,
                                float* __restrict__ U32,
                                float* __restrict__ V32,
                                float* __restrict__ inv_sigma32) {
  const int rank = min(max(*d_rank, 0), r);
  const int64_t nu = (int64_t)mp * r, nv = (int64_t)np * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       e < nu + nv + r; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nu) {
      const int k = (int)(e / mp), i = (int)(e - (int64_t)k * mp);
      const float u = (k < rank) ? (float)U[i + (int64_t)k * mp] : 0.0f;
      U32[e] = u;
      if (Lu) Lu[rows[i] + k * ldu] = u;
    } else if (e < nu + nv) {
      const int64_t f = e - nu;
      const int k = (int)(f / np), j = (int)(f - (int64_t)k * np);
      const double v = (k < rank) ? V[j + (int64_t)k * np] : 0.0;
      V32[f] = (float)v;
      if (Lv) Lv[cols[j] + k * ldv] = (k < rank) ? (float)(v * sigma[k]) : 0.0f;
    } else {
      const int k = (int)(e - nu - nv);
      inv_sigma32[k] = (k < rank) ? (float)(1.0 / sigma[k]) : 0.0f;
    }
  }
}

}  // namespace
}  // namespace pcp

extern "C" pcp_status pcp_spass(const float* dM, int64_t ldm, const float* dLu,
                                int64_t ldu, const float* dLv, int64_t ldv,
                                int32_t r, float* dS, int64_t lds, int64_t m,
                                int64_t n, void* stream) {
  PCP_ARG(m >= 0 && n >= 0, "pcp_spass: negative size");
  PCP_ARG(r >= 0 && r <= pcp::kSpassMaxR, "pcp_spass: r=%d outside [0, %d]",
          r, pcp::kSpassMaxR);
  if (m == 0 || n == 0) return PCP_OK;
  PCP_ARG(ldm >= m && lds >= m && ldu >= m && ldv >= n,
          "pcp_spass: leading dimension too small");
  PCP_ARG(dM && dS && (r == 0 || (dLu && dLv)), "pcp_spass: null pointer");
  PCP_ARG((m + pcp::kTileM - 1) / pcp::kTileM < (1LL << 31) &&
              (n + pcp::kTileN - 1) / pcp::kTileN < 65536,
          "pcp_spass: matrix too large for one launch");
  const int vec_ok = ((((uintptr_t)dM) | ((uintptr_t)dS)) % 16 == 0) &&
                     (ldm % 4 == 0) && (lds % 4 == 0);
  dim3 grid((unsigned)((m + pcp::kTileM - 1) / pcp::kTileM),
            (unsigned)((n + pcp::kTileN - 1) / pcp::kTileN));
  const size_t smem = sizeof(float) * (size_t)r * (pcp::kTileM + pcp::kTileN);
  if (smem > 48 * 1024) {
    PCP_CUDA(cudaFuncSetAttribute(pcp::spass_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  }
  pcp::spass_kernel<<<grid, pcp::kSpassThreads, smem, (cudaStream_t)stream>>>(
      dM, ldm, dLu, ldu, dLv, ldv, r, dS, lds, m, n, vec_ok);
  PCP_CUDA(cudaGetLastError());
  return PCP_OK;
}

namespace pcp {
pcp_status gather_seed(const float* dM, int64_t ldm, const int32_t* d_rows,
                       int32_t mp, const int32_t* d_cols, int32_t np,
                       double* dMs, int32_t* d_bad, cudaStream_t st) {
  const int64_t total = (int64_t)mp * np;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  gather_seed_kernel<<<blocks, 256, 0, st>>>(dM, ldm, d_rows, mp, d_cols, np,
                                             dMs, d_bad);
  PCP_CUDA(cudaGetLastError());
  return PCP_OK;
}
}  // namespace pcp

extern "C" pcp_status pcp_gather_seed(const float* dM, int64_t ldm,
                                      const int32_t* d_rows, int32_t mp,
                                      const int32_t* d_cols, int32_t np,
                                      double* dMs, void* stream) {
  PCP_ARG(mp >= 1 && np >= 1, "pcp_gather_seed: empty seed");
  PCP_ARG(dM && d_rows && d_cols && dMs, "pcp_gather_seed: null pointer");
  return pcp::gather_seed(dM, ldm, d_rows, mp, d_cols, np, dMs, nullptr,
                          (cudaStream_t)stream);
}

extern "C" pcp_status pcp_assemble_factors(
    const double* dU, const double* dSigma, const double* dV, int32_t mp,
    int32_t np, int32_t ku, const int32_t* d_rank, int32_t r,
    const int32_t* d_rows, const int32_t* d_cols, float* dLu, int64_t ldu,
    float* dLv, int64_t ldv, float* dU32, float* dV32, float* d_inv_sigma32,
    void* stream) {
  PCP_ARG(mp >= 1 && np >= 1 && r >= 1 && ku >= r,
          "pcp_assemble_factors: bad sizes (mp=%d np=%d r=%d ku=%d)", mp, np,
          r, ku);
  PCP_ARG(dU && dSigma && dV && d_rank && d_rows && d_cols && dU32 && dV32 &&
              d_inv_sigma32,
          "pcp_assemble_factors: null pointer");
  const int64_t total = (int64_t)(mp + np) * r + r;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  pcp::assemble_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
      dU, dSigma, dV, mp, np, d_rank, r, d_rows, d_cols, dLu, ldu, dLv, ldv,
      dU32, dV32, d_inv_sigma32);
  PCP_CUDA(cudaGetLastError());
  return PCP_OK;
}
