// Streaming stages of Algorithm 2: the seed gather (Eq. partition), the
// factor assembly of the generalized Nystrom representation (Eq. l1s'), and
// the S pass S = M - L with L = Lu Lv^T (Algorithm 2 output).
//
// S pass on GB300: HBM bound for r up to ~40 (8 bytes moved per entry, 2r
// flops).  Persistent grid (a few CTAs per SM) walking a contiguous range of
// 128 x 32 tiles, row block major so consecutive tiles share their Lu tile.
// Each thread owns 4 consecutive rows (one float4 per column) of 4 columns;
// the next tile's four float4 loads of M are issued before the current
// tile's rank-r products, so loads stay in flight while the CTA computes.
// Lu / Lv tiles sit in shared memory laid out k-major (a thread reads its 4
// Lu entries as one float4 and the warp-shared 4 Lv entries as one broadcast
// float4 per k); the Lv tile is double-buffered.  M is read with an
// evict-first (streaming) hint and S written with a streaming store.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.cuh"

namespace pcp {
namespace {

constexpr int kSpassThreads = 256;
constexpr int kSpassMaxR = 64;

constexpr int kPTileM = 128;  // rows per tile (32 lanes x 4)
constexpr int kPTileN = 32;   // columns per tile (8 warps x 4)
constexpr int kPCols = 4;     // columns per thread

struct SpassArgs {
  const float* M;
  int64_t ldm;
  const float* Lu;
  int64_t ldu;
  const float* Lv;
  int64_t ldv;
  int r;
  float* S;
  int64_t lds;
  int64_t m, n;
  int vec_ok;
  int64_t ntm, ntn, ntiles;
};

__device__ __forceinline__ void spass_load_m(const SpassArgs& a, int64_t t,
                                             float4 (&mv)[kPCols]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t ti = t / a.ntn, tj = t - ti * a.ntn;
  const int64_t ib = ti * kPTileM + 4 * lane;
  const bool full = a.vec_ok && (ib + 3 < a.m);
#pragma unroll
  for (int c = 0; c < kPCols; ++c) {
    const int64_t jc = tj * kPTileN + w * kPCols + c;
    if (jc < a.n && full) {
      mv[c] = __ldcs(reinterpret_cast<const float4*>(a.M + ib + jc * a.ldm));
    } else {
      float q4[4] = {0.f, 0.f, 0.f, 0.f};
      if (jc < a.n)
        for (int q = 0; q < 4; ++q)
          if (ib + q < a.m) q4[q] = __ldcs(a.M + ib + q + jc * a.ldm);
      mv[c] = make_float4(q4[0], q4[1], q4[2], q4[3]);
    }
  }
}

__device__ __forceinline__ void spass_load_lu(const SpassArgs& a, int64_t ti,
                                              float* su) {
  const int64_t i0 = ti * kPTileM;
  for (int idx = threadIdx.x; idx < a.r * kPTileM; idx += kSpassThreads) {
    const int k = idx >> 7, ii = idx & (kPTileM - 1);
    const int64_t i = i0 + ii;
    su[idx] = (i < a.m) ? __ldg(a.Lu + i + (int64_t)k * a.ldu) : 0.0f;
  }
}

__device__ __forceinline__ void spass_load_lv(const SpassArgs& a, int64_t tj,
                                              float* sv) {
  const int64_t j0 = tj * kPTileN;
  for (int idx = threadIdx.x; idx < a.r * kPTileN; idx += kSpassThreads) {
    const int k = idx >> 5, jj = idx & (kPTileN - 1);
    const int64_t jc = j0 + jj;
    sv[idx] = (jc < a.n) ? __ldg(a.Lv + jc + (int64_t)k * a.ldv) : 0.0f;
  }
}

__global__ void __launch_bounds__(kSpassThreads, 3)
    spass_kernel(const SpassArgs a) {
  extern __shared__ __align__(16) float sp_smem[];
  float* su = sp_smem;                        // r x 128, k-major
  float* sv0 = su + a.r * kPTileM;            // r x 32, k-major, x2
  const int svstride = a.r * kPTileN;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int64_t per = (a.ntiles + gridDim.x - 1) / gridDim.x;
  int64_t t = (int64_t)blockIdx.x * per;
  const int64_t tend = min(a.ntiles, t + per);
  if (t >= tend) return;

  float4 nxt[kPCols];
  spass_load_m(a, t, nxt);
  int64_t ti_cur = t / a.ntn;
  spass_load_lu(a, ti_cur, su);
  spass_load_lv(a, t - ti_cur * a.ntn, sv0);
  __syncthreads();
  int buf = 0;
  for (; t < tend; ++t) {
    float4 mv[kPCols];
#pragma unroll
    for (int c = 0; c < kPCols; ++c) mv[c] = nxt[c];
    const bool more = t + 1 < tend;
    int64_t ti_next = ti_cur;
    if (more) {
      spass_load_m(a, t + 1, nxt);  // in flight during this tile's math
      ti_next = (t + 1) / a.ntn;
      spass_load_lv(a, (t + 1) - ti_next * a.ntn, sv0 + (buf ^ 1) * svstride);
    }
    const float* sv = sv0 + buf * svstride;
    float acc[kPCols][4];
#pragma unroll
    for (int c = 0; c < kPCols; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[c][q] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < a.r; ++k) {
      const float4 u =
          *reinterpret_cast<const float4*>(su + k * kPTileM + 4 * lane);
      const float4 v =
          *reinterpret_cast<const float4*>(sv + k * kPTileN + w * kPCols);
      const float vv[4] = {v.x, v.y, v.z, v.w};
      const float uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int c = 0; c < kPCols; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[c][q] = fmaf(uu[q], vv[c], acc[c][q]);
    }
    {
      const int64_t ti = ti_cur, tj = t - ti_cur * a.ntn;
      const int64_t ib = ti * kPTileM + 4 * lane;
      const bool full = a.vec_ok && (ib + 3 < a.m);
#pragma unroll
      for (int c = 0; c < kPCols; ++c) {
        const int64_t jc = tj * kPTileN + w * kPCols + c;
        if (jc >= a.n) continue;
        const float4 o = make_float4(mv[c].x - acc[c][0], mv[c].y - acc[c][1],
                                     mv[c].z - acc[c][2], mv[c].w - acc[c][3]);
        if (full) {
          __stcs(reinterpret_cast<float4*>(a.S + ib + jc * a.lds), o);
        } else {
          const float q4[4] = {o.x, o.y, o.z, o.w};
          for (int q = 0; q < 4; ++q)
            if (ib + q < a.m) __stcs(a.S + ib + q + jc * a.lds, q4[q]);
        }
      }
    }
    __syncthreads();  // every thread is done with su and this Lv buffer
    if (more && ti_next != ti_cur) {
      spass_load_lu(a, ti_next, su);
      ti_cur = ti_next;
    }
    __syncthreads();
    buf ^= 1;
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

// Batched forms: blockIdx.y selects the instance.
__global__ void gather_batched_kernel(const GatherTask* __restrict__ tasks) {
  const GatherTask t = tasks[blockIdx.y];
  const int64_t total = (int64_t)t.mp * t.np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / t.mp), i = (int)(e - (int64_t)j * t.mp);
    const float v = __ldg(t.M + t.rows[i] + (int64_t)t.cols[j] * t.ldm);
    if (t.bad && !isfinite(v)) atomicAdd(t.bad, 1);
    t.Ms[e] = (double)v;
  }
}

__global__ void assemble_batched_kernel(const AssembleTask* __restrict__ tasks) {
  const AssembleTask t = tasks[blockIdx.y];
  const int r = t.r;
  const int rank = min(max(*t.d_rank, 0), r);
  const int64_t nu = (int64_t)t.mp * r, nv = (int64_t)t.np * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       e < nu + nv + r; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nu) {
      const int k = (int)(e / t.mp), i = (int)(e - (int64_t)k * t.mp);
      const float u = (k < rank) ? (float)t.U[i + (int64_t)k * t.mp] : 0.0f;
      t.U32[e] = u;
      t.Lu[t.rows[i] + k * t.ldu] = u;
    } else if (e < nu + nv) {
      const int64_t f = e - nu;
      const int k = (int)(f / t.np), j = (int)(f - (int64_t)k * t.np);
      const double v = (k < rank) ? t.V[j + (int64_t)k * t.np] : 0.0;
      t.V32[f] = (float)v;
      t.Lv[t.cols[j] + k * t.ldv] = (k < rank) ? (float)(v * t.Sigma[k]) : 0.0f;
    } else {
      const int k = (int)(e - nu - nv);
      t.inv_sigma32[k] = (k < rank) ? (float)(1.0 / t.Sigma[k]) : 0.0f;
    }
  }
}

}  // namespace

pcp_status gather_batched_async(const GatherTask* tasks, int count,
                                void* h_buf, void* d_buf, cudaStream_t st,
                                bool upload, bool launch) {
  if (count <= 0) return PCP_OK;
  std::memcpy(h_buf, tasks, sizeof(GatherTask) * count);
  if (upload)
    PCP_CUDA(cudaMemcpyAsync(d_buf, h_buf, sizeof(GatherTask) * count,
                             cudaMemcpyHostToDevice, st));
  if (!launch) return PCP_OK;
  int64_t biggest = 1;
  for (int i = 0; i < count; ++i)
    biggest = std::max<int64_t>(biggest, (int64_t)tasks[i].mp * tasks[i].np);
  const int bx = (int)std::min<int64_t>((biggest + 255) / 256, 64);
  gather_batched_kernel<<<dim3(bx, count), 256, 0, st>>>(
      static_cast<const GatherTask*>(d_buf));
  PCP_CUDA(cudaGetLastError());
  return PCP_OK;
}

pcp_status assemble_batched_async(const AssembleTask* tasks, int count,
                                  void* h_buf, void* d_buf, cudaStream_t st,
                                  bool upload, bool launch) {
  if (count <= 0) return PCP_OK;
  std::memcpy(h_buf, tasks, sizeof(AssembleTask) * count);
  if (upload)
    PCP_CUDA(cudaMemcpyAsync(d_buf, h_buf, sizeof(AssembleTask) * count,
                             cudaMemcpyHostToDevice, st));
  if (!launch) return PCP_OK;
  int64_t biggest = 1;
  for (int i = 0; i < count; ++i)
    biggest = std::max<int64_t>(
        biggest, (int64_t)(tasks[i].mp + tasks[i].np + 1) * tasks[i].r);
  const int bx = (int)std::min<int64_t>((biggest + 255) / 256, 64);
  assemble_batched_kernel<<<dim3(bx, count), 256, 0, st>>>(
      static_cast<const AssembleTask*>(d_buf));
  PCP_CUDA(cudaGetLastError());
  return PCP_OK;
}

}  // namespace pcp

extern "C" pcp_status pcp_spass(const float* dM, int64_t ldm, const float* dLu,
                                int64_t ldu, const float* dLv, int64_t ldv,
                                int32_t r, float* dS, int64_t lds, int64_t m,
                                int64_t n, void* stream) {
  return pcp_spass_impl(dM, ldm, dLu, ldu, dLv, ldv, r, dS, lds, m, n,
                        PCP_SPASS_AUTO, stream);
}

extern "C" pcp_status pcp_spass_impl(const float* dM, int64_t ldm,
                                     const float* dLu, int64_t ldu,
                                     const float* dLv, int64_t ldv, int32_t r,
                                     float* dS, int64_t lds, int64_t m,
                                     int64_t n, int32_t impl, void* stream) {
  PCP_ARG(m >= 0 && n >= 0, "pcp_spass: negative size");
  PCP_ARG(r >= 0 && r <= pcp::kSpassMaxR, "pcp_spass: r=%d outside [0, %d]",
          r, pcp::kSpassMaxR);
  PCP_ARG(impl == PCP_SPASS_AUTO || impl == PCP_SPASS_SIMT ||
              impl == PCP_SPASS_TENSOR,
          "pcp_spass: unknown kernel choice %d", impl);
  if (m == 0 || n == 0) return PCP_OK;
  PCP_ARG(ldm >= m && lds >= m && ldu >= m && ldv >= n,
          "pcp_spass: leading dimension too small");
  PCP_ARG(dM && dS && (r == 0 || (dLu && dLv)), "pcp_spass: null pointer");
  if (impl != PCP_SPASS_SIMT) {
    if (pcp::spass_tc_fits(dM, ldm, dS, lds, r, m, n))
      return pcp::spass_tc_launch(dM, ldm, dLu, ldu, dLv, ldv, r, dS, lds, m,
                                  n, (cudaStream_t)stream);
    if (impl == PCP_SPASS_TENSOR) {
      pcp::set_error(
          "pcp_spass: tensor-core form needs 1 <= r <= 64, m >= 128, n >= 64 "
          "and 16-byte aligned M / S columns (r=%d m=%lld n=%lld)",
          r, (long long)m, (long long)n);
      return PCP_ERR_UNSUPPORTED;
    }
  }
  const int vec_ok = ((((uintptr_t)dM) | ((uintptr_t)dS)) % 16 == 0) &&
                     (ldm % 4 == 0) && (lds % 4 == 0);
  pcp::SpassArgs a;
  a.M = dM;
  a.ldm = ldm;
  a.Lu = dLu;
  a.ldu = ldu;
  a.Lv = dLv;
  a.ldv = ldv;
  a.r = r;
  a.S = dS;
  a.lds = lds;
  a.m = m;
  a.n = n;
  a.vec_ok = vec_ok;
  a.ntm = (m + pcp::kPTileM - 1) / pcp::kPTileM;
  a.ntn = (n + pcp::kPTileN - 1) / pcp::kPTileN;
  a.ntiles = a.ntm * a.ntn;
  const size_t smem =
      sizeof(float) * (size_t)r * (pcp::kPTileM + 2 * pcp::kPTileN);
  if (smem > 48 * 1024) {
    PCP_CUDA(cudaFuncSetAttribute(pcp::spass_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  }
  int per_sm = 0;
  PCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, pcp::spass_kernel, pcp::kSpassThreads, smem));
  const int64_t slots = (int64_t)std::max(per_sm, 1) * pcp::device_sm_count();
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.ntiles, slots));
  pcp::spass_kernel<<<grid, pcp::kSpassThreads, smem, (cudaStream_t)stream>>>(
      a);
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
