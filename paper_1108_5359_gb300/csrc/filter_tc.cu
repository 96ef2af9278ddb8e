// l1 filtering (Section 3.2), tensor-core form of Algorithm 1.
//
// The same ADM steps as filter.cu (per problem: e = S_{1/beta}(x - A z +
// y/beta), z = A^T (x - e + y/beta), y += beta (x - A z - e), beta grows by
// rho up to beta_bar, stop when ||x - A z - e||_inf < eps max(||x - e||_inf,
// kStopNormFloor ||x||_inf)) in the same FP32 form (state d = x - e, so
// that no step subtracts two copies of an outlier), with the two products
// of every iteration on the tensor cores:
//
//   w^T (16 x p) = z^T (16 x r) A^T (r x p)     (A z for 16 problems)
//   z^T (16 x r) = u^T (16 x p) A (p x r)       (A^T u, u = x - e + y/beta)
//
// as mma.sync m16n8k8 TF32 with FP32 accumulation (problems are the M
// dimension).  The accumulator fragment of the first product holds, per
// thread, entries 2t and 2t+1 of problems g and g+8 (g = lane/4,
// t = lane%4); x, y, d live in registers in exactly that layout, so the
// elementwise ADM step needs no data movement, and the same four values
// are the A-operand fragment of the second product once its k index is
// permuted (k slot t <-> entry 2t, slot t+4 <-> entry 2t+1; the B operand
// rows are read with the same permutation).  z^T is reduced across the
// 8 warps (each owns a slab of entries) through shared memory in a fixed
// order and read back with the same permutation on the r index.
//
// Precision: one-pass low-precision products for the first lowp_iters
// iterations (TF32, 10-bit mantissa, or BF16, 7-bit mantissa, as
// mma.sync m16n8k8 bf16 whose A fragment holds the two entries 2t, 2t+1 of
// a row in one register: the same values as the TF32 fragment's slots t and
// t+4), then split products (a = hi + lo, three passes: lo*hi + hi*lo +
// hi*hi, ~2^-21 relative) until the stop test, which is only taken on
// split-product iterations.  lowp_iters = 0 gives the FP32-accurate form
// throughout.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace pcp {

namespace {

constexpr int kTcWarps = 8;
constexpr int kTcThreads = kTcWarps * 32;
constexpr int kTcProblems = 16;

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi,
                                           uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t a0,
                                         const uint32_t a1, const uint32_t a2,
                                         const uint32_t a3, const uint32_t b0,
                                         const uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// two FP32 values rounded to BF16 in one register, lo in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t a01,
                                         const uint32_t a23,
                                         const uint32_t b01) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a01), "r"(a23), "r"(b01));
}

// Product modes: one-pass TF32, split TF32 (FP32-accurate), one-pass BF16.
enum { kOneTf32 = 0, kSplitTf32 = 1, kOneBf16 = 2 };

// d += a * b with a, b given as FP32 values (a in the TF32 fragment's slot
// order): one low-precision pass into d, or the three passes of the split
// operands, hi*hi into d and the two cross terms into dl (a second
// accumulator, so the dependent chains are half as long; the caller adds
// dl into d at the end).
template <int kMode>
__device__ __forceinline__ void mma_f32(float (&d)[4], float (&dl)[4],
                                        const float (&a)[4], const float b0,
                                        const float b1) {
  if (kMode == kOneBf16) {
    mma_bf16(d, pack_bf16(a[0], a[2]), pack_bf16(a[1], a[3]),
             pack_bf16(b0, b1));
  } else if (kMode == kSplitTf32) {
    uint32_t ah[4], al[4], bh0, bl0, bh1, bl1;
#pragma unroll
    for (int q = 0; q < 4; ++q) split_tf32(a[q], ah[q], al[q]);
    split_tf32(b0, bh0, bl0);
    split_tf32(b1, bh1, bl1);
    mma_tf32(dl, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(dl, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
  } else {
    mma_tf32(d, tf32_rna(a[0]), tf32_rna(a[1]), tf32_rna(a[2]),
             tf32_rna(a[3]), tf32_rna(b0), tf32_rna(b1));
  }
}

// An A-operand fragment prepared once and used for several products: the
// TF32 value (one-pass) or its hi / lo split.
struct TcFrag {
  uint32_t h[4], l[4];
};

template <int kMode>
__device__ __forceinline__ void tc_prep(TcFrag& f, const float (&a)[4]) {
  if (kMode == kOneBf16) {
    f.h[0] = pack_bf16(a[0], a[2]);
    f.h[1] = pack_bf16(a[1], a[3]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (kMode == kSplitTf32)
        split_tf32(a[q], f.h[q], f.l[q]);
      else
        f.h[q] = tf32_rna(a[q]);
    }
  }
}

// d (+ dl) += a * b for a prepared fragment a.
template <int kMode>
__device__ __forceinline__ void mma_pre(float (&d)[4], float (&dl)[4],
                                        const TcFrag& a, const float b0,
                                        const float b1) {
  if (kMode == kOneBf16) {
    mma_bf16(d, a.h[0], a.h[1], pack_bf16(b0, b1));
  } else if (kMode == kSplitTf32) {
    uint32_t bh0, bl0, bh1, bl1;
    split_tf32(b0, bh0, bl0);
    split_tf32(b1, bh1, bl1);
    mma_tf32(dl, a.l[0], a.l[1], a.l[2], a.l[3], bh0, bh1);
    mma_tf32(dl, a.h[0], a.h[1], a.h[2], a.h[3], bl0, bl1);
    mma_tf32(d, a.h[0], a.h[1], a.h[2], a.h[3], bh0, bh1);
  } else {
    mma_tf32(d, a.h[0], a.h[1], a.h[2], a.h[3], tf32_rna(b0),
             tf32_rna(b1));
  }
}

// Row pitch (floats) of A and of the z buffers in shared memory: >= 8 RB
// and = 8 mod 32, so the 64-bit fragment loads of the A z product are
// bank-conflict free (the A^T u product's 32-bit loads see a 2-way
// conflict).
template <int RB>
constexpr int tc_pitch() {
  return ((8 * RB + 23) / 32) * 32 + 8;
}

template <int RB, int NT>
constexpr size_t tc_smem_bytes() {
  return sizeof(float) *
         ((size_t)kTcWarps * NT * 8 * tc_pitch<RB>() +          // A
          (size_t)kTcWarps * kTcProblems * tc_pitch<RB>() +     // z partials
          (size_t)2 * kTcProblems * tc_pitch<RB>() +            // z (x2)
          (size_t)kTcWarps * kTcProblems +                      // max |res|
          (size_t)kTcWarps * kTcProblems +                      // max |x|
          (size_t)kTcWarps * kTcProblems);                      // max |d|
}

// One CTA: 16 problems (tile) of one set, 8 warps x NT tiles of 8 entries.
template <int RB, int NT, bool kBf16>
__device__ __forceinline__ void adm_tc_tile(const FilterArgs& a,
                                            const int tile) {
  constexpr int RP = tc_pitch<RB>();
  constexpr int PP = kTcWarps * NT * 8;  // padded problem length
  extern __shared__ __align__(16) float smem[];
  float* As = smem;                                  // [PP][RP]
  float* zred = As + PP * RP;                        // [W][16][RP]
  float* zs = zred + kTcWarps * kTcProblems * RP;    // [2][16][RP]
  float* rmx = zs + 2 * kTcProblems * RP;            // [W][16]
  float* xmx = rmx + kTcWarps * kTcProblems;         // [W][16]
  float* dmx = xmx + kTcWarps * kTcProblems;         // [W][16]
  __shared__ int s_done[kTcProblems];
  __shared__ int s_new[kTcProblems];
  __shared__ int s_all;

  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int p = a.p;
  int reff = a.r;
  if (a.d_rank) reff = min(max(*a.d_rank, 0), a.r);
  const int j0 = tile * kTcProblems;

  // Stage A (p x r, column-major) row-major, zero padded.
  for (int idx = tid; idx < PP * RP; idx += kTcThreads) {
    const int row = idx / RP, k = idx - row * RP;
    As[idx] = (row < p && k < reff) ? a.A[row + (int64_t)k * a.lda] : 0.0f;
  }
  if (tid < kTcProblems) s_done[tid] = (j0 + tid >= a.N);

  // x for (problems g, g+8) x (entries 2t, 2t+1) of each of my NT tiles;
  // fragment order: [0] = (g, 2t), [1] = (g, 2t+1), [2] = (g+8, 2t),
  // [3] = (g+8, 2t+1).
  float x[NT][4], y[NT][4], d[NT][4];  // d = x - e
  const int jA = j0 + g, jB = j0 + g + 8;
  const bool vA = jA < a.N, vB = jB < a.N;
  const int64_t qA = vA ? (int64_t)a.qidx[jA] * a.sq : 0;
  const int64_t qB = vB ? (int64_t)a.qidx[jB] * a.sq : 0;
  float xmA = 0.0f, xmB = 0.0f;
#pragma unroll
  for (int i = 0; i < NT; ++i) {
    const int e0 = (w * NT + i) * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ent = e0 + h;
      float va = 0.0f, vb = 0.0f;
      if (ent < p) {
        const int64_t po = (int64_t)a.pidx[ent] * a.sp;
        if (vA) va = __ldg(a.M + po + qA);
        if (vB) vb = __ldg(a.M + po + qB);
      }
      x[i][h] = va;
      x[i][2 + h] = vb;
      xmA = fmaxf(xmA, fabsf(va));
      xmB = fmaxf(xmB, fabsf(vb));
    }
  }
  xmA = fmaxf(xmA, __shfl_xor_sync(0xffffffffu, xmA, 1));
  xmA = fmaxf(xmA, __shfl_xor_sync(0xffffffffu, xmA, 2));
  xmB = fmaxf(xmB, __shfl_xor_sync(0xffffffffu, xmB, 1));
  xmB = fmaxf(xmB, __shfl_xor_sync(0xffffffffu, xmB, 2));
  if (t == 0) {
    xmx[w * kTcProblems + g] = xmA;
    xmx[w * kTcProblems + g + 8] = xmB;
  }
  __syncthreads();
  float xiA = 0.0f, xiB = 0.0f;
#pragma unroll
  for (int q = 0; q < kTcWarps; ++q) {
    xiA = fmaxf(xiA, xmx[q * kTcProblems + g]);
    xiB = fmaxf(xiB, xmx[q * kTcProblems + g + 8]);
  }
  // A zero problem has the exact solution z = 0: its first z is 0 and the
  // stop test (0 < eps * 0 is false) is replaced by "done at once" below.
  const float invA = xiA > 0.0f ? 1.0f / xiA : 0.0f;
  const float invB = xiB > 0.0f ? 1.0f / xiB : 0.0f;
  float betaA = xiA > 0.0f ? a.beta0_scale * invA : 1.0f;
  float betaB = xiB > 0.0f ? a.beta0_scale * invB : 1.0f;
  const float bbarA = betaA * a.beta_bar_ratio;
  const float bbarB = betaB * a.beta_bar_ratio;
  if (tid < kTcProblems) {
    float xm = 0.0f;
    for (int q = 0; q < kTcWarps; ++q) xm = fmaxf(xm, xmx[q * kTcProblems + tid]);
    if (!(xm > 0.0f)) s_done[tid] = s_done[tid] | 2;  // zero problem
  }

  // Iteration 1, step 1 with z_0 = y_0 = 0: e_1 = S_{1/beta_0}(x); partial
  // products of z_1 = A^T (x - e_1).
  // second accumulators for the split products' cross terms, except on
  // the largest shapes where they would spill
  constexpr bool kDual = !(NT == 8 && RB >= 7);
  float zacc[RB][4], zlo_store[kDual ? RB : 1][4];
  float (*zlo)[4] = kDual ? zlo_store : zacc;
#pragma unroll
  for (int rb = 0; rb < RB; ++rb)
#pragma unroll
    for (int q = 0; q < 4; ++q) zacc[rb][q] = zlo[rb][q] = 0.0f;
  auto zsum = [&](int rb, int q) {
    return kDual ? zacc[rb][q] + zlo[rb][q] : zacc[rb][q];
  };
  {
    const float ibA = 1.0f / betaA, ibB = 1.0f / betaB;
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      float u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float ib = q < 2 ? ibA : ibB;
        d[i][q] = clip(x[i][q], ib);  // x - S_{1/beta_0}(x)
        y[i][q] = 0.0f;
        u[q] = d[i][q];
      }
      const int n0 = (w * NT + i) * 8;
      const float af[4] = {u[0], u[2], u[1], u[3]};
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) {
        const float b0 = As[(n0 + 2 * t) * RP + rb * 8 + g];
        const float b1 = As[(n0 + 2 * t + 1) * RP + rb * 8 + g];
        if (a.lowp_iters == 0)
          mma_f32<kSplitTf32>(zacc[rb], zlo[rb], af, b0, b1);
        else if (kBf16)
          mma_f32<kOneBf16>(zacc[rb], zlo[rb], af, b0, b1);
        else
          mma_f32<kOneTf32>(zacc[rb], zlo[rb], af, b0, b1);
      }
    }
  }

  int cur = 0;
  int it = 1;  // index of the z whose partial products are in zacc
  float rmA = 0.0f, rmB = 0.0f;  // residual max of the last pass
  float dmA = 0.0f, dmB = 0.0f;  // max |x - e| of the last pass
  bool last_split = false;       // the last pass used split products
  while (true) {
    // ---- publish partials of z_it and the last pass's residual max -----
#pragma unroll
    for (int rb = 0; rb < RB; ++rb) {
      float* zr = zred + (w * kTcProblems) * RP + rb * 8 + 2 * t;
      *reinterpret_cast<float2*>(zr + g * RP) =
          make_float2(zsum(rb, 0), zsum(rb, 1));
      *reinterpret_cast<float2*>(zr + (g + 8) * RP) =
          make_float2(zsum(rb, 2), zsum(rb, 3));
    }
    if (it > 1) {
      rmA = fmaxf(rmA, __shfl_xor_sync(0xffffffffu, rmA, 1));
      rmA = fmaxf(rmA, __shfl_xor_sync(0xffffffffu, rmA, 2));
      rmB = fmaxf(rmB, __shfl_xor_sync(0xffffffffu, rmB, 1));
      rmB = fmaxf(rmB, __shfl_xor_sync(0xffffffffu, rmB, 2));
      dmA = fmaxf(dmA, __shfl_xor_sync(0xffffffffu, dmA, 1));
      dmA = fmaxf(dmA, __shfl_xor_sync(0xffffffffu, dmA, 2));
      dmB = fmaxf(dmB, __shfl_xor_sync(0xffffffffu, dmB, 1));
      dmB = fmaxf(dmB, __shfl_xor_sync(0xffffffffu, dmB, 2));
      if (t == 0) {
        rmx[w * kTcProblems + g] = rmA;
        rmx[w * kTcProblems + g + 8] = rmB;
        dmx[w * kTcProblems + g] = dmA;
        dmx[w * kTcProblems + g + 8] = dmB;
      }
    }
    __syncthreads();  // (A)
    // ---- stop test for z_{it-1} (in zs[cur]) ------------------------------
    if (tid < kTcProblems) {
      int nw = 0;
      const int sd = s_done[tid];
      if (it == 1) {
        if (sd == 2) nw = 1;  // zero problem: z = 0 now
      } else if (sd == 0) {
        float rm = 0.0f, xm = 0.0f, dm = 0.0f;
        for (int q = 0; q < kTcWarps; ++q) {
          rm = fmaxf(rm, rmx[q * kTcProblems + tid]);
          xm = fmaxf(xm, xmx[q * kTcProblems + tid]);
          dm = fmaxf(dm, dmx[q * kTcProblems + tid]);
        }
        if (last_split && rm < a.eps * fmaxf(dm, kStopNormFloor * xm))
          nw = 1;
        else if (it - 1 >= a.max_iter)
          nw = 2;
      }
      s_new[tid] = nw;
      if (nw) s_done[tid] = 1;
    }
    // ---- z_it = sum of the warps' partials (fixed order) -------------------
    {
      float* zn = zs + (cur ^ 1) * kTcProblems * RP;
      for (int idx = tid; idx < kTcProblems * 8 * RB; idx += kTcThreads) {
        const int row = idx / (8 * RB), k = idx - row * (8 * RB);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < kTcWarps; ++q)
          s += zred[(q * kTcProblems + row) * RP + k];
        zn[row * RP + k] = s;
      }
    }
    __syncthreads();  // (B)
    // ---- outputs of the problems that stopped on z_{it-1} ----------------
    {
      const float* zc = zs + cur * kTcProblems * RP;
      for (int idx = tid; idx < kTcProblems * a.r; idx += kTcThreads) {
        const int row = idx / a.r, k = idx - row * a.r;
        const int nw = s_new[row];
        if (!nw || j0 + row >= a.N) continue;
        const float zv = (it == 1) ? 0.0f : zc[row * RP + k];
        const float sc = a.scale ? a.scale[k] : 1.0f;
        a.Z[(int64_t)a.qidx[j0 + row] + k * a.ldz] =
            (k < reff) ? zv * sc : 0.0f;
        if (k == 0 && a.iters_out)
          a.iters_out[j0 + row] = (nw == 1) ? (it - 1) : -(it - 1);
      }
    }
    if (tid == 0) {
      int all = 1;
      for (int q = 0; q < kTcProblems; ++q) all &= (s_done[q] & 1);
      s_all = all;
    }
    __syncthreads();
    if (s_all) break;
    cur ^= 1;

    // ---- one pass: A z_it, residual, dual step, next shrinkage, A^T u ----
    const bool split = it > a.lowp_iters;
    const bool bf16 = !split && kBf16;
    float zf[RB][4];
    {
      const float* zc = zs + cur * kTcProblems * RP;
#pragma unroll
      for (int kb = 0; kb < RB; ++kb) {
        const float2 lo = *reinterpret_cast<const float2*>(
            zc + g * RP + kb * 8 + 2 * t);
        const float2 hi = *reinterpret_cast<const float2*>(
            zc + (g + 8) * RP + kb * 8 + 2 * t);
        zf[kb][0] = lo.x;  // (g, slot t)     = z[g][2t]
        zf[kb][1] = hi.x;  // (g+8, slot t)   = z[g+8][2t]
        zf[kb][2] = lo.y;  // (g, slot t+4)   = z[g][2t+1]
        zf[kb][3] = hi.y;  // (g+8, slot t+4) = z[g+8][2t+1]
      }
    }
    const float bnA = fminf(a.rho * betaA, bbarA);
    const float bnB = fminf(a.rho * betaB, bbarB);
    const float ibnA = 1.0f / bnA, ibnB = 1.0f / bnB;
    rmA = rmB = dmA = dmB = 0.0f;
#pragma unroll
    for (int rb = 0; rb < RB; ++rb)
#pragma unroll
      for (int q = 0; q < 4; ++q) zacc[rb][q] = zlo[rb][q] = 0.0f;
    // z fragments split once per iteration where registers allow
    constexpr bool kPreZ = NT <= 4;
    TcFrag zpre[kPreZ ? RB : 1];
    if (kPreZ) {
#pragma unroll
      for (int kb = 0; kb < RB; ++kb) {
        if (split)
          tc_prep<kSplitTf32>(zpre[kPreZ ? kb : 0], zf[kb]);
        else if (bf16)
          tc_prep<kOneBf16>(zpre[kPreZ ? kb : 0], zf[kb]);
        else
          tc_prep<kOneTf32>(zpre[kPreZ ? kb : 0], zf[kb]);
      }
    }
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int n0 = (w * NT + i) * 8;
      float wz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      float wl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kb = 0; kb < RB; ++kb) {
        const float2 bb = *reinterpret_cast<const float2*>(
            As + (n0 + g) * RP + kb * 8 + 2 * t);
        if (kPreZ) {
          if (split)
            mma_pre<kSplitTf32>(wz, wl, zpre[kPreZ ? kb : 0], bb.x, bb.y);
          else if (bf16)
            mma_pre<kOneBf16>(wz, wl, zpre[kPreZ ? kb : 0], bb.x, bb.y);
          else
            mma_pre<kOneTf32>(wz, wl, zpre[kPreZ ? kb : 0], bb.x, bb.y);
        } else {
          if (split)
            mma_f32<kSplitTf32>(wz, wl, zf[kb], bb.x, bb.y);
          else if (bf16)
            mma_f32<kOneBf16>(wz, wl, zf[kb], bb.x, bb.y);
          else
            mma_f32<kOneTf32>(wz, wl, zf[kb], bb.x, bb.y);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) wz[q] += wl[q];
      float u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float beta = q < 2 ? betaA : betaB;
        const float ibn = q < 2 ? ibnA : ibnB;
        const float res = d[i][q] - wz[q];
        if (q < 2) {
          rmA = fmaxf(rmA, fabsf(res));
          dmA = fmaxf(dmA, fabsf(d[i][q]));
        } else {
          rmB = fmaxf(rmB, fabsf(res));
          dmB = fmaxf(dmB, fabsf(d[i][q]));
        }
        y[i][q] = fmaf(beta, res, y[i][q]);
        const float yb = y[i][q] * ibn;
        const float c = clip(x[i][q] - wz[q] + yb, ibn);
        d[i][q] = wz[q] - yb + c;
        u[q] = wz[q] + c;
      }
      const float af[4] = {u[0], u[2], u[1], u[3]};
      if (kPreZ) {
        // u split once per tile (measured faster for NT <= 4; on the
        // widest shape splitting per product schedules better)
        TcFrag uf;
        if (split)
          tc_prep<kSplitTf32>(uf, af);
        else if (bf16)
          tc_prep<kOneBf16>(uf, af);
        else
          tc_prep<kOneTf32>(uf, af);
#pragma unroll
        for (int rb = 0; rb < RB; ++rb) {
          const float b0 = As[(n0 + 2 * t) * RP + rb * 8 + g];
          const float b1 = As[(n0 + 2 * t + 1) * RP + rb * 8 + g];
          if (split)
            mma_pre<kSplitTf32>(zacc[rb], zlo[rb], uf, b0, b1);
          else if (bf16)
            mma_pre<kOneBf16>(zacc[rb], zlo[rb], uf, b0, b1);
          else
            mma_pre<kOneTf32>(zacc[rb], zlo[rb], uf, b0, b1);
        }
      } else {
#pragma unroll
        for (int rb = 0; rb < RB; ++rb) {
          const float b0 = As[(n0 + 2 * t) * RP + rb * 8 + g];
          const float b1 = As[(n0 + 2 * t + 1) * RP + rb * 8 + g];
          if (split)
            mma_f32<kSplitTf32>(zacc[rb], zlo[rb], af, b0, b1);
          else if (bf16)
            mma_f32<kOneBf16>(zacc[rb], zlo[rb], af, b0, b1);
          else
            mma_f32<kOneTf32>(zacc[rb], zlo[rb], af, b0, b1);
        }
      }
    }
    betaA = bnA;
    betaB = bnB;
    last_split = split;
    ++it;
  }
}

// Two CTAs per SM (<= 128 registers a thread) when the state fits and two
// copies of the shared memory do; else one.
template <int RB, int NT>
constexpr int tc_min_blocks() {
  // shapes whose state fits in 128 registers without spilling (checked
  // with -Xptxas -v)
  return (((NT == 2 && RB <= 4) || (NT == 4 && RB <= 3)) &&
          2 * tc_smem_bytes<RB, NT>() <= 220 * 1024)
             ? 2
             : 1;
}

template <int RB, int NT>
__global__ void __launch_bounds__(kTcThreads, tc_min_blocks<RB, NT>())
    adm_tc_kernel(const FilterArgs a) {
  // the BF16 low-precision passes get their own copy of the tile code (one
  // more product mode in the same code raised register pressure into spills)
  if (a.lowp_bf16)
    adm_tc_tile<RB, NT, true>(a, blockIdx.x);
  else
    adm_tc_tile<RB, NT, false>(a, blockIdx.x);
}

template <int RB, int NT>
__global__ void __launch_bounds__(kTcThreads, tc_min_blocks<RB, NT>())
    adm_tc_batched_kernel(const FilterArgs* __restrict__ sets,
                          const int32_t* __restrict__ tiles) {
  const FilterArgs a = sets[tiles[2 * blockIdx.x]];
  if (a.skip != nullptr && *a.skip != 0) return;  // whole CTA, one set
  if (a.lowp_bf16)
    adm_tc_tile<RB, NT, true>(a, tiles[2 * blockIdx.x + 1]);
  else
    adm_tc_tile<RB, NT, false>(a, tiles[2 * blockIdx.x + 1]);
}

template <int RB, int NT>
cudaError_t launch_tc(const FilterArgs* a, const FilterArgs* d_sets,
                      const int32_t* d_tiles, int ntiles, cudaStream_t st) {
  constexpr size_t smem = tc_smem_bytes<RB, NT>();
  static std::atomic<bool> configured{false};  // same value from any thread
  if (!configured.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(
        adm_tc_kernel<RB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(adm_tc_batched_kernel<RB, NT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    configured.store(true, std::memory_order_release);
  }
  if (a) {
    const int grid = (a->N + kTcProblems - 1) / kTcProblems;
    adm_tc_kernel<RB, NT><<<grid, kTcThreads, smem, st>>>(*a);
  } else {
    adm_tc_batched_kernel<RB, NT><<<ntiles, kTcThreads, smem, st>>>(d_sets,
                                                                  d_tiles);
  }
  return cudaGetLastError();
}

// shape = (NT index) * 8 + (RB - 1); NT in {2, 4, 8} (p <= 128, 256, 512)
template <int NT>
cudaError_t dispatch_rb(int rb, const FilterArgs* a, const FilterArgs* d_sets,
                        const int32_t* d_tiles, int ntiles, cudaStream_t st) {
  switch (rb) {
    case 1: return launch_tc<1, NT>(a, d_sets, d_tiles, ntiles, st);
    case 2: return launch_tc<2, NT>(a, d_sets, d_tiles, ntiles, st);
    case 3: return launch_tc<3, NT>(a, d_sets, d_tiles, ntiles, st);
    case 4: return launch_tc<4, NT>(a, d_sets, d_tiles, ntiles, st);
    case 5: return launch_tc<5, NT>(a, d_sets, d_tiles, ntiles, st);
    case 6: return launch_tc<6, NT>(a, d_sets, d_tiles, ntiles, st);
    case 7: return launch_tc<7, NT>(a, d_sets, d_tiles, ntiles, st);
    case 8: return launch_tc<8, NT>(a, d_sets, d_tiles, ntiles, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_shape(int shape, const FilterArgs* a,
                           const FilterArgs* d_sets, const int32_t* d_tiles,
                           int ntiles, cudaStream_t st) {
  const int ni = shape / 8, rb = shape % 8 + 1;
  if (ni == 0) return dispatch_rb<2>(rb, a, d_sets, d_tiles, ntiles, st);
  if (ni == 1) return dispatch_rb<4>(rb, a, d_sets, d_tiles, ntiles, st);
  if (ni == 2) return dispatch_rb<8>(rb, a, d_sets, d_tiles, ntiles, st);
  return cudaErrorInvalidValue;
}

}  // namespace

bool l1_filter_tc_fits(int p, int r) {
  return p >= 1 && p <= 512 && r >= 1 && r <= 64;
}

int tc_shape_class(int p, int r) {
  const int ni = p <= 128 ? 0 : (p <= 256 ? 1 : 2);
  return ni * 8 + (r + 7) / 8 - 1;
}

cudaError_t l1_filter_tc_launch(const FilterArgs& a, cudaStream_t st) {
  if (!l1_filter_tc_fits(a.p, a.r)) return cudaErrorInvalidValue;
  if (a.N <= 0) return cudaSuccess;
  return dispatch_shape(tc_shape_class(a.p, a.r), &a, nullptr, nullptr, 0,
                        st);
}

cudaError_t l1_filter_tc_batched_launch(int shape, const FilterArgs* d_sets,
                                        const int32_t* d_tiles, int ntiles,
                                        cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  return dispatch_shape(shape, nullptr, d_sets, d_tiles, ntiles, st);
}

}  // namespace pcp
