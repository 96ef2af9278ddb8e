// S pass S = M - Lu Lv^T (Algorithm 2 output) on the fifth-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory, M / S tiles moved
// by TMA (cp.async.bulk.tensor), one persistent CTA per SM.
//
// Roofline: 8 bytes of HBM traffic per entry (read M, write S) against 2r
// flops; at r = 50 the FP32 SIMT form needs as long for its FMAs as HBM
// needs for the bytes, so the rank-r product goes to the tensor pipe and
// the SMs only stream.  FP32 accuracy from split TF32: x = hi + lo with hi,
// lo rounded to TF32, L = lo_u hi_v + hi_u lo_v + hi_u hi_v accumulated in
// FP32 (the dropped lo lo term is ~2^-22 of each product).
//
// Tile: 128 rows (TMEM lanes) x 64 columns of M.  Per CTA, a contiguous
// range of tiles in row-block-major order, processed by a warp-specialised
// pipeline whose stages hand over through mbarriers:
//   * warp 0 (one thread): TMA loads of M tiles into an NS-stage ring;
//   * warps 2-3 and 8-9: operand producers: the 128 x K split Lu rows of
//     the current row block (A, rewritten when the row block changes, after
//     the MMAs of the previous tile are done) and the 64 x K split Lv rows
//     of each tile (B, double-buffered; the next tile's loads are issued
//     before the wait for a free buffer);
//   * warp 1 (one thread; the warp owns the TMEM allocation): 3 K/8
//     tcgen05.mma per tile into one of two 64-column accumulators, committed
//     to barriers that free the B buffer and hand the accumulator on;
//   * warps 4-7: epilogue: tcgen05.ld of the accumulator (warp 4 + q reads
//     lanes 32 q ..), S = M - L in place in the stage, one thread issues the
//     TMA store and frees the stage once the store has read it.
// M loads and S stores carry an L2 evict-first policy so that the factor
// rows, which every CTA reads, stay in L2.
// Operands use the no-swizzle K-major layout: a core matrix is 8 rows x 16
// bytes stored contiguously; the 8-row groups of a k-group are adjacent
// (stride 128 B) and k-groups follow each other (stride rows x 16 B), which
// makes element (i, k) of a 128-row block sit at float offset
// (k / 4) * 512 + 4 i + k % 4.
//
// Every mbarrier wait is bounded by %globaltimer; a wait that runs out
// counts into a device word (read by the solve's diagnostics), stops the
// CTA's tile loop, drains the copies and MMAs it issued (again bounded),
// frees its tensor memory and returns.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace pcp {

__device__ int g_spass_tc_timeouts = 0;

namespace {

constexpr int kTcRows = 128;   // tile rows = TMEM lanes = MMA M
constexpr int kTcCols = 64;    // tile columns = MMA N
constexpr int kTcThreads = 320;  // 10 warps, see the role map below
constexpr uint32_t kTileBytes = kTcRows * kTcCols * sizeof(float);
constexpr uint32_t kTmemCols = 2 * kTcCols;  // two accumulator buffers
constexpr int kMaxStages = 6;

struct SpassTcArgs {
  const float* Lu;
  int64_t ldu;
  const float* Lv;
  int64_t ldv;
  int r;
  int ns;  // M stages
  int64_t m, n;
  int64_t ntn, ntiles;
  unsigned long long timeout_ns;
};

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// M is read once and S written once: both streams carry an L2 evict-first
// policy so that the factor rows (re-read by every CTA) stay in L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;"
               : "=l"(p));
  return p;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map,
                                            int x, int y, uint32_t bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::"
      "complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar),
      "l"(policy)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x,
                                             int y, uint32_t src,
                                             uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint "
      "[%0, {%1, %2}], [%3], %4;" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(src), "l"(policy)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// the store groups except the newest one have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: start address, leading (k-group) and
// stride (8-row group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo,
                                              uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) |
         ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::tf32: F32 accumulator, A and B TF32, both
// K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            ((uint32_t)(kTcCols >> 3) << 17) |
                            ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a,
                                         uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(bar)
      : "memory");
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
        "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]),
        "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- roles ---------------------------------------------------------------------
// warp 0: TMA producer of M tiles; warp 1: TMEM owner and MMA issuer;
// warps 2-3 and 8-9: operand producers (split Lu / Lv rows); warps 4-7:
// epilogue (warp 4 + q reads TMEM lanes 32 q .. 32 q + 31).
constexpr int kOpThreads = 128;
constexpr int kEpiThreads = 128;

struct Bars {
  uint64_t mfull[kMaxStages];   // M tile landed (TMA transaction count)
  uint64_t mempty[kMaxStages];  // its S tile has been read out by TMA
  uint64_t bfull[2];            // B operand written (128 arrivals)
  uint64_t bempty[2];           // MMAs that read it are done (commit)
  uint64_t accfull[2];          // accumulator complete (commit)
  uint64_t accempty[2];         // epilogue has read it (128 arrivals)
  uint64_t afull;               // A operand written (128 arrivals)
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar)
               : "memory");
}

// Bounded wait that also gives up once another role has aborted; the first
// wait to run out raises the CTA's abort flag and counts the event.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity,
                                           unsigned long long timeout_ns,
                                           int* abort) {
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*reinterpret_cast<volatile int*>(abort)) return false;
    if (globaltimer_ns() - t0 > timeout_ns) {
      if (atomicExch(abort, 1) == 0) atomicAdd(&g_spass_tc_timeouts, 1);
      return false;
    }
  }
}

// bounded wait without the abort short-cut (drain after an abort)
__device__ __forceinline__ void wait_phase_drain(uint32_t bar, uint32_t parity,
                                                 unsigned long long timeout_ns) {
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try(bar, parity) && globaltimer_ns() - t0 <= timeout_ns) {
  }
}

// barrier 1 over the four epilogue warps, with an OR vote
__device__ __forceinline__ bool epi_sync_or(bool v) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)v)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, 128;" ::: "memory");
}

// ---- operand staging ---------------------------------------------------------------
// Split rows [row0, row0 + ROWS) of X (column-major, ld) into TF32 hi / lo
// blocks in the K-major core-matrix layout (float offset (k/4) ROWS 4 +
// 4 i + k%4); rows past nrows and k >= r are 0.  Item it = (k-group, row i)
// = kg ROWS + i: four coalesced column loads, one 16-byte store per block at
// float4 index it.  A pass covers IPT items per thread; loads and stores are
// separate calls so that loads can be issued ahead of the wait for the
// destination buffer.
template <int K, int ROWS, int IPT>
struct RowPass {
  static constexpr int kItems = ROWS * (K / 4);
  float x[IPT][4];
  __device__ __forceinline__ void load(const float* __restrict__ X, int64_t ld,
                                       int64_t row0, int64_t nrows, int r,
                                       int base, int ot) {
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int it = base + q * kOpThreads + ot;
      const int i = it % ROWS, kg = it / ROWS;
      const int64_t gi = row0 + i;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = 4 * kg + kk;
        x[q][kk] = (it < kItems && k < r && gi < nrows)
                       ? __ldg(X + gi + (int64_t)k * ld)
                       : 0.0f;
      }
    }
  }
  __device__ __forceinline__ void store(float* hi, int base, int ot) const {
    float4* hi4 = reinterpret_cast<float4*>(hi);
    float4* lo4 = reinterpret_cast<float4*>(hi + ROWS * K);
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int it = base + q * kOpThreads + ot;
      if (it < kItems) {
        float h[4], l[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          h[kk] = to_tf32(x[q][kk]);
          l[kk] = to_tf32(x[q][kk] - h[kk]);
        }
        hi4[it] = make_float4(h[0], h[1], h[2], h[3]);
        lo4[it] = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
  }
};

// the 3 K/8 MMAs of one tile: lo_u hi_v, hi_u lo_v, hi_u hi_v
template <int K>
__device__ __forceinline__ void issue_tile(uint32_t a_hi, uint32_t b_hi,
                                           uint32_t d_tmem) {
  constexpr uint32_t kLboA = kTcRows * 16, kLboB = kTcCols * 16;
  const uint32_t a_lo = a_hi + kTcRows * K * 4, b_lo = b_hi + kTcCols * K * 4;
  const uint32_t pa[3] = {a_lo, a_hi, a_hi};
  const uint32_t pb[3] = {b_hi, b_lo, b_hi};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int s = 0; s < K / 8; ++s)
      mma_tf32(d_tmem, smem_desc(pa[p] + s * 2 * kLboA, kLboA, 128),
               smem_desc(pb[p] + s * 2 * kLboB, kLboB, 128),
               (p | s) ? 1u : 0u);
}

template <int K>
__global__ void __launch_bounds__(kTcThreads, 1)
    spass_tc_kernel(const __grid_constant__ CUtensorMap tmM,
                    const __grid_constant__ CUtensorMap tmS,
                    const SpassTcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t per = (a.ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per;
  const int64_t t1 = min(a.ntiles, t0 + per);
  if (t0 >= t1) return;
  const int cnt = (int)(t1 - t0);
  const int NS = a.ns;

  // shared memory map: A (hi, lo) | B[2] (hi, lo) | M stages | barriers
  float* As = reinterpret_cast<float*>(sm);
  float* Bs = As + 2 * kTcRows * K;
  unsigned char* Mst = sm + 4 * (2 * kTcRows * K + 4 * kTcCols * K);
  Bars* bb = reinterpret_cast<Bars*>(Mst + (size_t)NS * kTileBytes);
  int* abort = &bb->abort;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_addr(&bb->mfull[s]), 1);
      mbar_init(smem_addr(&bb->mempty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_addr(&bb->bfull[b]), kOpThreads);
      mbar_init(smem_addr(&bb->bempty[b]), 1);
      mbar_init(smem_addr(&bb->accfull[b]), 1);
      mbar_init(smem_addr(&bb->accempty[b]), kEpiThreads);
    }
    mbar_init(smem_addr(&bb->afull), kOpThreads);
    bb->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(
                     reinterpret_cast<uint64_t>(&tmM))
                 : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(
                     reinterpret_cast<uint64_t>(&tmS))
                 : "memory");
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(smem_addr(&bb->tmem)),
        "r"(kTmemCols)
        : "memory");
    asm volatile(
        "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::
            : "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(&bb->tmem);

  auto tile_i = [&](int u) { return (t0 + u) / a.ntn; };
  auto tile_j = [&](int u) { return (t0 + u) % a.ntn; };
  const unsigned long long tmo = a.timeout_ns;
  int loads = 0, mmas = 0;  // issued (threads 0 and 32)

  if (tid == 0) {
    // ---- TMA producer: M tiles into the stage ring ----------------------------
    const uint64_t pol = evict_first_policy();
    for (int v = 0; v < cnt; ++v) {
      const int s = v % NS;
      if (v >= NS &&
          !wait_phase(smem_addr(&bb->mempty[s]), ((v / NS) - 1) & 1, tmo, abort))
        break;
      const uint32_t bar = smem_addr(&bb->mfull[s]);
      mbar_expect_tx(bar, kTileBytes);
      tma_load_2d(smem_addr(Mst + (size_t)s * kTileBytes), &tmM,
                  (int)(tile_i(v) * kTcRows), (int)(tile_j(v) * kTcCols), bar,
                  pol);
      loads = v + 1;
    }
  } else if (tid == 32) {
    // ---- MMA issuer -----------------------------------------------------------------
    int q = 0;
    for (int v = 0; v < cnt; ++v) {
      if (v == 0 || tile_i(v) != tile_i(v - 1)) {
        if (!wait_phase(smem_addr(&bb->afull), q & 1, tmo, abort)) break;
        ++q;
      }
      if (!wait_phase(smem_addr(&bb->bfull[v & 1]), (v >> 1) & 1, tmo, abort))
        break;
      if (v >= 2 && !wait_phase(smem_addr(&bb->accempty[v & 1]),
                                ((v >> 1) - 1) & 1, tmo, abort))
        break;
      tc_fence_after();
      issue_tile<K>(smem_addr(As), smem_addr(Bs + (v & 1) * 2 * kTcCols * K),
                    tmem + (v & 1) * kTcCols);
      mma_commit(smem_addr(&bb->accfull[v & 1]));
      mma_commit(smem_addr(&bb->bempty[v & 1]));
      mmas = v + 1;
    }
  } else if (warp == 2 || warp == 3 || warp >= 8) {
    // ---- operand producers ---------------------------------------------------------
    // B of tile v + 1 is loaded into registers right after B of tile v is
    // stored, so its loads are in flight while the buffer is still busy.
    const int ot = warp >= 8 ? tid - 192 : tid - 64;
    constexpr int kIB = K / 8;  // B items per thread: 64 (K/4) / 128
    using PassB = RowPass<K, kTcCols, kIB>;
    using PassA = RowPass<K, kTcRows, 8>;
    PassB pb;
    pb.load(a.Lv, a.ldv, tile_j(0) * kTcCols, a.n, a.r, 0, ot);
    for (int v = 0; v < cnt; ++v) {
      if (v == 0 || tile_i(v) != tile_i(v - 1)) {
        // A is read by the MMAs of every earlier tile: wait for tile v - 1
        if (v >= 1 && !wait_phase(smem_addr(&bb->bempty[(v - 1) & 1]),
                                  ((v - 1) >> 1) & 1, tmo, abort))
          break;
        for (int base = 0; base < PassA::kItems; base += 8 * kOpThreads) {
          PassA pa;
          pa.load(a.Lu, a.ldu, tile_i(v) * kTcRows, a.m, a.r, base, ot);
          pa.store(As, base, ot);
        }
        fence_proxy_async();
        mbar_arrive(smem_addr(&bb->afull));
      }
      if (v >= 2 && !wait_phase(smem_addr(&bb->bempty[v & 1]),
                                ((v - 2) >> 1) & 1, tmo, abort))
        break;
      pb.store(Bs + (v & 1) * 2 * kTcCols * K, 0, ot);
      fence_proxy_async();
      mbar_arrive(smem_addr(&bb->bfull[v & 1]));
      if (v + 1 < cnt)
        pb.load(a.Lv, a.ldv, tile_j(v + 1) * kTcCols, a.n, a.r, 0, ot);
    }
  } else if (warp >= 4 && warp < 8) {
    // ---- epilogue: S = M - L in place in the stage, TMA store ---------------
    const int et = tid - 128;  // = TMEM lane
    const uint64_t pol = evict_first_policy();
    const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int v = 0; v < cnt; ++v) {
      const bool ok =
          wait_phase(smem_addr(&bb->accfull[v & 1]), (v >> 1) & 1, tmo,
                     abort) &&
          wait_phase(smem_addr(&bb->mfull[v % NS]), (v / NS) & 1, tmo, abort);
      if (epi_sync_or(!ok)) break;
      tc_fence_after();
      uint32_t acc[2][32];
      tmem_ld32(tlane + (v & 1) * kTcCols, acc[0]);
      tmem_ld32(tlane + (v & 1) * kTcCols + 32, acc[1]);
      tc_fence_before();
      mbar_arrive(smem_addr(&bb->accempty[v & 1]));
      float* Ms = reinterpret_cast<float*>(Mst + (size_t)(v % NS) * kTileBytes);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          float* p = Ms + (h * 32 + c) * kTcRows + et;
          *p = *p - __uint_as_float(acc[h][c]);
        }
      fence_proxy_async();
      epi_sync();
      if (et == 0) {
        tma_store_2d(&tmS, (int)(tile_i(v) * kTcRows),
                     (int)(tile_j(v) * kTcCols), smem_addr(Ms), pol);
        bulk_wait_read_all_but_one();  // the store of tile v - 1 has left
        if (v >= 1) mbar_arrive(smem_addr(&bb->mempty[(v - 1) % NS]));
      }
    }
    if (et == 0) bulk_wait_all();
  }

  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort)) {
    // drain what this CTA issued: the newest load of every stage, the newest
    // MMA group (bounded; no abort short-cut)
    if (tid == 0)
      for (int v = max(0, loads - NS); v < loads; ++v)
        wait_phase_drain(smem_addr(&bb->mfull[v % NS]), (v / NS) & 1, tmo);
    if (tid == 32 && mmas > 0)
      wait_phase_drain(smem_addr(&bb->accfull[(mmas - 1) & 1]),
                       ((mmas - 1) >> 1) & 1, tmo);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

size_t tc_smem_bytes(int K, int ns) {
  return (size_t)4 * (2 * kTcRows * K + 4 * kTcCols * K) +
         (size_t)ns * kTileBytes + sizeof(Bars);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t,
                                 void*, const cuuint64_t*, const cuuint64_t*,
                                 const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const float* base, int64_t ld, int64_t m,
              int64_t n) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {kTcRows, kTcCols};
  const cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
             const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int K>
pcp_status launch_k(const CUtensorMap& mm, const CUtensorMap& ms,
                    const SpassTcArgs& a0, cudaStream_t st) {
  // the opt-in limit and the attribute are per process; host threads that
  // race here query or set the same values
  static std::atomic<int> optin_cache{0};
  int optin = optin_cache.load(std::memory_order_acquire);
  if (!optin) {
    int dev = 0;
    PCP_CUDA(cudaGetDevice(&dev));
    PCP_CUDA(cudaDeviceGetAttribute(
        &optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    optin_cache.store(optin, std::memory_order_release);
  }
  SpassTcArgs a = a0;
  const size_t fixed = tc_smem_bytes(K, 0);
  a.ns = (int)std::min<size_t>(kMaxStages, ((size_t)optin - fixed) / kTileBytes);
  if (a.ns < 3) return PCP_ERR_UNSUPPORTED;
  const size_t smem = tc_smem_bytes(K, a.ns);
  static std::atomic<size_t> smem_set{0};
  if (smem_set.load(std::memory_order_acquire) != smem) {
    PCP_CUDA(cudaFuncSetAttribute(spass_tc_kernel<K>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    smem_set.store(smem, std::memory_order_release);
  }
  const int grid =
      (int)std::max<int64_t>(1, std::min<int64_t>(a.ntiles, device_sm_count()));
  spass_tc_kernel<K><<<grid, kTcThreads, smem, st>>>(mm, ms, a);
  PCP_CUDA(cudaGetLastError());
  return PCP_OK;
}

}  // namespace

bool spass_tc_fits(const float* dM, int64_t ldm, float* dS, int64_t lds,
                   int r, int64_t m, int64_t n) {
  return r >= 1 && r <= 64 && m >= kTcRows && n >= kTcCols &&
         m < (1ll << 31) && n < (1ll << 31) &&
         ((uintptr_t)dM % 16 == 0) && ((uintptr_t)dS % 16 == 0) &&
         (ldm % 4 == 0) && (lds % 4 == 0) && encode_fn() != nullptr;
}

pcp_status spass_tc_launch(const float* dM, int64_t ldm, const float* dLu,
                           int64_t ldu, const float* dLv, int64_t ldv, int r,
                           float* dS, int64_t lds, int64_t m, int64_t n,
                           cudaStream_t st) {
  if (!spass_tc_fits(dM, ldm, dS, lds, r, m, n)) return PCP_ERR_UNSUPPORTED;
  CUtensorMap mm, ms;
  if (!make_map(&mm, dM, ldm, m, n) || !make_map(&ms, dS, lds, m, n))
    return PCP_ERR_UNSUPPORTED;
  SpassTcArgs a;
  a.Lu = dLu;
  a.ldu = ldu;
  a.Lv = dLv;
  a.ldv = ldv;
  a.r = r;
  a.ns = 0;
  a.m = m;
  a.n = n;
  a.ntn = (n + kTcCols - 1) / kTcCols;
  a.ntiles = ((m + kTcRows - 1) / kTcRows) * a.ntn;
  a.timeout_ns = 1000000000ull;  // 1 s per wait
  switch ((r + 7) / 8) {
    case 1: return launch_k<8>(mm, ms, a, st);
    case 2: return launch_k<16>(mm, ms, a, st);
    case 3: return launch_k<24>(mm, ms, a, st);
    case 4: return launch_k<32>(mm, ms, a, st);
    case 5: return launch_k<40>(mm, ms, a, st);
    case 6: return launch_k<48>(mm, ms, a, st);
    case 7: return launch_k<56>(mm, ms, a, st);
    default: return launch_k<64>(mm, ms, a, st);
  }
}

pcp_status spass_tc_read_timeouts(int* out) {
  PCP_CUDA(cudaMemcpyFromSymbol(out, g_spass_tc_timeouts, sizeof(int)));
  return PCP_OK;
}

}  // namespace pcp
