// Internal: the asynchronous halves of the batched solve, shared by
// pcp_l1filter_batch and the serving loop.
#pragma once

#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace pcp {

struct BatchInstance {
  int mp = 0, np = 0, k0 = 0, kmax = 0;
  double lam_seed = 0, lam_full = 0;
  std::vector<int64_t> rows, cols;
  int32_t *d_rows = nullptr, *d_cols = nullptr, *d_rbar = nullptr,
          *d_cbar = nullptr;
  void* d_work = nullptr;
  int32_t *d_iters = nullptr, *d_bad = nullptr;
  int* d_rank = nullptr;
};

// Per-instance diagnostics, reduced on the device at the end of a batch.
struct BatchSummary {
  int rank, iters, converged, rank_raw, bad, iters_max;
  long long unconverged, iters_sum;
  double residual;
  int skipped;  // filters skipped: the seed failed Eq. rank_test and grows
};

struct BatchHandle {
  int count = 0;
  std::vector<BatchInstance> inst;
  std::vector<pcp_problem> probs;
  void* d_base = nullptr;  // one stream-ordered allocation
  size_t bytes = 0;
  std::vector<char> h_gat, h_asm, h_sargs, h_filt, h_stask, h_ctask;
  BatchSummary* d_summary = nullptr;
  // stage boundaries (start, seed done, filters done, S pass done) when
  // the launch is timed
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<pcp_status> status;
  std::vector<char> skipped;  // per instance, from the summary
  // a batch plan's workspace: size_only asks batch_launch for the bytes
  // alone (no device work); prealloc uses d_base / bytes as given (never
  // freed by batch_finish); indices_ready skips the index uploads (already
  // on the device, e.g. while the launches are captured into a graph)
  bool size_only = false, prealloc = false, indices_ready = false;
};

// Section 3.5's grown seed: for a seed of mp x np whose raw rank rr failed
// Eq. rank_test, the next seed is (s_r rr) x (s_c rr) (never smaller than
// the current one); false when there is nothing to grow to, or the grown
// seed would pass half a side or 512.  One definition for the host's
// growth loop and the device's filter gate, so both decide alike.
__host__ __device__ inline bool grown_seed_dims(int rr, int mp, int np,
                                                int64_t m, int64_t n,
                                                double s_r, double s_c,
                                                int* gm, int* gn) {
  const long long a = llround(s_r * rr), b = llround(s_c * rr);
  *gm = a > mp ? (int)a : mp;
  *gn = b > np ? (int)b : np;
  return rr >= 1 && !(*gm == mp && *gn == np) && 2 * (int64_t)*gm <= m &&
         2 * (int64_t)*gn <= n && *gm <= 512 && *gn <= 512;
}

pcp_status batch_validate(const pcp_problem& pr, BatchInstance* bi);
// Section 3.5: the whole sampling order behind the library's seed sample,
// and the grown seed size for a failed rank test (false: stop growing).
std::vector<int64_t> sample_order(int64_t n, uint64_t seed);
bool grown_seed_size(const pcp_params& q, const pcp_info& inf, int* gm,
                     int* gn);
// Device workspace one instance needs (its share of a batch).
size_t batch_footprint(const pcp_problem& pr, const BatchInstance& bi);
// Enqueue the whole batch on st (asynchronous; allocates with
// cudaMallocAsync on st).  grow_gate (per instance, may be null): the
// caller grows a seed that fails Eq. rank_test (Section 3.5), so an
// instance with grow_seed whose seed fails the test and has a grown size
// skips its filters on the device (its outputs are left unwritten; the
// summary marks it skipped, and a skipped instance the caller then does not
// grow must be run again without the gate).
pcp_status batch_launch(int count, const pcp_problem* probs, cudaStream_t st,
                        BatchHandle* h, bool timed = false,
                        const unsigned char* grow_gate = nullptr);
// With infos: synchronise st, fill one pcp_info (and h->status) per
// instance.  Always releases the workspace (stream-ordered).
pcp_status batch_finish(BatchHandle* h, pcp_info* infos, cudaStream_t st,
                        float batch_ms);

}  // namespace pcp
