// Shared device/host helpers of the l1-filtering PCP library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "pcp_l1f.h"

namespace pcp {

// ---- error reporting (api.cu owns the thread-local message) --------------
void set_error(const char* fmt, ...);
pcp_status cuda_fail(cudaError_t e, const char* what, const char* file,
                     int line);

#define PCP_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) return ::pcp::cuda_fail(_e, #call, __FILE__, \
                                                   __LINE__);            \
  } while (0)

#define PCP_ARG(cond, ...)            \
  do {                                \
    if (!(cond)) {                    \
      ::pcp::set_error(__VA_ARGS__);  \
      return PCP_ERR_ARG;             \
    }                                 \
  } while (0)

// ---- host-side stage ranges ----------------------------------------------
// One NVTX range per stage of a solve (seed, filters, S pass), pushed while
// the stage's work is enqueued: a profiler that records NVTX (Nsight
// Systems, ncu --nvtx) groups the launches by stage; without one attached
// the calls do nothing.  next() closes the open range and opens the next.
class NvtxStages {
 public:
  explicit NvtxStages(const char* first) { nvtxRangePushA(first); }
  void next(const char* name) {
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  ~NvtxStages() { nvtxRangePop(); }
  NvtxStages(const NvtxStages&) = delete;
  NvtxStages& operator=(const NvtxStages&) = delete;
};

// ---- device helpers ------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Soft shrinkage S_eta(x) = sgn(x) max(|x| - eta, 0) (Section 2).
__device__ __forceinline__ float shrink(float x, float eta) {
  return copysignf(fmaxf(fabsf(x) - eta, 0.0f), x);
}
__device__ __forceinline__ double shrink(double x, double eta) {
  return copysign(fmax(fabs(x) - eta, 0.0), x);
}
// The part of x that the shrinkage removes: x - S_eta(x), i.e. x clipped to
// [-eta, eta].
__device__ __forceinline__ float clip(float x, float eta) {
  return fminf(fmaxf(x, -eta), eta);
}

// Largest number of CTAs the library launches per device in one
// cooperative grid; bounds per-block scratch arrays.
constexpr int kMaxCoopBlocks = 1024;

int device_sm_count();

}  // namespace pcp
