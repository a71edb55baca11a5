// Shared device/host helpers of the tucker_gb300 library (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tucker_gb300.h"

namespace tk {

// Error words written by kernels (bit flags, read by the host after a call).
enum : unsigned {
  DEV_ERR_BARRIER_TIMEOUT = 1u,   // a grid barrier gave up waiting
  DEV_ERR_BOUNDS = 2u,            // an index check failed and the access was skipped
  DEV_ERR_MBAR_TIMEOUT = 4u,      // an mbarrier wait gave up
};

template <typename T> struct dtype_of;
template <> struct dtype_of<float> { static constexpr tucker_dtype value = TUCKER_F32; };
template <> struct dtype_of<double> { static constexpr tucker_dtype value = TUCKER_F64; };

inline size_t dtype_size(tucker_dtype d) { return d == TUCKER_F64 ? 8 : 4; }

// Process-wide count of kernels this library has launched (diagnostics).
void count_launches(int n);

// Lets kernel f take the largest dynamic shared memory the current device
// allows (its opt-in maximum less f's static shared memory), once per
// (device, kernel).  A per-launch setting sized to the launch races when
// several host threads launch f with different sizes: the attribute is
// global to the kernel, and one thread's smaller value fails the other's
// larger launch.
cudaError_t allow_max_dyn_smem(const void* f);

// Slab view of mode n of a tensor with dims J: element (l, i, r) at
// l + L*(i + I*r) with L = prod_{k<n} J_k, I = J_n, Rt = prod_{k>n} J_k.
// L0 = J_0 (n > 0) is the fastest sub-index of l.
struct SlabView {
  int64_t L, I, Rt, L0;
};

inline SlabView slab_view(int ndim, const int64_t* dims, int n) {
  SlabView v{1, dims[n], 1, 1};
  for (int k = 0; k < n; ++k) v.L *= dims[k];
  for (int k = n + 1; k < ndim; ++k) v.Rt *= dims[k];
  if (n > 0) v.L0 = dims[0];
  return v;
}

// Grid-wide barrier for a cooperatively launched kernel (all CTAs resident).
// Every wait is bounded: after `limit` polls the CTA records
// DEV_ERR_BARRIER_TIMEOUT in *err and returns false; callers then exit.
struct GridBarrier {
  unsigned* count;     // arrivals in the current generation
  unsigned* gen;       // generation counter
  unsigned* err;       // error word
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrival: one release-add per CTA on a counter that only grows (barrier k
// completes when it reaches k * gridDim.x); departure: acquire polling.  The
// CTA's writes are ordered before thread 0's release by the preceding
// __syncthreads.  The counter starts at 0 (memset by the host).
// team > 0: the barrier spans `team` CTAs that share b.count (a team of a
// larger cooperative grid) instead of the whole grid.
__device__ __forceinline__ bool grid_sync(const GridBarrier& b, unsigned& my_gen,
                                          unsigned long long limit = (1ull << 24),
                                          unsigned team = 0) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (my_gen + 1) * (team ? team : gridDim.x);
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(b.count), "r"(1u) : "memory");
    unsigned long long it = 0;
    while (ld_acquire_u32(b.count) < target) {
      if (++it > limit) { atomicOr(b.err, DEV_ERR_BARRIER_TIMEOUT); ok = 0; break; }
      if ((it & 1023) == 0 && (ld_acquire_u32(b.err) & DEV_ERR_BARRIER_TIMEOUT)) { ok = 0; break; }
      if (it > 4096) __nanosleep(64);
    }
    my_gen += 1;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace tk
