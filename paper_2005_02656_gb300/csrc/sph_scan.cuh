// Exclusive scan of int32 counts into int64 starts on the device, three
// passes (per-block sums, one block over the block sums, per-block apply).
// Used by the reverse-list build (sph_adjoint.cu) and the gravity tree
// (sph_gravity.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {
namespace scan {

constexpr int kScanItems = 4096;  // per scan block (1024 threads x 4)

// Exclusive scan of cnt[0..n) into start[0..n], three passes.
static __device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    int64_t s = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) wsum[lane] = s;
  }
  __syncthreads();
  const int64_t before = (w > 0 ? wsum[w - 1] : 0) + x - v;
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

static __global__ void __launch_bounds__(1024) k_scan_sum(const int32_t* cnt, int64_t n, int64_t* part) {
  const int64_t base = blockIdx.x * (int64_t)kScanItems + threadIdx.x * 4;
  int64_t s = 0;
  for (int i = 0; i < 4; ++i)
    if (base + i < n) s += cnt[base + i];
  int64_t tot;
  block_exclusive(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(1024) k_scan_parts(int64_t* part, int nparts) {
  // one block: exclusive scan of the block sums, in chunks of 1024
  int64_t carry = 0;
  for (int b0 = 0; b0 < nparts; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const int64_t v = i < nparts ? part[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive(v, &tot);
    if (i < nparts) part[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) part[nparts] = carry;
}

static __global__ void __launch_bounds__(1024) k_scan_apply(const int32_t* cnt, int64_t n,
                                                     const int64_t* part, int nparts,
                                                     int64_t* start) {
  const int64_t base = blockIdx.x * (int64_t)kScanItems + threadIdx.x * 4;
  int64_t v[4], s = 0;
  for (int i = 0; i < 4; ++i) {
    v[i] = base + i < n ? cnt[base + i] : 0;
    s += v[i];
  }
  int64_t tot;
  int64_t ex = block_exclusive(s, &tot) + part[blockIdx.x];
  for (int i = 0; i < 4; ++i) {
    if (base + i < n) start[base + i] = ex;
    ex += v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) start[n] = part[nparts];
}


// Host: start[0..n] = exclusive scan of cnt[0..n), start[n] = total.  part
// needs ceil(n / kScanItems) + 1 entries.
static inline void exclusive_scan(const int32_t* cnt, int64_t n, int64_t* part, int64_t* start,
                                  cudaStream_t st) {
  const int nparts = (int)((n + kScanItems - 1) / kScanItems);
  k_scan_sum<<<nparts > 0 ? nparts : 1, 1024, 0, st>>>(cnt, n, part);
  k_scan_parts<<<1, 1024, 0, st>>>(part, nparts);
  k_scan_apply<<<nparts > 0 ? nparts : 1, 1024, 0, st>>>(cnt, n, part, nparts, start);
}

}  // namespace scan
}  // namespace sph
