// sph_diagnostics_noalloc: the conservation sums of a state without any
// device allocation, for callers that cannot allocate device memory.
//
// The per-block partial sums and the last-block counter live in one
// file-scope static device array (kNaBlocks blocks, ~512 KB, held by every
// device that loads the library until the process exits).  One block of 256
// threads reduces a fixed chunk of kNaChunk particles, so the array bounds the
// state size: n <= kNaBlocks * kNaChunk = 16,777,216 particles.
//
// Host code must not pass the symbol itself to a kernel (on the host it is a
// stand-in, not a device address): the first call on a device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it per device (an atomic slot, so host threads making their first calls at
// the same time store the same address without a data race).  All calls
// share the array, so calls that overlap on the GPU (different streams, or
// different host threads) race and give wrong sums.
//
// The call ends by copying the sums to the host and synchronising the
// stream, which a stream under graph capture does not allow: a capturing
// stream is refused before any other CUDA call, leaving the capture intact.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/sph.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 8;
constexpr int64_t kNaChunk = (int64_t)kNaThreads * kNaPerThread;  // particles per block
constexpr int kNaBlocks = 8192;
constexpr int kNaSums = 8;
constexpr int64_t kNaMaxN = (int64_t)kNaBlocks * kNaChunk;
// layout: [0, kNaBlocks * kNaSums) partials, then kNaSums results, then the
// counter (as a double-sized slot)
constexpr int kNaResult = kNaBlocks * kNaSums;
constexpr int kNaCounter = kNaResult + kNaSums;
constexpr int kNaDoubles = kNaCounter + 2;

static __device__ __align__(256) double g_na_scratch[kNaDoubles];

constexpr int kMaxDevices = 64;
std::atomic<double*> g_na_ptr[kMaxDevices] = {};

__global__ void __launch_bounds__(kNaThreads) k_diag_noalloc(
    const double* x, const double* y, const double* z, const double* vx, const double* vy,
    const double* vz, const double* m, const double* u, int64_t n, double* scratch) {
  double acc[kNaSums] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t base = (int64_t)blockIdx.x * kNaChunk;
  for (int r = 0; r < kNaPerThread; ++r) {
    const int64_t p = base + (int64_t)r * kNaThreads + threadIdx.x;
    if (p < n) {
      const double mp = m[p], xp = x[p], yp = y[p], zp = z[p];
      const double vxp = vx[p], vyp = vy[p], vzp = vz[p];
      acc[0] += mp * vxp;
      acc[1] += mp * vyp;
      acc[2] += mp * vzp;
      acc[3] += 0.5 * mp * (vxp * vxp + vyp * vyp + vzp * vzp);
      acc[4] += mp * u[p];
      acc[5] += mp * (yp * vzp - zp * vyp);
      acc[6] += mp * (zp * vxp - xp * vzp);
      acc[7] += mp * (xp * vyp - yp * vxp);
    }
  }
  __shared__ double sh[kNaThreads / 32][kNaSums];
  for (int k = 0; k < kNaSums; ++k)
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int k = 0; k < kNaSums; ++k) sh[w][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < kNaSums) {
    double s = 0.0;
    for (int ww = 0; ww < kNaThreads / 32; ++ww) s += sh[ww][threadIdx.x];
    scratch[blockIdx.x * kNaSums + threadIdx.x] = s;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaCounter);
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < kNaSums) {
    // compensated sum over blocks in block order: deterministic
    double s = 0.0, comp = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
      const double yk = ((const volatile double*)scratch)[b * kNaSums + threadIdx.x] - comp;
      const double t = s + yk;
      comp = (t - s) - yk;
      s = t;
    }
    scratch[kNaResult + threadIdx.x] = s;
  }
  if (threadIdx.x == 0) *reinterpret_cast<unsigned int*>(scratch + kNaCounter) = 0u;
}

}  // namespace

extern "C" int sph_diagnostics_noalloc(const sph_state* state, double* out, sph_stream_t stream) {
  if (!state || !out) return SPH_ERR_INVALID_ARG;
  if (state->n < 0 || state->n > kNaMaxN) return SPH_ERR_INVALID_ARG;  // beyond the static scratch
  if (state->n > 0 && (!state->x || !state->y || !state->z || !state->vx || !state->vy ||
                       !state->vz || !state->m || !state->u))
    return SPH_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // a stream under capture cannot be synchronised: refuse it untouched
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return SPH_ERR_INVALID_ARG;
  }
  if (cap != cudaStreamCaptureStatusNone) return SPH_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPH_ERR_CUDA;
  double* scratch = g_na_ptr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // once per device, with that device current: the scratch's device address
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
    scratch = static_cast<double*>(p);
    g_na_ptr[dev].store(scratch, std::memory_order_release);
  }
  if (state->n == 0) {
    for (int k = 0; k < kNaSums; ++k) out[k] = 0.0;
    return SPH_OK;
  }
  const int blocks = (int)((state->n + kNaChunk - 1) / kNaChunk);
  k_diag_noalloc<<<blocks, kNaThreads, 0, st>>>(state->x, state->y, state->z, state->vx,
                                                state->vy, state->vz, state->m, state->u,
                                                state->n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + kNaResult, kNaSums * sizeof(double),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
