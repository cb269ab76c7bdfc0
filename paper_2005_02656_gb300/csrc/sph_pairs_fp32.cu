// FP32-mixed pair sums of the single-box step: density + EOS (Eq. 1), the
// IAD matrix, and momentum/energy with artificial viscosity (Eqs. 2-5).  NSUB
// threads per target particle (consecutive lanes split its list and add their
// partial sums by a fixed butterfly), grid-stride over the sorted particles (a
// warp's targets are neighbours in Morton order, so their neighbours share L1
// lines); the per-particle bodies are in sph_pairs32.cuh.
#include <cuda_runtime.h>

#include "sph_pairs32.cuh"

namespace sph {

namespace {

using pairs32::F32;
using pairs32::Lists;

constexpr int kThreads = 128;
// Lanes sharing one target's neighbour list in the momentum kernel.  Its
// 80-byte neighbour records make it bound by L1 gathers; four lanes on one
// list measured 6.2 ms against 7.8 ms with one (8.4M particles), while the
// density and IAD kernels (16-byte records) are fastest with one lane.  The
// ensemble's default configuration uses the same split.
constexpr int kMomentumLanes = 4;

template <int NSUB>
__global__ void __launch_bounds__(kThreads) k_density_p(const Grid* gp, F32 f, OutView o,
                                                        const double* u, Lists L, int64_t n,
                                                        float Bn, int sinc_n, double gamma,
                                                        bool gradh, uint32_t* err) {
  const Grid g = *gp;
  const int64_t nt = n * NSUB, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < nt; t0 += stride) {
    const int64_t t = t0 + threadIdx.x;
    const bool on = t < nt;
    pairs32::density_one<NSUB>(on ? t / NSUB : 0, g, f, o, u, L, Bn, sinc_n, gamma, err, on,
                               (int)(t % NSUB), gradh);
  }
}

template <int NSUB>
__global__ void __launch_bounds__(kThreads) k_iad_p(const Grid* gp, F32 f, OutView o, Lists L,
                                                    int64_t n, int sinc_n, uint32_t* err) {
  const Grid g = *gp;
  const int64_t nt = n * NSUB, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < nt; t0 += stride) {
    const int64_t t = t0 + threadIdx.x;
    const bool on = t < nt;
    pairs32::iad_one<NSUB>(on ? t / NSUB : 0, g, f, o, L, sinc_n, err, on, (int)(t % NSUB));
  }
}

template <int NSUB>
__global__ void __launch_bounds__(kThreads) k_momentum_p(const Grid* gp, F32 f, OutView o,
                                                         Lists L, int64_t n, int sinc_n,
                                                         float alpha, uint32_t* err) {
  const Grid g = *gp;
  const int64_t nt = n * NSUB, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < nt; t0 += stride) {
    const int64_t t = t0 + threadIdx.x;
    const bool on = t < nt;
    pairs32::momentum_one<NSUB>(on ? t / NSUB : 0, g, f, o, L, sinc_n, alpha, err, on,
                                (int)(t % NSUB));
  }
}

inline F32 f32_of(sph_ctx* ctx) {
  F32 f;
  f.pos = ctx->pos32;
  f.rec_d = ctx->rec_d;
  f.rec_i = ctx->rec_i;
  f.rec_m = ctx->rec_m;
  f.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab32 : nullptr;
  return f;
}

inline Lists lists_of(sph_ctx* ctx) {
  Lists l;
  l.nn = ctx->nn;
  l.nbr = ctx->nbr;
  l.max_nb = ctx->prm.max_nb;
  return l;
}

inline int blocks_for(int64_t n, int sm) {
  int64_t b = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_density_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st) {
  k_density_p<1><<<blocks_for(n, ctx->sm_count), kThreads, 0, st>>>(
      ctx->grid, f32_of(ctx), o, s.u, lists_of(ctx), n, (float)ctx->Bn, (int)ctx->prm.sinc_n,
      ctx->prm.gamma, ctx->prm.gradh != 0, ctx->err);
  ctx->launches += 1;
}

void launch_iad_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                    cudaStream_t st) {
  (void)s;
  k_iad_p<1><<<blocks_for(n, ctx->sm_count), kThreads, 0, st>>>(
      ctx->grid, f32_of(ctx), o, lists_of(ctx), n, (int)ctx->prm.sinc_n, ctx->err);
  ctx->launches += 1;
}

void launch_momentum_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st) {
  (void)s;
  k_momentum_p<kMomentumLanes><<<blocks_for(n * kMomentumLanes, ctx->sm_count), kThreads, 0, st>>>(
      ctx->grid, f32_of(ctx), o, lists_of(ctx), n, (int)ctx->prm.sinc_n, (float)ctx->prm.alpha,
      ctx->err);
  ctx->launches += 1;
}

}  // namespace sph
