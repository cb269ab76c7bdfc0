// FP32-mixed pair sums of the single-box step: density + EOS (Eq. 1), the
// IAD matrix, and momentum/energy with artificial viscosity (Eqs. 2-5).  One
// thread per target particle, grid-stride over the sorted particles (a warp's
// targets are neighbours in Morton order, so their neighbours share L1 lines);
// the per-particle bodies are in sph_pairs32.cuh.
#include <cuda_runtime.h>

#include "sph_pairs32.cuh"

namespace sph {

namespace {

using pairs32::F32;
using pairs32::Lists;

constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) k_density_p(const Grid* gp, F32 f, OutView o,
                                                        const double* u, Lists L, int64_t n,
                                                        float Bn, int sinc_n, double gamma,
                                                        bool gradh, uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    pairs32::density_one(a, g, f, o, u, L, Bn, sinc_n, gamma, err, true, 0, gradh);
}

__global__ void __launch_bounds__(kThreads) k_iad_p(const Grid* gp, F32 f, OutView o, Lists L,
                                                    int64_t n, int sinc_n, uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    pairs32::iad_one(a, g, f, o, L, sinc_n, err);
}

__global__ void __launch_bounds__(kThreads) k_momentum_p(const Grid* gp, F32 f, OutView o,
                                                         Lists L, int64_t n, int sinc_n,
                                                         float alpha, uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    pairs32::momentum_one(a, g, f, o, L, sinc_n, alpha, err);
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
  k_density_p<<<blocks_for(n, ctx->sm_count), kThreads, 0, st>>>(
      ctx->grid, f32_of(ctx), o, s.u, lists_of(ctx), n, (float)ctx->Bn, (int)ctx->prm.sinc_n,
      ctx->prm.gamma, ctx->prm.gradh != 0, ctx->err);
  ctx->launches += 1;
}

void launch_iad_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                    cudaStream_t st) {
  (void)s;
  k_iad_p<<<blocks_for(n, ctx->sm_count), kThreads, 0, st>>>(
      ctx->grid, f32_of(ctx), o, lists_of(ctx), n, (int)ctx->prm.sinc_n, ctx->err);
  ctx->launches += 1;
}

void launch_momentum_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st) {
  (void)s;
  k_momentum_p<<<blocks_for(n, ctx->sm_count), kThreads, 0, st>>>(
      ctx->grid, f32_of(ctx), o, lists_of(ctx), n, (int)ctx->prm.sinc_n, (float)ctx->prm.alpha,
      ctx->err);
  ctx->launches += 1;
}

}  // namespace sph
