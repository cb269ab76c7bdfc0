// FP32-mixed pair sums: density + EOS (Eq. 1), the IAD matrix, and
// momentum/energy with artificial viscosity (Eqs. 2-5).
//
// One warp per occupied cell; the warps of a CTA are independent (each owns
// the cell's stencil in shared memory, so no CTA barrier is involved).  Each
// target particle of the cell gets `tpp` lanes (the largest power of two with
// tpp * targets <= 32) that walk interleaved entries of its neighbour list;
// an entry gives the neighbour's particle index and the FP32 shift of its
// cell relative to the target's cell (sph_tile.cuh), so a pair separation is
// (offset_b + shift) - offset_a in FP32 with no FP64 operation.  Neighbour
// data is gathered through L1/L2 from packed per-particle records:
//   rec_d (density)  = (offset x, y, z, m)                       16 B
//   rec_i (IAD)      = (offset x, y, z, m/rho)                   16 B
//   rec_m (momentum) = (offset, 1/h^2), (v, m), (B_n/h^3, P/rho^2, c, 1/rho),
//                      (C00 C01 C02 C11), (C12 C22 - -)          80 B
// Partial sums are combined with warp shuffles.  Results go to the caller's
// FP64 arrays and to the records the next kernel gathers.
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

namespace sph {

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;

struct F32 {
  const float4* pos;    // offset in own cell x, y, z, h
  const float4* rec_d;  // offset x, y, z, m
  float4* rec_i;        // offset x, y, z, m/rho
  float4* rec_m;        // 5 float4 per particle
};

struct Tile {
  const uint32_t* occ;
  const uint32_t* tbl_start;
  const uint32_t* tbl_count;
  const int32_t* nn;
  const uint16_t* nbr;
  int max_nb;
};

struct WarpCell {
  Stencil S;
  float4 sh[kMaxStencil];  // stencil shifts as float4 (one 16-byte load)
};

__device__ __forceinline__ float wrap_axis(float d, const Grid& g, int ax) {
  if (d > g.halfL32[ax])
    d -= g.L32[ax];
  else if (d < -g.halfL32[ax])
    d += g.L32[ax];
  return d;
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int tpp) {
  for (int o = tpp >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_tpp(int na) {
  int t = 1;
  while (t < 32 && (t * 2) * na <= 32) t *= 2;
  return t;
}

// Sets up the warp's cell; returns false if the cell was skipped (overflow).
__device__ __forceinline__ bool setup_cell(const Grid& g, const Tile& T, uint32_t cell,
                                           WarpCell& C) {
  const int lane = threadIdx.x & 31;
  build_stencil_warp(g, T.occ[cell], T.tbl_start, T.tbl_count, C.S);
  if (lane < C.S.ncell)
    C.sh[lane] = make_float4(C.S.shift[lane][0], C.S.shift[lane][1], C.S.shift[lane][2], 0.0f);
  __syncwarp();
  return C.S.off[C.S.ncell] <= kMaxSlots && C.S.maxpop <= kMaxCellPop;
}

// FP32 separation b - a from the neighbour's offset and its cell shift.
__device__ __forceinline__ void rel(const Grid& g, bool wrap, float4 rb, float4 sh, float4 pa,
                                    float& dx, float& dy, float& dz) {
  dx = (rb.x + sh.x) - pa.x;
  dy = (rb.y + sh.y) - pa.y;
  dz = (rb.z + sh.z) - pa.z;
  if (wrap) {
    if (g.periodic[0]) dx = wrap_axis(dx, g, 0);
    if (g.periodic[1]) dy = wrap_axis(dy, g, 1);
    if (g.periodic[2]) dz = wrap_axis(dz, g, 2);
  }
}

// ---------------------------------------------------------------- density --
__global__ void __launch_bounds__(kThreads) k_density_w(const Grid* gp, F32 f, OutView o,
                                                        const double* u, Tile T, float Bn,
                                                        int sinc_n, double gamma, uint32_t* err) {
  __shared__ WarpCell cells[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpCell& C = cells[warp];
  const Grid g = *gp;
  const bool wrap = g.wrap32 != 0;
  const uint32_t nw = gridDim.x * kWarps;
  for (uint32_t cell = blockIdx.x * kWarps + warp; cell < g.n_occ; cell += nw) {
    if (!setup_cell(g, T, cell, C)) continue;
    const int a0 = C.S.a0, na = C.S.na;
    const int tpp = warp_tpp(na), tpw = 32 / tpp, sub = lane & (tpp - 1);
    for (int t0 = 0; t0 < na; t0 += tpw) {
      const int i = t0 + lane / tpp;
      const bool active = i < na;
      const int a = a0 + (active ? i : 0);
      const float4 pa = f.pos[a];
      const float hinv2 = 1.0f / (pa.w * pa.w);
      const float norm = Bn * hinv2 / pa.w;
      const int cnt = active ? min(T.nn[a], T.max_nb) : 0;
      const uint16_t* row = T.nbr + (int64_t)a * T.max_nb;
      float acc = 0.0f;
      int k = sub;
      // two independent entries per iteration for memory-level parallelism
      for (; k + tpp < cnt; k += 2 * tpp) {
        const uint32_t e0 = row[k], e1 = row[k + tpp];
        const float4 r0 = f.rec_d[entry_particle(C.S, e0)];
        const float4 r1 = f.rec_d[entry_particle(C.S, e1)];
        const float4 s0 = C.sh[e0 >> kOffBits], s1 = C.sh[e1 >> kOffBits];
        float dx, dy, dz, ex, ey, ez;
        rel(g, wrap, r0, s0, pa, dx, dy, dz);
        rel(g, wrap, r1, s1, pa, ex, ey, ez);
        const float q0 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float q1 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        acc = fmaf(r0.w, kernel_w32(q0 * hinv2, norm, sinc_n), acc);
        acc = fmaf(r1.w, kernel_w32(q1 * hinv2, norm, sinc_n), acc);
      }
      if (k < cnt) {
        const uint32_t e0 = row[k];
        const float4 r0 = f.rec_d[entry_particle(C.S, e0)];
        float dx, dy, dz;
        rel(g, wrap, r0, C.sh[e0 >> kOffBits], pa, dx, dy, dz);
        const float q0 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        acc = fmaf(r0.w, kernel_w32(q0 * hinv2, norm, sinc_n), acc);
      }
      acc = group_sum(acc, tpp);
      if (active && sub == 0) {
        const float ma = f.rec_d[a].w;
        const float rho = fmaf(ma, norm, acc);
        const double rho64 = (double)rho;
        const double p = (gamma - 1.0) * rho64 * u[a];
        const double c = sqrt(gamma * p / rho64);
        o.rho[a] = rho64;
        o.p[a] = p;
        o.c[a] = c;
        const float inv_rho = 1.0f / rho;
        f.rec_i[a] = make_float4(pa.x, pa.y, pa.z, ma * inv_rho);
        float4* m = f.rec_m + 5 * (int64_t)a;
        m[0] = make_float4(pa.x, pa.y, pa.z, hinv2);
        m[2] = make_float4(norm, (float)(p / (rho64 * rho64)), (float)c, inv_rho);
        if (!isfinite(rho64) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
      }
    }
  }
}

// -------------------------------------------------------------------- IAD --
__global__ void __launch_bounds__(kThreads) k_iad_w(const Grid* gp, F32 f, OutView o, Tile T,
                                                    int sinc_n, uint32_t* err) {
  __shared__ WarpCell cells[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpCell& C = cells[warp];
  const Grid g = *gp;
  const bool wrap = g.wrap32 != 0;
  const uint32_t nw = gridDim.x * kWarps;
  for (uint32_t cell = blockIdx.x * kWarps + warp; cell < g.n_occ; cell += nw) {
    if (!setup_cell(g, T, cell, C)) continue;
    const int a0 = C.S.a0, na = C.S.na;
    const int tpp = warp_tpp(na), tpw = 32 / tpp, sub = lane & (tpp - 1);
    for (int t0 = 0; t0 < na; t0 += tpw) {
      const int i = t0 + lane / tpp;
      const bool active = i < na;
      const int a = a0 + (active ? i : 0);
      const float4 pa = f.pos[a];
      const float4 ma = f.rec_m[5 * (int64_t)a];      // (offset, 1/h^2)
      const float norm = f.rec_m[5 * (int64_t)a + 2].x;
      const float inv_h = 1.0f / pa.w;
      const int cnt = active ? min(T.nn[a], T.max_nb) : 0;
      const uint16_t* row = T.nbr + (int64_t)a * T.max_nb;
      float t00 = 0, t01 = 0, t02 = 0, t11 = 0, t12 = 0, t22 = 0;
      for (int k = sub; k < cnt; k += tpp) {
        const uint32_t e = row[k];
        const float4 rb = f.rec_i[entry_particle(C.S, e)];
        float dx, dy, dz;
        rel(g, wrap, rb, C.sh[e >> kOffBits], pa, dx, dy, dz);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        // separation scaled by 1/h_a keeps tau of order one in FP32
        dx *= inv_h;
        dy *= inv_h;
        dz *= inv_h;
        const float w = rb.w * kernel_w32(r2 * ma.w, norm, sinc_n);
        const float wx = w * dx, wy = w * dy, wz = w * dz;
        t00 = fmaf(wx, dx, t00);
        t01 = fmaf(wx, dy, t01);
        t02 = fmaf(wx, dz, t02);
        t11 = fmaf(wy, dy, t11);
        t12 = fmaf(wy, dz, t12);
        t22 = fmaf(wz, dz, t22);
      }
      t00 = group_sum(t00, tpp);
      t01 = group_sum(t01, tpp);
      t02 = group_sum(t02, tpp);
      t11 = group_sum(t11, tpp);
      t12 = group_sum(t12, tpp);
      t22 = group_sum(t22, tpp);
      if (active && sub == 0) {
        const float c00 = t11 * t22 - t12 * t12;
        const float c01 = t02 * t12 - t01 * t22;
        const float c02 = t01 * t12 - t02 * t11;
        const float c11 = t00 * t22 - t02 * t02;
        const float c12 = t01 * t02 - t00 * t12;
        const float c22 = t00 * t11 - t01 * t01;
        const float det = t00 * c00 + t01 * c01 + t02 * c02;
        float tmax = fmaxf(fmaxf(fabsf(t00), fabsf(t01)), fmaxf(fabsf(t02), fabsf(t11)));
        tmax = fmaxf(tmax, fmaxf(fabsf(t12), fabsf(t22)));
        float Cm[6];
        if (!isfinite(det) || fabsf(det) <= 1e-6f * tmax * tmax * tmax) {
          raise_flag(err, SPH_FLAG_SINGULAR_IAD);
          for (int q = 0; q < 6; ++q) Cm[q] = 0.0f;
        } else {
          const float sc = ma.w / det;  // C = tau_scaled^{-1} / h_a^2
          Cm[0] = c00 * sc;
          Cm[1] = c01 * sc;
          Cm[2] = c02 * sc;
          Cm[3] = c11 * sc;
          Cm[4] = c12 * sc;
          Cm[5] = c22 * sc;
        }
        float4* m = f.rec_m + 5 * (int64_t)a;
        m[3] = make_float4(Cm[0], Cm[1], Cm[2], Cm[3]);
        m[4] = make_float4(Cm[4], Cm[5], 0.0f, 0.0f);
        double* out = o.iad + 6 * (int64_t)a;
        for (int q = 0; q < 6; ++q) out[q] = (double)Cm[q];
      }
    }
  }
}

// ------------------------------------------------------- momentum/energy --
__global__ void __launch_bounds__(kThreads) k_momentum_w(const Grid* gp, F32 f, OutView o,
                                                         Tile T, int sinc_n, float alpha,
                                                         uint32_t* err) {
  __shared__ WarpCell cells[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpCell& C = cells[warp];
  const Grid g = *gp;
  const bool wrap = g.wrap32 != 0;
  const uint32_t nw = gridDim.x * kWarps;
  for (uint32_t cell = blockIdx.x * kWarps + warp; cell < g.n_occ; cell += nw) {
    if (!setup_cell(g, T, cell, C)) continue;
    const int a0 = C.S.a0, na = C.S.na;
    const int tpp = warp_tpp(na), tpw = 32 / tpp, sub = lane & (tpp - 1);
    for (int t0 = 0; t0 < na; t0 += tpw) {
      const int i = t0 + lane / tpp;
      const bool active = i < na;
      const int a = a0 + (active ? i : 0);
      const float4* ra = f.rec_m + 5 * (int64_t)a;
      const float4 pa = ra[0];       // offset, 1/h_a^2
      const float4 va = ra[1];       // v, m
      const float4 qa = ra[2];       // B_n/h^3, P/rho^2, c, 1/rho
      const float4 Aa = ra[3], Ba = ra[4];
      const float a00 = Aa.x, a01 = Aa.y, a02 = Aa.z, a11 = Aa.w, a12 = Ba.x, a22 = Ba.y;
      const float Xa = qa.y, csa = qa.z, ira = qa.w;
      const int cnt = active ? min(T.nn[a], T.max_nb) : 0;
      const uint16_t* row = T.nbr + (int64_t)a * T.max_nb;
      float accx = 0, accy = 0, accz = 0, du = 0;
      // one pair of Eqs. 2-5 (x_ab = -d, d = x_b - x_a)
      auto pair = [&](const float4* rb, float4 sh) {
        const float4 b0 = rb[0];
        float dx, dy, dz;
        rel(g, wrap, b0, sh, pa, dx, dy, dz);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float4 b2 = rb[2];
        const float Wa = kernel_w32(r2 * pa.w, qa.x, sinc_n);
        const float Wb = kernel_w32(r2 * b0.w, b2.x, sinc_n);  // clamped at t = 4 (S = 0)
        const float Cadx = fmaf(a02, dz, fmaf(a01, dy, a00 * dx));
        const float Cady = fmaf(a12, dz, fmaf(a11, dy, a01 * dx));
        const float Cadz = fmaf(a22, dz, fmaf(a12, dy, a02 * dx));
        const float4 b3 = rb[3], b4 = rb[4];
        const float Cbdx = fmaf(b3.z, dz, fmaf(b3.y, dy, b3.x * dx));
        const float Cbdy = fmaf(b4.x, dz, fmaf(b3.w, dy, b3.y * dx));
        const float Cbdz = fmaf(b4.y, dz, fmaf(b4.x, dy, b3.z * dx));
        const float4 vb = rb[1];
        const float vabx = va.x - vb.x, vaby = va.y - vb.y, vabz = va.z - vb.z;
        const float xv = -fmaf(dz, vabz, fmaf(dy, vaby, dx * vabx));
        // Eq. 5 without a branch: w_ab = x_ab.v_ab / r, Pi = 0 unless approaching
        const float w = xv * rsqrtf(r2);
        const float vsig = csa + b2.z - 3.0f * w;
        const float Pi = xv < 0.0f ? -0.5f * alpha * vsig * w : 0.0f;
        const float irb = b2.w;
        const float mb = vb.w;
        const float fa = mb * Wa * fmaf(0.5f * Pi, ira, Xa);
        const float fb = mb * Wb * fmaf(0.5f * Pi, irb, b2.y);
        accx -= fmaf(fa, Cadx, fb * Cbdx);
        accy -= fmaf(fa, Cady, fb * Cbdy);
        accz -= fmaf(fa, Cadz, fb * Cbdz);
        const float vCa = fmaf(vabz, Cadz, fmaf(vaby, Cady, vabx * Cadx));
        const float vCb = fmaf(vabz, Cbdz, fmaf(vaby, Cbdy, vabx * Cbdx));
        du = fmaf(mb, fmaf(Wa * fmaf(0.25f * Pi, ira, Xa), vCa, 0.25f * Pi * irb * Wb * vCb), du);
      };
      // entries are decoded one step ahead so the next record's address is
      // known while the current pair computes
      int k = sub;
      uint32_t e = k < cnt ? row[k] : 0u;
      while (k < cnt) {
        const float4* rb = f.rec_m + 5 * (int64_t)entry_particle(C.S, e);
        const float4 sh = C.sh[e >> kOffBits];
        k += tpp;
        e = k < cnt ? row[k] : 0u;
        pair(rb, sh);
      }
      accx = group_sum(accx, tpp);
      accy = group_sum(accy, tpp);
      accz = group_sum(accz, tpp);
      du = group_sum(du, tpp);
      if (active && sub == 0) {
        o.ax[a] = accx;
        o.ay[a] = accy;
        o.az[a] = accz;
        o.du[a] = du;
        if (!isfinite(accx) || !isfinite(accy) || !isfinite(accz) || !isfinite(du))
          raise_flag(err, SPH_FLAG_NONFINITE);
      }
    }
  }
}

inline F32 f32_of(sph_ctx* ctx) {
  F32 f;
  f.pos = ctx->pos32;
  f.rec_d = ctx->rec_d;
  f.rec_i = ctx->rec_i;
  f.rec_m = ctx->rec_m;
  return f;
}

inline Tile tile_of(sph_ctx* ctx) {
  Tile t;
  t.occ = ctx->occ;
  t.tbl_start = ctx->tbl_start;
  t.tbl_count = ctx->tbl_count;
  t.nn = ctx->nn;
  t.nbr = ctx->nbr;
  t.max_nb = ctx->prm.max_nb;
  return t;
}

template <typename K>
int grid_of(K kernel, int sm) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
  return (per_sm > 0 ? per_sm : 1) * sm;
}

int g_blocks[3] = {0, 0, 0};

}  // namespace

void launch_density_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st) {
  (void)n;
  if (!g_blocks[0]) g_blocks[0] = grid_of(k_density_w, ctx->sm_count);
  k_density_w<<<g_blocks[0], kThreads, 0, st>>>(ctx->grid, f32_of(ctx), o, s.u, tile_of(ctx),
                                                (float)ctx->Bn, (int)ctx->prm.sinc_n,
                                                ctx->prm.gamma, ctx->err);
  ctx->launches += 1;
}

void launch_iad_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                    cudaStream_t st) {
  (void)s;
  (void)n;
  if (!g_blocks[1]) g_blocks[1] = grid_of(k_iad_w, ctx->sm_count);
  k_iad_w<<<g_blocks[1], kThreads, 0, st>>>(ctx->grid, f32_of(ctx), o, tile_of(ctx),
                                            (int)ctx->prm.sinc_n, ctx->err);
  ctx->launches += 1;
}

void launch_momentum_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st) {
  (void)s;
  (void)n;
  if (!g_blocks[2]) g_blocks[2] = grid_of(k_momentum_w, ctx->sm_count);
  k_momentum_w<<<g_blocks[2], kThreads, 0, st>>>(ctx->grid, f32_of(ctx), o, tile_of(ctx),
                                                 (int)ctx->prm.sinc_n, (float)ctx->prm.alpha,
                                                 ctx->err);
  ctx->launches += 1;
}

}  // namespace sph
