// FP64 pair sums: density + EOS (Eq. 1), the IAD matrix, and momentum/energy
// with artificial viscosity (Eqs. 2-5).  One warp per occupied cell (the
// warps of a CTA are independent); each target particle gets `tpp` lanes
// walking interleaved entries of its neighbour list, mapping entries to
// particles through the cell's stencil (sph_tile.cuh) and gathering the
// neighbours' FP64 fields through L1/L2 (particles are in Morton cell order,
// so a cell's neighbours share cache lines).  On this part
// the FP64 pipe bounds these kernels, so per-pair divisions are hoisted into
// per-particle arrays (m/rho, P/rho^2, 1/rho, 1/h^2, B_n/h^3).
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

namespace sph {

namespace {

struct Aux64 {
  double* vol;     // m / rho
  double* X;       // P / rho^2
  double* inv_rho;
  double* hinv2;   // 1 / h^2
  double* wnorm;   // B_n / h^3
};

__device__ __forceinline__ void sep64(const Grid& g, double xa, double ya, double za, double xb,
                                      double yb, double zb, double& dx, double& dy, double& dz) {
  dx = min_image(xb - xa, g.Lbox[0], g.halfL[0], g.periodic[0]);
  dy = min_image(yb - ya, g.Lbox[1], g.halfL[1], g.periodic[1]);
  dz = min_image(zb - za, g.Lbox[2], g.halfL[2], g.periodic[2]);
}

struct Tile64 {
  const uint32_t* occ;
  const uint32_t* tbl_start;
  const uint32_t* tbl_count;
  const int32_t* nn;
  const uint16_t* nbr;
  int max_nb;
};

constexpr int kWarps64 = 4;
constexpr int kThreads64 = 32 * kWarps64;

__device__ __forceinline__ int warp_tpp64(int na) {
  int t = 1;
  while (t < 32 && (t * 2) * na <= 32) t *= 2;
  return t;
}

template <typename T>
__device__ __forceinline__ T group_sum64(T v, int tpp) {
  for (int o = tpp >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kThreads64) k_density64(const Grid* gp, StateView s, OutView o,
                                                          Aux64 aux, Tile64 T, double Bn,
                                                          int sinc_n, double gamma,
                                                          uint32_t* err) {
  __shared__ Stencil cells[kWarps64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Stencil& S = cells[warp];
  const Grid g = *gp;
  const uint32_t nw = gridDim.x * kWarps64;
  for (uint32_t cell = blockIdx.x * kWarps64 + warp; cell < g.n_occ; cell += nw) {
    build_stencil_warp(g, T.occ[cell], T.tbl_start, T.tbl_count, S);
    if (S.off[S.ncell] <= kMaxSlots && S.maxpop <= kMaxCellPop) {
      const int tpp = warp_tpp64(S.na);
      const int tpc = 32 / tpp;
      const int sub = lane & (tpp - 1);
      for (int c0 = 0; c0 < S.na; c0 += tpc) {
        const int i = c0 + lane / tpp;
        const bool active = i < S.na;
        const int64_t a = S.a0 + (active ? i : 0);
        const double xa = s.x[a], ya = s.y[a], za = s.z[a], ha = s.h[a];
        const double hinv2 = 1.0 / (ha * ha);
        const double norm = Bn * hinv2 / ha;
        const int cnt = active ? min(T.nn[a], T.max_nb) : 0;
        const uint16_t* list = T.nbr + a * T.max_nb;
        double acc = 0.0;
        for (int k = sub; k < cnt; k += tpp) {
          const int64_t b = entry_particle(S, list[k]);
          double dx, dy, dz;
          sep64(g, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
          const double r2 = dx * dx + dy * dy + dz * dz;
          acc += s.m[b] * kernel_w64(fmin(r2 * hinv2, 4.0), norm, sinc_n);
        }
        acc = group_sum64(acc, tpp);
        if (active && sub == 0) {
          const double rho = s.m[a] * norm + acc;  // self term: W(0, h_a) = B_n / h_a^3
          const double p = (gamma - 1.0) * rho * s.u[a];
          const double c = sqrt(gamma * p / rho);
          o.rho[a] = rho;
          o.p[a] = p;
          o.c[a] = c;
          const double inv_rho = 1.0 / rho;
          aux.inv_rho[a] = inv_rho;
          aux.vol[a] = s.m[a] * inv_rho;
          aux.X[a] = p * inv_rho * inv_rho;
          aux.hinv2[a] = hinv2;
          aux.wnorm[a] = norm;
          if (!isfinite(rho) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads64) k_iad64(const Grid* gp, StateView s, OutView o,
                                                      Aux64 aux, Tile64 T, int sinc_n,
                                                      uint32_t* err) {
  __shared__ Stencil cells[kWarps64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Stencil& S = cells[warp];
  const Grid g = *gp;
  const uint32_t nw = gridDim.x * kWarps64;
  for (uint32_t cell = blockIdx.x * kWarps64 + warp; cell < g.n_occ; cell += nw) {
    build_stencil_warp(g, T.occ[cell], T.tbl_start, T.tbl_count, S);
    if (S.off[S.ncell] <= kMaxSlots && S.maxpop <= kMaxCellPop) {
      const int tpp = warp_tpp64(S.na);
      const int tpc = 32 / tpp;
      const int sub = lane & (tpp - 1);
      for (int c0 = 0; c0 < S.na; c0 += tpc) {
        const int i = c0 + lane / tpp;
        const bool active = i < S.na;
        const int64_t a = S.a0 + (active ? i : 0);
        const double xa = s.x[a], ya = s.y[a], za = s.z[a];
        const double hinv2 = aux.hinv2[a], norm = aux.wnorm[a];
        const int cnt = active ? min(T.nn[a], T.max_nb) : 0;
        const uint16_t* list = T.nbr + a * T.max_nb;
        double t00 = 0, t01 = 0, t02 = 0, t11 = 0, t12 = 0, t22 = 0;
        for (int k = sub; k < cnt; k += tpp) {
          const int64_t b = entry_particle(S, list[k]);
          double dx, dy, dz;
          sep64(g, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
          const double r2 = dx * dx + dy * dy + dz * dz;
          const double w = aux.vol[b] * kernel_w64(fmin(r2 * hinv2, 4.0), norm, sinc_n);
          const double wx = w * dx, wy = w * dy, wz = w * dz;
          t00 += wx * dx;
          t01 += wx * dy;
          t02 += wx * dz;
          t11 += wy * dy;
          t12 += wy * dz;
          t22 += wz * dz;
        }
        t00 = group_sum64(t00, tpp);
        t01 = group_sum64(t01, tpp);
        t02 = group_sum64(t02, tpp);
        t11 = group_sum64(t11, tpp);
        t12 = group_sum64(t12, tpp);
        t22 = group_sum64(t22, tpp);
        if (active && sub == 0) {
          // inverse of the symmetric matrix by cofactors
          const double c00 = t11 * t22 - t12 * t12;
          const double c01 = t02 * t12 - t01 * t22;
          const double c02 = t01 * t12 - t02 * t11;
          const double c11 = t00 * t22 - t02 * t02;
          const double c12 = t01 * t02 - t00 * t12;
          const double c22 = t00 * t11 - t01 * t01;
          const double det = t00 * c00 + t01 * c01 + t02 * c02;
          double tmax = fmax(fmax(fabs(t00), fabs(t01)), fmax(fabs(t02), fabs(t11)));
          tmax = fmax(tmax, fmax(fabs(t12), fabs(t22)));
          double* out = o.iad + 6 * a;
          if (!isfinite(det) || fabs(det) <= 1e-12 * tmax * tmax * tmax) {
            raise_flag(err, SPH_FLAG_SINGULAR_IAD);
            for (int q = 0; q < 6; ++q) out[q] = 0.0;
          } else {
            const double id = 1.0 / det;
            out[0] = c00 * id;
            out[1] = c01 * id;
            out[2] = c02 * id;
            out[3] = c11 * id;
            out[4] = c12 * id;
            out[5] = c22 * id;
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads64) k_momentum64(const Grid* gp, StateView s, OutView o,
                                                           Aux64 aux, Tile64 T, int sinc_n,
                                                           double alpha, uint32_t* err) {
  __shared__ Stencil cells[kWarps64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Stencil& S = cells[warp];
  const Grid g = *gp;
  const uint32_t nw = gridDim.x * kWarps64;
  for (uint32_t cell = blockIdx.x * kWarps64 + warp; cell < g.n_occ; cell += nw) {
    build_stencil_warp(g, T.occ[cell], T.tbl_start, T.tbl_count, S);
    if (S.off[S.ncell] <= kMaxSlots && S.maxpop <= kMaxCellPop) {
      const int tpp = warp_tpp64(S.na);
      const int tpc = 32 / tpp;
      const int sub = lane & (tpp - 1);
      for (int c0 = 0; c0 < S.na; c0 += tpc) {
        const int i = c0 + lane / tpp;
        const bool active = i < S.na;
        const int64_t a = S.a0 + (active ? i : 0);
        const double xa = s.x[a], ya = s.y[a], za = s.z[a];
        const double vxa = s.vx[a], vya = s.vy[a], vza = s.vz[a];
        const double hinv2a = aux.hinv2[a], norma = aux.wnorm[a];
        const double Xa = aux.X[a], ira = aux.inv_rho[a], ca = o.c[a];
        const double* Ca = o.iad + 6 * a;
        const double a00 = Ca[0], a01 = Ca[1], a02 = Ca[2], a11 = Ca[3], a12 = Ca[4], a22 = Ca[5];
        const int cnt = active ? min(T.nn[a], T.max_nb) : 0;
        const uint16_t* list = T.nbr + a * T.max_nb;
        double accx = 0, accy = 0, accz = 0, du = 0;
        for (int k = sub; k < cnt; k += tpp) {
          const int64_t b = entry_particle(S, list[k]);
          double dx, dy, dz;
          sep64(g, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
          const double r2 = dx * dx + dy * dy + dz * dz;
          const double Wa = kernel_w64(fmin(r2 * hinv2a, 4.0), norma, sinc_n);
          const double tb = r2 * aux.hinv2[b];
          const double Wb = tb < 4.0 ? kernel_w64(tb, aux.wnorm[b], sinc_n) : 0.0;
          // C_a d and C_b d, d = x_b - x_a
          const double Cadx = a00 * dx + a01 * dy + a02 * dz;
          const double Cady = a01 * dx + a11 * dy + a12 * dz;
          const double Cadz = a02 * dx + a12 * dy + a22 * dz;
          const double* Cb = o.iad + 6 * b;
          const double b00 = Cb[0], b01 = Cb[1], b02 = Cb[2], b11 = Cb[3], b12 = Cb[4],
                       b22 = Cb[5];
          const double Cbdx = b00 * dx + b01 * dy + b02 * dz;
          const double Cbdy = b01 * dx + b11 * dy + b12 * dz;
          const double Cbdz = b02 * dx + b12 * dy + b22 * dz;
          const double vabx = vxa - s.vx[b], vaby = vya - s.vy[b], vabz = vza - s.vz[b];
          const double xv = -(dx * vabx + dy * vaby + dz * vabz);  // x_ab . v_ab
          const double irb = aux.inv_rho[b];
          double Pi = 0.0;
          if (xv < 0.0) {
            const double w = xv * rsqrt(r2);
            const double vsig = ca + o.c[b] - 3.0 * w;
            Pi = -0.5 * alpha * vsig * w;
          }
          const double mb = s.m[b];
          const double fa = mb * Wa * (Xa + 0.5 * Pi * ira);
          const double fb = mb * Wb * (aux.X[b] + 0.5 * Pi * irb);
          accx -= fa * Cadx + fb * Cbdx;
          accy -= fa * Cady + fb * Cbdy;
          accz -= fa * Cadz + fb * Cbdz;
          const double vCa = vabx * Cadx + vaby * Cady + vabz * Cadz;
          const double vCb = vabx * Cbdx + vaby * Cbdy + vabz * Cbdz;
          du += mb * (Wa * (Xa + 0.25 * Pi * ira) * vCa + 0.25 * Pi * irb * Wb * vCb);
        }
        accx = group_sum64(accx, tpp);
        accy = group_sum64(accy, tpp);
        accz = group_sum64(accz, tpp);
        du = group_sum64(du, tpp);
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
}

inline Aux64 aux_of(sph_ctx* ctx) {
  Aux64 a;
  a.vol = ctx->vol;
  a.X = ctx->X;
  a.inv_rho = ctx->inv_rho;
  a.hinv2 = ctx->vol + 3 * ctx->n_max;
  a.wnorm = ctx->vol + 4 * ctx->n_max;
  return a;
}

inline Tile64 tile64_of(sph_ctx* ctx) {
  Tile64 t;
  t.occ = ctx->occ;
  t.tbl_start = ctx->tbl_start;
  t.tbl_count = ctx->tbl_count;
  t.nn = ctx->nn;
  t.nbr = ctx->nbr;
  t.max_nb = ctx->prm.max_nb;
  return t;
}

template <typename K>
int grid64(K kernel, int sm) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads64, 0);
  return (per_sm > 0 ? per_sm : 1) * sm;
}

int g_blocks64[3] = {0, 0, 0};

}  // namespace

void launch_density_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st) {
  (void)n;
  if (!g_blocks64[0]) g_blocks64[0] = grid64(k_density64, ctx->sm_count);
  k_density64<<<g_blocks64[0], kThreads64, 0, st>>>(ctx->grid, s, o, aux_of(ctx), tile64_of(ctx),
                                                    ctx->Bn, (int)ctx->prm.sinc_n,
                                                    ctx->prm.gamma, ctx->err);
  ctx->launches += 1;
}

void launch_iad_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                    cudaStream_t st) {
  (void)n;
  if (!g_blocks64[1]) g_blocks64[1] = grid64(k_iad64, ctx->sm_count);
  k_iad64<<<g_blocks64[1], kThreads64, 0, st>>>(ctx->grid, s, o, aux_of(ctx), tile64_of(ctx),
                                                (int)ctx->prm.sinc_n, ctx->err);
  ctx->launches += 1;
}

void launch_momentum_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st) {
  (void)n;
  if (!g_blocks64[2]) g_blocks64[2] = grid64(k_momentum64, ctx->sm_count);
  k_momentum64<<<g_blocks64[2], kThreads64, 0, st>>>(ctx->grid, s, o, aux_of(ctx),
                                                     tile64_of(ctx), (int)ctx->prm.sinc_n,
                                                     ctx->prm.alpha, ctx->err);
  ctx->launches += 1;
}

}  // namespace sph
