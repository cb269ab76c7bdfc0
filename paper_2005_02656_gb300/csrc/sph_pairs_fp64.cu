// FP64 pair sums: density + EOS (Eq. 1), the IAD matrix, and momentum/energy
// with artificial viscosity (Eqs. 2-5).  One thread per target particle,
// grid-stride over the sorted particles, walking its neighbour list (entries:
// sph_tile.cuh) and gathering the neighbours' FP64 fields through L1/L2
// (particles are in Morton cell order, so a warp's neighbours share lines).
// Separations are FP64 minimum-image differences of the positions, the image
// taken from the list entry's cell shift (sep64).  On this
// part the FP64 pipe bounds these kernels, so per-pair divisions are hoisted
// into per-particle arrays (m/rho, P/rho^2, 1/rho, 1/h^2, B_n/h^3), and the
// kernel value W_ab(h_a) of each list entry is evaluated once, by the density
// pass, and read back by IAD and momentum (Lists64::w).
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

namespace sph {

namespace {

constexpr int kThreads64 = 128;

struct Aux64 {
  const int32_t* cell3;  // packed cell coordinates of each sorted particle
  double* vol;     // m / rho
  double* X;       // P / rho^2
  double* inv_rho;
  double* hinv2;   // 1 / h^2
  double* wnorm;   // B_n / h^3
  const double2* ktab;  // SPH_KERNEL_TABLE values, NULL for the exact kernel
};

struct Lists64 {
  const int32_t* nn;
  const uint32_t* nbr;
  double* w;  // W_ab(h_a) per entry, same layout as nbr
  int max_nb;
};

// FP64 minimum-image separation x_b - x_a of a list entry.  With at least
// three cells on every periodic axis (Grid::wrap32 == 0) the image is known
// from the entry's cell shift: the neighbour's cell is ca + shift before
// wrapping, and an index below 0 or past the last cell means its image lies
// one period down or up.  That is the same subtraction or addition of the
// period that the minimum-image test would pick for a neighbour (closer than
// 2h < L/2), decided by integer arithmetic instead of six FP64 comparisons
// (the FP64 pipe bounds these kernels).  Otherwise the comparisons decide.
__device__ __forceinline__ void sep64(const Grid& g, const int ca[3], uint32_t e, double xa,
                                      double ya, double za, double xb, double yb, double zb,
                                      double& dx, double& dy, double& dz) {
  dx = xb - xa;
  dy = yb - ya;
  dz = zb - za;
  if (g.wrap32) {
    dx = min_image(dx, g.Lbox[0], g.halfL[0], g.periodic[0]);
    dy = min_image(dy, g.Lbox[1], g.halfL[1], g.periodic[1]);
    dz = min_image(dz, g.Lbox[2], g.halfL[2], g.periodic[2]);
    return;
  }
  const int c = (int)(e >> kIndexBits);
  const int sz = c / 9, sy = (c - 9 * sz) / 3, sx = c - 9 * sz - 3 * sy;
  const int u[3] = {ca[0] + sx - 1, ca[1] + sy - 1, ca[2] + sz - 1};
  double* d[3] = {&dx, &dy, &dz};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (u[ax] < 0)
      *d[ax] = __dsub_rn(*d[ax], g.Lbox[ax]);
    else if (u[ax] >= g.nc[ax])
      *d[ax] = __dadd_rn(*d[ax], g.Lbox[ax]);
  }
}

// GRADH: also the grad-h terms, Omega_a = 1 + h_a/(3 rho_a) sum_b m_b dW/dh_a.
// With dW/dh = -(3 W + v dW/dv) / h and sum_b m_b W = rho_a (self term
// included) this is Omega_a = -(2 / (3 rho_a)) sum_{b != a} m_b t dW/dt,
// t = v^2 (the self term has t = 0); X = P / (Omega rho^2) then carries it
// into Eqs. 2-3.
template <bool GRADH>
__global__ void __launch_bounds__(kThreads64) k_density64(const Grid* gp, StateView s, OutView o,
                                                          Aux64 aux, Lists64 L, int64_t n,
                                                          double Bn, int sinc_n, double gamma,
                                                          uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const double xa = s.x[a], ya = s.y[a], za = s.z[a], ha = s.h[a];
    int cell_a[3];
    unpack_cell(aux.cell3[a], cell_a[0], cell_a[1], cell_a[2]);
    const double hinv2 = 1.0 / (ha * ha);
    const double norm = Bn * hinv2 / ha;
    const int cnt = min(L.nn[a], L.max_nb);
    const uint32_t* list = L.nbr + a * L.max_nb;
    double* wrow = L.w + a * L.max_nb;
    double acc = 0.0, gsum = 0.0;
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = list[k];
      const int64_t b = entry_index(e);
      double dx, dy, dz;
      sep64(g, cell_a, e, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double t = fmin(r2 * hinv2, 4.0);
      if (GRADH) {
        double W, dW;
        kernel_w64_d(t, norm, sinc_n, W, dW);
        acc += s.m[b] * W;
        gsum += s.m[b] * t * dW;
        wrow[k] = W;
      } else {
        const double W = kw64(t, norm, sinc_n, aux.ktab);
        acc += s.m[b] * W;
        wrow[k] = W;
      }
    }
    const double rho = s.m[a] * norm + acc;  // self term: W(0, h_a) = B_n / h_a^3
    const double p = (gamma - 1.0) * rho * s.u[a];
    const double c = sqrt(gamma * p / rho);
    o.rho[a] = rho;
    o.p[a] = p;
    o.c[a] = c;
    const double inv_rho = 1.0 / rho;
    aux.inv_rho[a] = inv_rho;
    aux.vol[a] = s.m[a] * inv_rho;
    if (GRADH) {
      const double omega = -2.0 * gsum * inv_rho / 3.0;
      aux.X[a] = p * inv_rho * inv_rho / omega;
      if (o.omega) o.omega[a] = omega;
    } else {
      aux.X[a] = p * inv_rho * inv_rho;
    }
    aux.hinv2[a] = hinv2;
    aux.wnorm[a] = norm;
    if (!isfinite(rho) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
  }
}

__global__ void __launch_bounds__(kThreads64) k_iad64(const Grid* gp, StateView s, OutView o,
                                                      Aux64 aux, Lists64 L, int64_t n,
                                                      int sinc_n, uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const double xa = s.x[a], ya = s.y[a], za = s.z[a];
    int cell_a[3];
    unpack_cell(aux.cell3[a], cell_a[0], cell_a[1], cell_a[2]);
    const int cnt = min(L.nn[a], L.max_nb);
    const uint32_t* list = L.nbr + a * L.max_nb;
    const double* wrow = L.w + a * L.max_nb;
    double t00 = 0, t01 = 0, t02 = 0, t11 = 0, t12 = 0, t22 = 0;
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = list[k];
      const int64_t b = entry_index(e);
      double dx, dy, dz;
      sep64(g, cell_a, e, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
      const double w = aux.vol[b] * wrow[k];
      const double wx = w * dx, wy = w * dy, wz = w * dz;
      t00 += wx * dx;
      t01 += wx * dy;
      t02 += wx * dz;
      t11 += wy * dy;
      t12 += wy * dz;
      t22 += wz * dz;
    }
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

__global__ void __launch_bounds__(kThreads64) k_momentum64(const Grid* gp, StateView s, OutView o,
                                                           Aux64 aux, Lists64 L, int64_t n,
                                                           int sinc_n, double alpha,
                                                           uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const double xa = s.x[a], ya = s.y[a], za = s.z[a];
    int cell_a[3];
    unpack_cell(aux.cell3[a], cell_a[0], cell_a[1], cell_a[2]);
    const double vxa = s.vx[a], vya = s.vy[a], vza = s.vz[a];
    const double Xa = aux.X[a], ira = aux.inv_rho[a], ca = o.c[a];
    const double* Ca = o.iad + 6 * a;
    const double a00 = Ca[0], a01 = Ca[1], a02 = Ca[2], a11 = Ca[3], a12 = Ca[4], a22 = Ca[5];
    const int cnt = min(L.nn[a], L.max_nb);
    const uint32_t* list = L.nbr + a * L.max_nb;
    const double* wrow = L.w + a * L.max_nb;
    double accx = 0, accy = 0, accz = 0, du = 0;
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = list[k];
      const int64_t b = entry_index(e);
      double dx, dy, dz;
      sep64(g, cell_a, e, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double Wa = wrow[k];
      const double tb = r2 * aux.hinv2[b];
      const double Wb = tb < 4.0 ? kw64(tb, aux.wnorm[b], sinc_n, aux.ktab) : 0.0;
      // C_a d and C_b d, d = x_b - x_a
      const double Cadx = a00 * dx + a01 * dy + a02 * dz;
      const double Cady = a01 * dx + a11 * dy + a12 * dz;
      const double Cadz = a02 * dx + a12 * dy + a22 * dz;
      const double* Cb = o.iad + 6 * b;
      const double b00 = Cb[0], b01 = Cb[1], b02 = Cb[2], b11 = Cb[3], b12 = Cb[4], b22 = Cb[5];
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
    o.ax[a] = accx;
    o.ay[a] = accy;
    o.az[a] = accz;
    o.du[a] = du;
    if (!isfinite(accx) || !isfinite(accy) || !isfinite(accz) || !isfinite(du))
      raise_flag(err, SPH_FLAG_NONFINITE);
  }
}

inline Aux64 aux_of(sph_ctx* ctx) {
  Aux64 a;
  a.cell3 = ctx->cell3;
  a.vol = ctx->vol;
  a.X = ctx->X;
  a.inv_rho = ctx->inv_rho;
  a.hinv2 = ctx->vol + 3 * ctx->n_max;
  a.wnorm = ctx->vol + 4 * ctx->n_max;
  a.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab64 : nullptr;
  return a;
}

inline Lists64 lists64_of(sph_ctx* ctx) {
  Lists64 t;
  t.nn = ctx->nn;
  t.nbr = ctx->nbr;
  t.w = ctx->wcache;
  t.max_nb = ctx->prm.max_nb;
  return t;
}

inline int blocks64(int64_t n, int sm) {
  int64_t b = (n + kThreads64 - 1) / kThreads64;
  const int64_t cap = (int64_t)sm * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_density_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st) {
  auto kern = ctx->prm.gradh ? k_density64<true> : k_density64<false>;
  kern<<<blocks64(n, ctx->sm_count), kThreads64, 0, st>>>(
      ctx->grid, s, o, aux_of(ctx), lists64_of(ctx), n, ctx->Bn, (int)ctx->prm.sinc_n,
      ctx->prm.gamma, ctx->err);
  ctx->launches += 1;
}

void launch_iad_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                    cudaStream_t st) {
  k_iad64<<<blocks64(n, ctx->sm_count), kThreads64, 0, st>>>(
      ctx->grid, s, o, aux_of(ctx), lists64_of(ctx), n, (int)ctx->prm.sinc_n, ctx->err);
  ctx->launches += 1;
}

void launch_momentum_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st) {
  k_momentum64<<<blocks64(n, ctx->sm_count), kThreads64, 0, st>>>(
      ctx->grid, s, o, aux_of(ctx), lists64_of(ctx), n, (int)ctx->prm.sinc_n, ctx->prm.alpha,
      ctx->err);
  ctx->launches += 1;
}

}  // namespace sph
