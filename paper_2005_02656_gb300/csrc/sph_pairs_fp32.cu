// FP32-mixed pair sums (density + EOS, IAD, momentum/energy).  Separations
// come from FP32 offsets to the cell origin plus the cell difference times the
// cell side (sph_device.cuh: sep32), so no FP64 operation is issued per pair;
// kernel values and the sums are FP32.  Results are also written to the
// caller's FP64 output arrays.  Positions, the time step and the update stay
// FP64 (sph_update.cu).
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

struct F32 {
  const float4* pos;  // offset x, y, z, h
  const int32_t* cell;
  const float4* vel;  // vx, vy, vz, m
  float4* q;          // 1/h^2, B_n/h^3, m/rho, 1/rho
  float2* xc;         // P/rho^2, c
  float4* cA;         // C00 C01 C02 C11
  float4* cB;         // C12 C22 P/rho^2 c
};

__device__ __forceinline__ void sep_f32(const Grid& g, float4 pa, int ca, float4 pb, int cb,
                                        float& dx, float& dy, float& dz) {
  int ax, ay, az, bx, by, bz;
  unpack_cell(ca, ax, ay, az);
  unpack_cell(cb, bx, by, bz);
  dx = sep32(pb.x, pa.x, bx, ax, g, 0);
  dy = sep32(pb.y, pa.y, by, ay, g, 1);
  dz = sep32(pb.z, pa.z, bz, az, g, 2);
}

__global__ void __launch_bounds__(256) k_density32(const Grid* gp, F32 f, OutView o,
                                                   const double* u, const int32_t* nn,
                                                   const int32_t* nbr, int64_t stride, int64_t n,
                                                   int max_nb, float Bn, int sinc_n, double gamma,
                                                   uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const float4 pa = f.pos[a];
    const int ca = f.cell[a];
    const float hinv2 = 1.0f / (pa.w * pa.w);
    const float norm = Bn * hinv2 / pa.w;
    const float ma = f.vel[a].w;
    float rho = ma * norm;
    int cnt = nn[a];
    cnt = cnt < max_nb ? cnt : max_nb;
    for (int k = 0; k < cnt; ++k) {
      const int64_t b = nbr[(int64_t)k * stride + a];
      float dx, dy, dz;
      sep_f32(g, pa, ca, f.pos[b], f.cell[b], dx, dy, dz);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      rho += f.vel[b].w * kernel_w32(r2 * hinv2, norm, sinc_n);
    }
    // EOS in FP64 on the FP32 density
    const double rho64 = (double)rho;
    const double p = (gamma - 1.0) * rho64 * u[a];
    const double c = sqrt(gamma * p / rho64);
    o.rho[a] = rho64;
    o.p[a] = p;
    o.c[a] = c;
    const float inv_rho = 1.0f / rho;
    f.q[a] = make_float4(hinv2, norm, ma * inv_rho, inv_rho);
    f.xc[a] = make_float2((float)(p / (rho64 * rho64)), (float)c);
    if (!isfinite(rho64) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
  }
}

__global__ void __launch_bounds__(256) k_iad32(const Grid* gp, F32 f, OutView o, const int32_t* nn,
                                               const int32_t* nbr, int64_t stride, int64_t n,
                                               int max_nb, int sinc_n, uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const float4 pa = f.pos[a];
    const int ca = f.cell[a];
    const float4 qa = f.q[a];
    const float inv_h = 1.0f / pa.w;
    float t00 = 0, t01 = 0, t02 = 0, t11 = 0, t12 = 0, t22 = 0;
    int cnt = nn[a];
    cnt = cnt < max_nb ? cnt : max_nb;
    for (int k = 0; k < cnt; ++k) {
      const int64_t b = nbr[(int64_t)k * stride + a];
      float dx, dy, dz;
      sep_f32(g, pa, ca, f.pos[b], f.cell[b], dx, dy, dz);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      // scaled separation d / h_a keeps tau of order one in FP32
      dx *= inv_h;
      dy *= inv_h;
      dz *= inv_h;
      const float w = f.q[b].z * kernel_w32(r2 * qa.x, qa.y, sinc_n);
      const float wx = w * dx, wy = w * dy, wz = w * dz;
      t00 = fmaf(wx, dx, t00);
      t01 = fmaf(wx, dy, t01);
      t02 = fmaf(wx, dz, t02);
      t11 = fmaf(wy, dy, t11);
      t12 = fmaf(wy, dz, t12);
      t22 = fmaf(wz, dz, t22);
    }
    const float c00 = t11 * t22 - t12 * t12;
    const float c01 = t02 * t12 - t01 * t22;
    const float c02 = t01 * t12 - t02 * t11;
    const float c11 = t00 * t22 - t02 * t02;
    const float c12 = t01 * t02 - t00 * t12;
    const float c22 = t00 * t11 - t01 * t01;
    const float det = t00 * c00 + t01 * c01 + t02 * c02;
    float tmax = fmaxf(fmaxf(fabsf(t00), fabsf(t01)), fmaxf(fabsf(t02), fabsf(t11)));
    tmax = fmaxf(tmax, fmaxf(fabsf(t12), fabsf(t22)));
    float C[6];
    if (!isfinite(det) || fabsf(det) <= 1e-6f * tmax * tmax * tmax) {
      raise_flag(err, SPH_FLAG_SINGULAR_IAD);
      for (int j = 0; j < 6; ++j) C[j] = 0.0f;
    } else {
      const float s = qa.x / det;  // undo the 1/h_a scaling: C = tau_scaled^{-1} / h_a^2
      C[0] = c00 * s;
      C[1] = c01 * s;
      C[2] = c02 * s;
      C[3] = c11 * s;
      C[4] = c12 * s;
      C[5] = c22 * s;
    }
    const float2 xc = f.xc[a];
    f.cA[a] = make_float4(C[0], C[1], C[2], C[3]);
    f.cB[a] = make_float4(C[4], C[5], xc.x, xc.y);
    double* out = o.iad + 6 * a;
    for (int j = 0; j < 6; ++j) out[j] = (double)C[j];
  }
}

__global__ void __launch_bounds__(256) k_momentum32(const Grid* gp, F32 f, OutView o,
                                                    const int32_t* nn, const int32_t* nbr,
                                                    int64_t stride, int64_t n, int max_nb,
                                                    int sinc_n, float alpha, uint32_t* err) {
  const Grid g = *gp;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const float4 pa = f.pos[a];
    const int ca = f.cell[a];
    const float4 qa = f.q[a];
    const float4 va = f.vel[a];
    const float4 Aa = f.cA[a], Ba = f.cB[a];
    const float a00 = Aa.x, a01 = Aa.y, a02 = Aa.z, a11 = Aa.w, a12 = Ba.x, a22 = Ba.y;
    const float Xa = Ba.z, csa = Ba.w, ira = qa.w;
    float accx = 0, accy = 0, accz = 0, du = 0;
    int cnt = nn[a];
    cnt = cnt < max_nb ? cnt : max_nb;
    for (int k = 0; k < cnt; ++k) {
      const int64_t b = nbr[(int64_t)k * stride + a];
      float dx, dy, dz;
      sep_f32(g, pa, ca, f.pos[b], f.cell[b], dx, dy, dz);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const float4 qb = f.q[b];
      const float Wa = kernel_w32(r2 * qa.x, qa.y, sinc_n);
      const float tb = r2 * qb.x;
      const float Wb = tb < 4.0f ? kernel_w32(tb, qb.y, sinc_n) : 0.0f;
      const float Cadx = a00 * dx + a01 * dy + a02 * dz;
      const float Cady = a01 * dx + a11 * dy + a12 * dz;
      const float Cadz = a02 * dx + a12 * dy + a22 * dz;
      const float4 Ab = f.cA[b], Bb = f.cB[b];
      const float Cbdx = Ab.x * dx + Ab.y * dy + Ab.z * dz;
      const float Cbdy = Ab.y * dx + Ab.w * dy + Bb.x * dz;
      const float Cbdz = Ab.z * dx + Bb.x * dy + Bb.y * dz;
      const float4 vb = f.vel[b];
      const float vabx = va.x - vb.x, vaby = va.y - vb.y, vabz = va.z - vb.z;
      const float xv = -(dx * vabx + dy * vaby + dz * vabz);
      const float irb = qb.w;
      float Pi = 0.0f;
      if (xv < 0.0f) {
        const float w = xv * rsqrtf(r2);
        const float vsig = csa + Bb.w - 3.0f * w;
        Pi = -0.5f * alpha * vsig * w;
      }
      const float mb = vb.w;
      const float fa = mb * Wa * (Xa + 0.5f * Pi * ira);
      const float fb = mb * Wb * (Bb.z + 0.5f * Pi * irb);
      accx -= fa * Cadx + fb * Cbdx;
      accy -= fa * Cady + fb * Cbdy;
      accz -= fa * Cadz + fb * Cbdz;
      const float vCa = vabx * Cadx + vaby * Cady + vabz * Cadz;
      const float vCb = vabx * Cbdx + vaby * Cbdy + vabz * Cbdz;
      du += mb * (Wa * (Xa + 0.25f * Pi * ira) * vCa + 0.25f * Pi * irb * Wb * vCb);
    }
    o.ax[a] = accx;
    o.ay[a] = accy;
    o.az[a] = accz;
    o.du[a] = du;
    if (!isfinite(accx) || !isfinite(accy) || !isfinite(accz) || !isfinite(du))
      raise_flag(err, SPH_FLAG_NONFINITE);
  }
}

inline int blocks_for(int64_t n, int sm) {
  int64_t b = (n + 255) / 256;
  int64_t cap = (int64_t)sm * 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

inline F32 f32_of(sph_ctx* ctx) {
  F32 f;
  f.pos = ctx->pos32;
  f.cell = ctx->cell3;
  f.vel = ctx->vel32;
  f.q = ctx->q32;
  f.xc = ctx->xc32;
  f.cA = ctx->cA32;
  f.cB = ctx->cB32;
  return f;
}

}  // namespace

void launch_density_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st) {
  k_density32<<<blocks_for(n, ctx->sm_count), 256, 0, st>>>(
      ctx->grid, f32_of(ctx), o, s.u, ctx->nn, ctx->nbr, ctx->n_max, n, ctx->prm.max_nb,
      (float)ctx->Bn, (int)ctx->prm.sinc_n, ctx->prm.gamma, ctx->err);
  ctx->launches += 1;
}

void launch_iad_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                    cudaStream_t st) {
  (void)s;
  k_iad32<<<blocks_for(n, ctx->sm_count), 256, 0, st>>>(ctx->grid, f32_of(ctx), o, ctx->nn,
                                                        ctx->nbr, ctx->n_max, n, ctx->prm.max_nb,
                                                        (int)ctx->prm.sinc_n, ctx->err);
  ctx->launches += 1;
}

void launch_momentum_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st) {
  (void)s;
  k_momentum32<<<blocks_for(n, ctx->sm_count), 256, 0, st>>>(
      ctx->grid, f32_of(ctx), o, ctx->nn, ctx->nbr, ctx->n_max, n, ctx->prm.max_nb,
      (int)ctx->prm.sinc_n, (float)ctx->prm.alpha, ctx->err);
  ctx->launches += 1;
}

}  // namespace sph
