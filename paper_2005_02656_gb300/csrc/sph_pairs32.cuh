// Per-particle bodies of the FP32-mixed pair sums (density + EOS, IAD,
// momentum/energy), shared by the single-box kernels (sph_pairs_fp32.cu) and
// the ensemble's persistent kernel (sph_ensemble.cu).  Each function computes
// target particle a of the box described by the Grid g.
//
// Each neighbour-list entry (sph_tile.cuh) carries the neighbour's index and
// the shift of its cell relative to the target's cell, so a pair separation
// is (offset_b + shift) - offset_a in FP32 with no FP64 operation and no table
// lookup.  Lists are read four entries per 16-byte load; neighbour data is
// gathered through L1/L2 from packed records:
//   rec_d (density)  = (offset x, y, z, m)                       16 B
//   rec_i (IAD)      = (offset x, y, z, m/rho)                   16 B
//   rec_m (momentum) = (offset, 1/h^2), (v, m), (B_n/h^3, P/rho^2, c, 1/rho),
//                      (C00 C01 C02 C11), (C12 C22 - -)          80 B
#pragma once

#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

namespace sph {
namespace pairs32 {

struct F32 {
  const float4* pos;    // offset in own cell x, y, z, h
  const float4* rec_d;  // offset x, y, z, m
  float4* rec_i;        // offset x, y, z, m/rho
  float4* rec_m;        // 5 float4 per particle
  const float2* ktab;   // SPH_KERNEL_TABLE values, NULL for the exact kernel
};

struct Lists {
  const int32_t* nn;
  const uint32_t* nbr;
  int max_nb;
};

__device__ __forceinline__ float wrap_axis(float d, const Grid& g, int ax) {
  if (d > g.halfL32[ax])
    d -= g.L32[ax];
  else if (d < -g.halfL32[ax])
    d += g.L32[ax];
  return d;
}

// FP32 separation b - a from the neighbour's offset and the entry's shift.
__device__ __forceinline__ void rel(const Grid& g, bool wrap, uint32_t e, float4 rb, float4 pa,
                                    float& dx, float& dy, float& dz) {
  float sx, sy, sz;
  entry_shift(e, g, sx, sy, sz);
  dx = (rb.x + sx) - pa.x;
  dy = (rb.y + sy) - pa.y;
  dz = (rb.z + sz) - pa.z;
  if (wrap) {
    if (g.periodic[0]) dx = wrap_axis(dx, g, 0);
    if (g.periodic[1]) dy = wrap_axis(dy, g, 1);
    if (g.periodic[2]) dz = wrap_axis(dz, g, 2);
  }
}

// Calls body(entry) for the cnt entries of a row, reading 4 per 16-byte load.
template <typename Body>
__device__ __forceinline__ void for_entries(const uint32_t* row, int cnt, Body body) {
  const uint4* r4 = reinterpret_cast<const uint4*>(row);
  int k = 0;
  for (; k + 4 <= cnt; k += 4) {
    const uint4 e = r4[k >> 2];
    body(e.x);
    body(e.y);
    body(e.z);
    body(e.w);
  }
  if (k < cnt) {
    const uint4 e = r4[k >> 2];
    body(e.x);
    if (k + 1 < cnt) body(e.y);
    if (k + 2 < cnt) body(e.z);
  }
}

// The entries of a row owned by sub-lane `sub` of a group of NSUB lanes that
// share one target: entries k = sub, sub + NSUB, ... for NSUB >= 4, 16-byte
// chunks c = sub, sub + NSUB, ... for NSUB = 2.  NSUB = 1 is for_entries
// (every entry, in order).
template <int NSUB, typename Body>
__device__ __forceinline__ void for_entries_part(const uint32_t* row, int cnt, int sub,
                                                 Body body) {
  if (NSUB == 1) {
    for_entries(row, cnt, body);
    return;
  }
  if (NSUB >= 4) {
    // the NSUB lanes of a target read NSUB consecutive entries at a time:
    // neighbours in the same cell, adjacent in memory, so a warp-wide gather
    // touches fewer lines (momentum 6.22 -> 6.11 ms at 8.4M particles)
    for (int k = sub; k < cnt; k += NSUB) body(__ldg(row + k));
    return;
  }
  // two lanes: every other 16-byte group of four entries (measured better
  // than interleaved single entries for two lanes, 6.29 against 7.03 ms)
  const uint4* r4 = reinterpret_cast<const uint4*>(row);
  for (int c = sub; 4 * c < cnt; c += NSUB) {
    const uint4 e = r4[c];
    const int k = 4 * c;
    body(e.x);
    if (k + 1 < cnt) body(e.y);
    if (k + 2 < cnt) body(e.z);
    if (k + 3 < cnt) body(e.w);
  }
}

// Sum over the NSUB lanes of a group (fixed butterfly; all 32 lanes of the
// warp must call it).
template <int NSUB>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = NSUB / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The functions below compute target a with NSUB lanes (NSUB = 1, 2 or 4;
// `sub` is the lane's index in its group, `on` false for lanes past the last
// target).  N > 0 fixes the kernel exponent n at compile time (the caller
// passes sinc_n = N), N = 0 takes sinc_n at run time.  With NSUB > 1 every lane of the warp must call them; lane sub = 0
// writes the results.

// ---------------------------------------------------------------- density --
// Eq. 1 (self term included) and the ideal-gas EOS for particle a; writes the
// FP64 outputs and the IAD / momentum records of a.  With gradh, also the
// grad-h terms Omega_a = -(2 / (3 rho_a)) sum_{b != a} m_b t dW/dt (the form
// of 1 + h/(3 rho) sum m dW/dh for this kernel, t = v^2), folded into the
// record's X = P / (Omega rho^2).
template <int NSUB = 1, int N = 0>
__device__ __forceinline__ void density_one(int64_t a, const Grid& g, const F32& f,
                                            const OutView& o, const double* u, const Lists& L,
                                            float Bn, int sinc_n, double gamma, uint32_t* err,
                                            bool on = true, int sub = 0, bool gradh = false) {
  const bool wrap = g.wrap32 != 0;
  if (N > 0) sinc_n = N;
  float4 pa = make_float4(0.f, 0.f, 0.f, 1.f);
  float hinv2 = 0.f, norm = 0.f, acc = 0.0f, gsum = 0.0f;
  if (on) {
    pa = f.pos[a];
    hinv2 = 1.0f / (pa.w * pa.w);
    norm = Bn * hinv2 / pa.w;
    const int cnt = min(L.nn[a], L.max_nb);
    for_entries_part<NSUB>(L.nbr + a * L.max_nb, cnt, sub, [&](uint32_t e) {
      const float4 rb = f.rec_d[entry_index(e)];
      float dx, dy, dz;
      rel(g, wrap, e, rb, pa, dx, dy, dz);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      acc = fmaf(rb.w, kw32(r2 * hinv2, norm, sinc_n, f.ktab), acc);
      if (gradh) gsum = fmaf(rb.w, kernel_tdw32(r2 * hinv2, norm, sinc_n), gsum);
    });
  }
  acc = group_sum<NSUB>(acc);
  if (gradh) gsum = group_sum<NSUB>(gsum);
  if (!on || sub != 0) return;
  const float ma = f.rec_d[a].w;
  const float rho = fmaf(ma, norm, acc);  // self term: W(0, h_a) = B_n / h_a^3
  const double rho64 = (double)rho;
  const double p = (gamma - 1.0) * rho64 * u[a];
  const double c = sqrt(gamma * p / rho64);
  o.rho[a] = rho64;
  o.p[a] = p;
  o.c[a] = c;
  const float inv_rho = 1.0f / rho;
  f.rec_i[a] = make_float4(pa.x, pa.y, pa.z, ma * inv_rho);
  float4* m = f.rec_m + 5 * a;
  m[0] = make_float4(pa.x, pa.y, pa.z, hinv2);
  double X = p / (rho64 * rho64);
  if (gradh) {
    const double omega = -2.0 * (double)gsum / (3.0 * rho64);
    X /= omega;
    if (o.omega) o.omega[a] = omega;
  }
  m[2] = make_float4(norm, (float)X, (float)c, inv_rho);
  if (!isfinite(rho64) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
}

// -------------------------------------------------------------------- IAD --
// tau_a and C_a = tau_a^{-1} for particle a (each pair weight divided by
// h_a^2, so that the sum tau_a / h_a^2 is of order one in FP32).
template <int NSUB = 1, int N = 0>
__device__ __forceinline__ void iad_one(int64_t a, const Grid& g, const F32& f, const OutView& o,
                                        const Lists& L, int sinc_n, uint32_t* err,
                                        bool on = true, int sub = 0) {
  const bool wrap = g.wrap32 != 0;
  if (N > 0) sinc_n = N;
  float t00 = 0, t01 = 0, t02 = 0, t11 = 0, t12 = 0, t22 = 0;
  float hinv2 = 0.f;
  if (on) {
    const float4 pa = f.pos[a];
    hinv2 = f.rec_m[5 * a].w;
    const float norm = f.rec_m[5 * a + 2].x;
    const int cnt = min(L.nn[a], L.max_nb);
    for_entries_part<NSUB>(L.nbr + a * L.max_nb, cnt, sub, [&](uint32_t e) {
      const float4 rb = f.rec_i[entry_index(e)];
      float dx, dy, dz;
      rel(g, wrap, e, rb, pa, dx, dy, dz);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      // the weight divided by h_a^2 keeps tau / h_a^2 of order one in FP32
      const float w = rb.w * kw32(r2 * hinv2, norm, sinc_n, f.ktab) * hinv2;
      const float wx = w * dx, wy = w * dy, wz = w * dz;
      t00 = fmaf(wx, dx, t00);
      t01 = fmaf(wx, dy, t01);
      t02 = fmaf(wx, dz, t02);
      t11 = fmaf(wy, dy, t11);
      t12 = fmaf(wy, dz, t12);
      t22 = fmaf(wz, dz, t22);
    });
  }
  t00 = group_sum<NSUB>(t00);
  t01 = group_sum<NSUB>(t01);
  t02 = group_sum<NSUB>(t02);
  t11 = group_sum<NSUB>(t11);
  t12 = group_sum<NSUB>(t12);
  t22 = group_sum<NSUB>(t22);
  if (!on || sub != 0) return;
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
    const float sc = hinv2 / det;  // C = tau_scaled^{-1} / h_a^2
    Cm[0] = c00 * sc;
    Cm[1] = c01 * sc;
    Cm[2] = c02 * sc;
    Cm[3] = c11 * sc;
    Cm[4] = c12 * sc;
    Cm[5] = c22 * sc;
  }
  float4* m = f.rec_m + 5 * a;
  m[3] = make_float4(Cm[0], Cm[1], Cm[2], Cm[3]);
  m[4] = make_float4(Cm[4], Cm[5], 0.0f, 0.0f);
  double* out = o.iad + 6 * a;
  for (int q = 0; q < 6; ++q) out[q] = (double)Cm[q];
}

// ------------------------------------------------------- momentum/energy --
// Eqs. 2-5 for particle a with viscosity coefficient alpha.
template <int NSUB = 1, int N = 0>
__device__ __forceinline__ void momentum_one(int64_t a, const Grid& g, const F32& f,
                                             const OutView& o, const Lists& L, int sinc_n,
                                             float alpha, uint32_t* err, bool on = true,
                                             int sub = 0) {
  const bool wrap = g.wrap32 != 0;
  if (N > 0) sinc_n = N;
  float accx = 0, accy = 0, accz = 0, du = 0;
  if (on) {
    const float4* ra = f.rec_m + 5 * a;
    const float4 pa = ra[0];       // offset, 1/h_a^2
    const float4 va = ra[1];       // v, m
    const float4 qa = ra[2];       // B_n/h^3, P/rho^2, c, 1/rho
    const float4 Aa = ra[3], Ba = ra[4];
    const float a00 = Aa.x, a01 = Aa.y, a02 = Aa.z, a11 = Aa.w, a12 = Ba.x, a22 = Ba.y;
    const float Xa = qa.y, csa = qa.z, ira = qa.w;
    const int cnt = min(L.nn[a], L.max_nb);
    for_entries_part<NSUB>(L.nbr + a * L.max_nb, cnt, sub, [&](uint32_t e) {
      // one pair of Eqs. 2-5 (x_ab = -d, d = x_b - x_a)
      const float4* rb = f.rec_m + 5 * (int64_t)entry_index(e);
      const float4 b0 = rb[0];
      float dx, dy, dz;
      rel(g, wrap, e, b0, pa, dx, dy, dz);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const float4 b2 = rb[2];
      // W_a and W_b together in paired FP32, clamped at t = 4 (S = 0)
      const float2 Wab = kw32x2(make_float2(r2 * pa.w, r2 * b0.w), make_float2(qa.x, b2.x),
                                sinc_n, f.ktab);
      const float Wa = Wab.x, Wb = Wab.y;
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
      // hP = Pi / 2 and qP = Pi / 4 (exact: scalings by powers of two)
      const float w = xv * rsqrtf(r2);
      const float vsig = csa + b2.z - 3.0f * w;
      const float hP = xv < 0.0f ? -0.25f * alpha * vsig * w : 0.0f;
      const float qP = 0.5f * hP;
      const float irb = b2.w;
      const float mb = vb.w;
      const float fa = mb * Wa * fmaf(hP, ira, Xa);
      const float fb = mb * Wb * fmaf(hP, irb, b2.y);
      // a -= fa C_a d + fb C_b d as two fused steps
      accx = fmaf(-fb, Cbdx, fmaf(-fa, Cadx, accx));
      accy = fmaf(-fb, Cbdy, fmaf(-fa, Cady, accy));
      accz = fmaf(-fb, Cbdz, fmaf(-fa, Cadz, accz));
      const float vCa = fmaf(vabz, Cadz, fmaf(vaby, Cady, vabx * Cadx));
      const float vCb = fmaf(vabz, Cbdz, fmaf(vaby, Cbdy, vabx * Cbdx));
      du = fmaf(mb, fmaf(Wa * fmaf(qP, ira, Xa), vCa, qP * irb * Wb * vCb), du);
    });
  }
  accx = group_sum<NSUB>(accx);
  accy = group_sum<NSUB>(accy);
  accz = group_sum<NSUB>(accz);
  du = group_sum<NSUB>(du);
  if (!on || sub != 0) return;
  o.ax[a] = accx;
  o.ay[a] = accy;
  o.az[a] = accz;
  o.du[a] = du;
  if (!isfinite(accx) || !isfinite(accy) || !isfinite(accz) || !isfinite(du))
    raise_flag(err, SPH_FLAG_NONFINITE);
}

}  // namespace pairs32
}  // namespace sph
