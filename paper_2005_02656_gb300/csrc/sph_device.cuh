// Device helpers shared by the kernels: the sinc kernel of Eq. 6 evaluated by
// a truncated Taylor series, the FP64 neighbour criterion, error flags and
// warp/block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Sinc kernel (section 4.1, Eq. 6): W(v, h) = B_n / h^3 * S(v)^n with
// S(v) = sin(pi v / 2) / (pi v / 2).  S is even in v, so it is evaluated as a
// polynomial in t = v^2 (no square root): the Maclaurin series of sin(x)/x,
//   S = sum_k (-1)^k x^(2k) / (2k+1)!,  x^2 = (pi/2)^2 t,
// truncated where the next term is below the working precision on t in [0, 4]
// (v in [0, 2]): 15 terms in FP64 (next term < 1.1e-19); 7 in FP32, where the
// truncation changes S^6 by at most 1.9e-9 while FP32 Horner rounding alone
// moves it by up to 1.8e-7 (both relative to S(0)^6 = 1).
// Coefficients are computed at compile time from their definition.
// ---------------------------------------------------------------------------
constexpr double kHalfPi2 = 2.4674011002723396547;  // (pi/2)^2

constexpr double sinc_coef(int k) {
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c *= -kHalfPi2 / ((2.0 * i) * (2.0 * i + 1.0));
  return c;
}

template <int K>
struct SincCoefs {
  double c[K];
  constexpr SincCoefs() : c() {
    for (int k = 0; k < K; ++k) c[k] = sinc_coef(k);
  }
};

constexpr int kSincTerms64 = 15;
constexpr int kSincTerms32 = 7;

__device__ __forceinline__ double sinc_poly64(double t) {
  constexpr SincCoefs<kSincTerms64> C{};
  double s = C.c[kSincTerms64 - 1];
#pragma unroll
  for (int k = kSincTerms64 - 2; k >= 0; --k) s = fma(s, t, C.c[k]);
  return s;
}

// S(t) and dS/dt of the FP64 series (Horner on both).
__device__ __forceinline__ void sinc_poly64_d(double t, double& S, double& dS) {
  constexpr SincCoefs<kSincTerms64> C{};
  double s = C.c[kSincTerms64 - 1];
  double d = (kSincTerms64 - 1) * C.c[kSincTerms64 - 1];
#pragma unroll
  for (int k = kSincTerms64 - 2; k >= 0; --k) {
    s = fma(s, t, C.c[k]);
    if (k >= 1) d = fma(d, t, k * C.c[k]);
  }
  S = s;
  dS = d;
}

__device__ __forceinline__ float sinc_poly32(float t) {
  constexpr SincCoefs<kSincTerms32> C{};
  float s = (float)C.c[kSincTerms32 - 1];
#pragma unroll
  for (int k = kSincTerms32 - 2; k >= 0; --k) s = fmaf(s, t, (float)C.c[k]);
  return s;
}

template <typename T>
__device__ __forceinline__ T ipow(T s, int n) {
  if (n == 6) {
    T s2 = s * s;
    return s2 * s2 * s2;
  }
  if (n <= 0) return T(1);
  T r = s;
  for (int i = 1; i < n; ++i) r *= s;
  return r;
}

// S(t), dS/dt and d2S/dt2 of the FP64 series.
__device__ __forceinline__ void sinc_poly64_d2(double t, double& S, double& dS, double& d2S) {
  constexpr SincCoefs<kSincTerms64> C{};
  double s = C.c[kSincTerms64 - 1];
  double d = (kSincTerms64 - 1) * C.c[kSincTerms64 - 1];
  double e = (kSincTerms64 - 1) * (kSincTerms64 - 2) * C.c[kSincTerms64 - 1];
#pragma unroll
  for (int k = kSincTerms64 - 2; k >= 0; --k) {
    s = fma(s, t, C.c[k]);
    if (k >= 1) d = fma(d, t, k * C.c[k]);
    if (k >= 2) e = fma(e, t, k * (k - 1) * C.c[k]);
  }
  S = s;
  dS = d;
  d2S = e;
}

// S(t) and dS/dt of the FP32 series.
__device__ __forceinline__ void sinc_poly32_d(float t, float& S, float& dS) {
  constexpr SincCoefs<kSincTerms32> C{};
  float s = (float)C.c[kSincTerms32 - 1];
  float d = (float)((kSincTerms32 - 1) * C.c[kSincTerms32 - 1]);
#pragma unroll
  for (int k = kSincTerms32 - 2; k >= 0; --k) {
    s = fmaf(s, t, (float)C.c[k]);
    if (k >= 1) d = fmaf(d, t, (float)(k * C.c[k]));
  }
  S = s;
  dS = d;
}

// W and dW/dt for t = v^2 (FP64); t is clamped at 4, where S = 0.
__device__ __forceinline__ void kernel_w64_d(double t, double norm, int n, double& W,
                                             double& dWdt) {
  t = fmin(t, 4.0);
  double S, dS;
  sinc_poly64_d(t, S, dS);
  const double Sn1 = ipow(S, n - 1);
  W = norm * Sn1 * S;
  dWdt = norm * n * Sn1 * dS;
}

// Tabulated kernel (SPH_KERNEL_TABLE): entry i holds (T_i, T_{i+1} - T_i),
// T_i = S(v_i)^n at v_i = 2 i / (N - 1); linear interpolation in v = sqrt(t).
__device__ __forceinline__ double kernel_w64_tab(double t, double norm, const double2* tab) {
  const double q = sqrt(fmin(t, 4.0)) * (0.5 * (kKernelTableN - 1));
  int i = (int)q;
  if (i > kKernelTableN - 2) i = kKernelTableN - 2;
  const double2 e = tab[i];
  return norm * (e.x + e.y * (q - (double)i));
}
__device__ __forceinline__ float kernel_w32_tab(float t, float norm, const float2* tab) {
  const float q = sqrtf(fminf(t, 4.0f)) * (0.5f * (kKernelTableN - 1));
  int i = (int)q;
  if (i > kKernelTableN - 2) i = kKernelTableN - 2;
  const float2 e = tab[i];
  return norm * fmaf(e.y, q - (float)i, e.x);
}

// dW/dt + t d2W/dt2 (FP64): the t-derivative of t dW/dt, the pair term of the
// grad-h sum's derivative; t is clamped at 4.
__device__ __forceinline__ double kernel_tdw_dt64(double t, double norm, int n) {
  t = fmin(t, 4.0);
  double S, dS, d2S;
  sinc_poly64_d2(t, S, dS, d2S);
  const double Sn1 = ipow(S, n - 1);
  const double Sn2 = n >= 2 ? ipow(S, n - 2) : 0.0;  // multiplied by n - 1 = 0 when n = 1
  const double dW = norm * n * Sn1 * dS;
  const double d2W = norm * n * ((n - 1) * Sn2 * dS * dS + Sn1 * d2S);
  return dW + t * d2W;
}

// W for t = v^2 < 4 (caller guarantees the neighbour criterion), norm = B_n/h^3.
__device__ __forceinline__ double kernel_w64(double t, double norm, int n) {
  return norm * ipow(sinc_poly64(t), n);
}
// t dW/dt (FP32), for the grad-h sum: v dW/dv = 2 t dW/dt.
__device__ __forceinline__ float kernel_tdw32(float t, float norm, int n) {
  t = fminf(t, 4.0f);
  float S, dS;
  sinc_poly32_d(t, S, dS);
  return norm * (float)n * ipow(S, n - 1) * dS * t;
}
__device__ __forceinline__ float kernel_w32(float t, float norm, int n) {
  // t can exceed 4 by rounding for pairs on the support edge; clamp so that the
  // truncated series does not grow there (S(2) = 0).
  t = fminf(t, 4.0f);
  return norm * ipow(sinc_poly32(t), n);
}

// kernel_w32 for two arguments at once (W_a and W_b of one pair): the clamp,
// the series and the powers in paired FP32, each component rounded exactly as
// the scalar kernel_w32 (the integer power for n = 6 as (s^2 s^2) s^2).
__device__ __forceinline__ float2 kernel_w32x2(float2 t, float2 norm, int n) {
  t = make_float2(fminf(t.x, 4.0f), fminf(t.y, 4.0f));
  constexpr SincCoefs<kSincTerms32> C{};
  float2 s = make_float2((float)C.c[kSincTerms32 - 1], (float)C.c[kSincTerms32 - 1]);
#pragma unroll
  for (int k = kSincTerms32 - 2; k >= 0; --k)
    s = __ffma2_rn(s, t, make_float2((float)C.c[k], (float)C.c[k]));
  float2 p;
  if (n == 6) {
    const float2 s2 = __fmul2_rn(s, s);
    p = __fmul2_rn(__fmul2_rn(s2, s2), s2);
  } else {
    p = make_float2(ipow(s.x, n), ipow(s.y, n));
  }
  return __fmul2_rn(norm, p);
}

// The kernel of the context's mode: the series, or the table when tab != NULL.
__device__ __forceinline__ double kw64(double t, double norm, int n, const double2* tab) {
  return tab ? kernel_w64_tab(t, norm, tab) : kernel_w64(t, norm, n);
}
__device__ __forceinline__ float kw32(float t, float norm, int n, const float2* tab) {
  return tab ? kernel_w32_tab(t, norm, tab) : kernel_w32(t, norm, n);
}
__device__ __forceinline__ float2 kw32x2(float2 t, float2 norm, int n, const float2* tab) {
  return tab ? make_float2(kernel_w32_tab(t.x, norm.x, tab), kernel_w32_tab(t.y, norm.y, tab))
             : kernel_w32x2(t, norm, n);
}

// ---------------------------------------------------------------------------
// Minimum-image component b - a on one axis (the reading of section 4.1's
// pair separation on periodic axes) and the FP64 neighbour criterion
// r^2 < (2 h_a)^2 with r^2 = (dx*dx + dy*dy) + dz*dz, evaluated with
// explicitly rounded operations so no multiply-add is fused.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double d, double L, double halfL, int periodic) {
  if (periodic) {
    if (d > halfL)
      d = __dsub_rn(d, L);
    else if (d < -halfL)
      d = __dadd_rn(d, L);
  }
  return d;
}

__device__ __forceinline__ bool exact_neighbor(const Grid& g, double xa, double ya, double za,
                                               double ha, double xb, double yb, double zb) {
  double dx = min_image(__dsub_rn(xb, xa), g.Lbox[0], g.halfL[0], g.periodic[0]);
  double dy = min_image(__dsub_rn(yb, ya), g.Lbox[1], g.halfL[1], g.periodic[1]);
  double dz = min_image(__dsub_rn(zb, za), g.Lbox[2], g.halfL[2], g.periodic[2]);
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  double two_h = __dmul_rn(2.0, ha);
  return r2 < __dmul_rn(two_h, two_h);
}

__device__ __forceinline__ void raise_flag(uint32_t* err, uint32_t f) { atomicOr(err, f); }

// Packed cell coordinates: 10 bits per axis.
__device__ __forceinline__ int32_t pack_cell(int ix, int iy, int iz) {
  return ix | (iy << 10) | (iz << 20);
}
__device__ __forceinline__ void unpack_cell(int32_t c, int& ix, int& iy, int& iz) {
  ix = c & 1023;
  iy = (c >> 10) & 1023;
  iz = (c >> 20) & 1023;
}

// FP32 separation b - a along one axis from cell-relative offsets:
// (off_b - off_a) + (cell_b - cell_a) * cs, with the cell difference taken
// modulo the period and a final FP32 minimum image for grids of < 3 cells.
__device__ __forceinline__ float sep32(float ob, float oa, int cb, int ca, const Grid& g, int ax) {
  int dc = cb - ca;
  if (g.periodic[ax]) {
    int nc = g.nc[ax];
    if (dc > nc / 2)
      dc -= nc;
    else if (dc < -(nc / 2))
      dc += nc;
  }
  float d = fmaf((float)dc, g.cs32[ax], ob - oa);
  if (g.periodic[ax]) {
    if (d > g.halfL32[ax])
      d -= g.L32[ax];
    else if (d < -g.halfL32[ax])
      d += g.L32[ax];
  }
  return d;
}

// Morton code of a cell: bit i of ix at 3i, iy at 3i+1, iz at 3i+2.
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// --- ordered integer keys of doubles ---
// a < b <=> okey(a) < okey(b) for all non-NaN a, b, with okey(-0.0) =
// okey(+0.0) = 0, so comparisons and min/max of doubles can run on the integer
// pipes (FP64 runs at 1/64 of the FP32 rate on this part).  NaN maps to
// if_nan, which the caller picks so that NaN acts as in the FP comparison.
constexpr long long kKeyInf = 0x7ff0000000000000LL;  // okey(+inf)
__device__ __forceinline__ long long okey(double v, long long if_nan) {
  const long long b = __double_as_longlong(v);
  const long long mag = b & 0x7fffffffffffffffLL;
  return mag > kKeyInf ? if_nan : (b < 0 ? -mag : mag);
}
__device__ __forceinline__ double from_okey(long long k) {
  return __longlong_as_double(k < 0 ? (-k | (long long)0x8000000000000000ULL) : k);
}

// Double to float rounded to nearest even, by integer arithmetic when the
// result is a normal float (FP64 conversions run on the FP64 pipe, at 1/64 of
// the FP32 rate on this part); zero, float-subnormal, overflowing and NaN
// inputs take the FP64 conversion.  Equal to (float)d for every d.
__device__ __forceinline__ float f32_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u >= 254u) return (float)d;  // float exponent field outside [1, 254]
  unsigned f = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;  // the 29 bits dropped
  f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;  // carries into
  return __int_as_float(f | (hi & 0x80000000u));                             // the exponent
}

// --- reductions ---
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sph
