// Global time step, integrator update and conservation sums, all FP64.
//
// k_timestep  dt_n = min(courant * min_a h_a / c_a, dt_growth * dt_{n-1}),
//             and, when energy_dt > 0, at most energy_dt * min_a u_a / |du_a|
//             over du_a != 0 (the opt-in energy-rate limit, a reading)
//             (section 4.2: the global minimum time step; the paper's
//             MPI_Allreduce becomes a block reduction plus a last-block
//             finalisation, so the result never leaves the device)
// k_update    section 4.1's second-order integrators, read as a variable-step
//             leapfrog for x and v and Adams-Bashforth for u; smoothing length
//             adapted toward the target neighbour count; periodic wrap; block
//             partial sums of momentum, energies, neighbour-count statistics
//             and (when angular_sums is set) angular momentum of the new state
//             (section 4.2: the optional conservation reduction)
// k_diag      the same sums for any state
// Cross-block totals are combined by the last block in a fixed-shape tree, so
// every reduction here is deterministic.
#include <cuda_runtime.h>

#include <climits>

#include "sph_device.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kThreads = 256;
constexpr int kParts = 16;  // doubles per block partial

__device__ __forceinline__ bool block_last(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// Block sum of NV doubles per thread into part[blockIdx.x * kParts + k].
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* part) {
  __shared__ double sh[kThreads / 32][NV];
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int k = 0; k < NV; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int ww = 0; ww < kThreads / 32; ++ww) s += sh[ww][threadIdx.x];
    part[blockIdx.x * kParts + threadIdx.x] = s;
  }
}

// The last block's reduction of the per-block partials part[b * kParts + k]:
// every thread takes the blocks b = tid, tid + blockDim, ... in order, then a
// fixed-shape warp and block tree combines them, so the result does not
// depend on timing.  Reads go to L2 (the partials were written by other
// blocks before their fence and counter increment).  Called by all threads of
// the block; out (shared) receives the NV results.
enum class Op { kSum, kMin, kMax };

__device__ __forceinline__ double op_apply(Op op, double a, double b) {
  return op == Op::kSum ? a + b : (op == Op::kMin ? fmin(a, b) : fmax(a, b));
}

template <int NV>
__device__ void finalize_block(const double* part, int nblocks, const Op (&op)[NV],
                               double* out) {
  __shared__ double sh[kThreads / 32][NV];
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k)
    v[k] = op[k] == Op::kSum ? 0.0 : (op[k] == Op::kMin ? INFINITY : -INFINITY);
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = op_apply(op[k], v[k], __ldcg(part + b * kParts + k));
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] = op_apply(op[k], v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    const int k = threadIdx.x;
    double r = sh[0][k];
    for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) r = op_apply(op[k], r, sh[ww][k]);
    out[k] = r;
  }
  __syncthreads();
}

// FP32 value of a positive double whose exponent lies in [-60, 60], taken from
// its high word by integer arithmetic (no FP64 instruction: FP64 runs at 1/64
// of the FP32 rate on this part).  The 20 mantissa bits of the high word are
// kept and the rest truncated, so the result is in [v (1 - 2^-20), v].  NaN
// for any other input (zero, negative, subnormal, outside the range, NaN).
__device__ __forceinline__ float f32_of_hi(double v) {
  const int hi = __double2hiint(v);
  const unsigned e = ((unsigned)hi >> 20) - (1023u - 60u);  // sign bit set: huge
  return e <= 120u ? __int_as_float((hi - ((1023 - 127) << 20)) << 3) : __int_as_float(0x7fc00000);
}

// Screen of the exact minimum of h/c: q32 approximates the quotient within
// 2^-18 relative (the two truncations above and __fdividef's 2 ulp), so a
// quotient whose q32 exceeds the running minimum's FP32 value by the factor
// 1 + 2^-16 is larger than that minimum and needs no FP64 division.
constexpr float kScreen = 1.0f + 0x1p-16f;

__global__ void __launch_bounds__(kThreads) k_timestep(const double* h, const double* c,
                                                       const double* u, const double* du,
                                                       int64_t n, double courant, double growth,
                                                       double energy_dt, double* dt_io,
                                                       double* diag, double* part,
                                                       unsigned int* counter, uint32_t* err) {
  double mn = INFINITY, mu = INFINITY;
  float lim = INFINITY;  // FP32 screen value of mn
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int kU = 4;  // particles per thread and pass: their loads overlap
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kU * stride) {
    double hv[kU], cv[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int64_t i = i0 + k * stride;
      hv[k] = i < n ? h[i] : 0.0;
      cv[k] = i < n ? c[i] : 1.0;
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      // exact division only where the screen cannot rule the quotient out
      // (NaN screen values: inputs outside the range of f32_of_hi)
      if (i0 + k * stride < n && !(__fdividef(f32_of_hi(hv[k]), f32_of_hi(cv[k])) > lim)) {
        mn = fmin(mn, hv[k] / cv[k]);
        lim = (float)mn * kScreen;
      }
    }
    if (energy_dt > 0.0) {
      for (int k = 0; k < kU; ++k) {
        const int64_t i = i0 + k * stride;
        if (i < n && du[i] != 0.0) mu = fmin(mu, u[i] / fabs(du[i]));
      }
    }
  }
  mn = warp_min(mn);
  mu = warp_min(mu);
  __shared__ double sh[2][kThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = mn;
    sh[1][threadIdx.x >> 5] = mu;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) {
      mn = fmin(mn, sh[0][w]);
      mu = fmin(mu, sh[1][w]);
    }
    part[blockIdx.x * kParts] = mn;
    part[blockIdx.x * kParts + 1] = mu;
  }
  if (!block_last(counter)) return;
  __threadfence();
  __shared__ double res[2];
  const Op ops[2] = {Op::kMin, Op::kMin};
  finalize_block<2>(part, gridDim.x, ops, res);
  if (threadIdx.x == 0) {
    const double m = res[0];
    const double prev = *dt_io;
    double dt = courant * m;
    if (energy_dt > 0.0) dt = fmin(dt, energy_dt * res[1]);  // no du != 0: res[1] = inf
    if (prev > 0.0) dt = fmin(dt, growth * prev);
    if (!isfinite(dt) || !(dt > 0.0)) raise_flag(err, SPH_FLAG_NONFINITE);
    diag[12] = prev;
    diag[8] = dt;
    *dt_io = dt;
    *counter = 0;
  }
}

// h factor of the rule h <- h (1 + (n_t / max(nn, 1))^(1/3)) / 2: the product
// h * [0.5 (1 + c)] equals (h * 0.5) * (1 + c) bit for bit (scaling by 0.5 is
// exact), so the table changes no result.
__device__ __forceinline__ double hfac_of(int ng, int cnt) {
  const int kk = cnt > 1 ? cnt : 1;
  return 0.5 * (1.0 + cbrt((double)ng / (double)kk));
}

__global__ void k_hfac_table(double* tab, int ng) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kHTab; k += gridDim.x * blockDim.x)
    tab[k] = hfac_of(ng, k);
}

// kAngular: also sum the angular momentum m (x x v) of the new state (12 more
// FP64 operations per particle; momentum and energy are always summed)
template <bool kAngular>
__global__ void __launch_bounds__(kThreads) k_update(StateView s, OutView o, StateView d,
                                                     const int32_t* nn, int64_t n,
                                                     sph_params prm, const double* hfac,
                                                     double* diag, double* part,
                                                     unsigned int* counter,
                                                     unsigned long long* stats) {
  const double dt = diag[8], dt_prev = diag[12];
  const double delta = 0.5 * (dt + dt_prev);
  const double q = dt_prev > 0.0 ? dt / (2.0 * dt_prev) : 0.0;
  double acc[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  // periodic wrap tests on ordered integer keys of the box corners (a NaN
  // position takes the key of box_lo: no wrap, as in the FP comparison)
  long long klo[3], khi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    klo[k] = okey(prm.box_lo[k], 0);
    khi[k] = okey(prm.box_hi[k], 0);
  }
  // neighbour-count statistics in integer arithmetic (FP64 runs at 1/64 of the
  // FP32 rate on this part); converted once per thread below
  long long csum = 0;
  int cmin = INT_MAX, cmax = INT_MIN;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double a3[3] = {o.ax[p], o.ay[p], o.az[p]};
    const double x3[3] = {s.x[p], s.y[p], s.z[p]};
    const double vh3[3] = {s.vxh[p], s.vyh[p], s.vzh[p]};
    double xn[3], vn[3], vhn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      vhn[k] = vh3[k] + a3[k] * delta;
      double xk = x3[k] + dt * vhn[k];
      if (prm.periodic[k]) {
        const double L = prm.box_hi[k] - prm.box_lo[k];
        const long long kx = okey(xk, klo[k]);
        if (kx >= khi[k])
          xk -= L;
        else if (kx < klo[k])
          xk += L;
      }
      xn[k] = xk;
      vn[k] = vhn[k] + 0.5 * dt * a3[k];
    }
    const double du = o.du[p];
    const double u = s.u[p];
    const double un = dt_prev > 0.0 ? u + dt * ((1.0 + q) * du - q * s.du_prev[p]) : u + dt * du;
    const int cnt = nn[p];
    double h = s.h[p];
    if (prm.ng_target > 0)
      h = h * (cnt >= 0 && cnt < kHTab ? __ldg(hfac + cnt) : hfac_of(prm.ng_target, cnt));
    const double m = s.m[p];
    // loaded before the first store (the compiler cannot tell that d aliases
    // none of the inputs, and a load after a store waits for its own round trip)
    const int64_t id = d.id ? s.id[p] : 0;
    d.x[p] = xn[0];
    d.y[p] = xn[1];
    d.z[p] = xn[2];
    d.vx[p] = vn[0];
    d.vy[p] = vn[1];
    d.vz[p] = vn[2];
    d.vxh[p] = vhn[0];
    d.vyh[p] = vhn[1];
    d.vzh[p] = vhn[2];
    d.u[p] = un;
    if (d.du_prev) d.du_prev[p] = du;  // NULL: the caller takes du_prev, m and id elsewhere
    d.h[p] = h;
    if (d.m) d.m[p] = m;
    if (d.id) d.id[p] = id;
    acc[0] += m * vn[0];
    acc[1] += m * vn[1];
    acc[2] += m * vn[2];
    // m |v|^2, halved once at the end: scaling by 0.5 is exact, so the sum
    // equals that of 0.5 m |v|^2 bit for bit
    acc[3] += m * (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
    acc[4] += m * un;
    if (kAngular) {
      acc[5] += m * (xn[1] * vn[2] - xn[2] * vn[1]);
      acc[6] += m * (xn[2] * vn[0] - xn[0] * vn[2]);
      acc[7] += m * (xn[0] * vn[1] - xn[1] * vn[0]);
    }
    csum += cnt;
    cmin = min(cmin, cnt);
    cmax = max(cmax, cnt);
  }
  acc[8] = 0.0;
  acc[9] = 0.0;
  acc[10] = (double)csum;  // exact: the sum is far below 2^53
  double nmin = cmin == INT_MAX ? INFINITY : (double)cmin;
  double nmax = cmax == INT_MIN ? -INFINITY : (double)cmax;
  nmin = warp_min(nmin);
  nmax = warp_max(nmax);
  __shared__ double shm[kThreads / 32][2];
  if ((threadIdx.x & 31) == 0) {
    shm[threadIdx.x >> 5][0] = nmin;
    shm[threadIdx.x >> 5][1] = nmax;
  }
  block_sums<11>(acc, part);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) {
      nmin = fmin(nmin, shm[w][0]);
      nmax = fmax(nmax, shm[w][1]);
    }
    part[blockIdx.x * kParts + 8] = nmin;
    part[blockIdx.x * kParts + 9] = nmax;
  }
  if (!block_last(counter)) return;
  __threadfence();
  __shared__ double res[11];
  const Op ops[11] = {Op::kSum, Op::kSum, Op::kSum, Op::kSum, Op::kSum, Op::kSum,
                      Op::kSum, Op::kSum, Op::kMin, Op::kMax, Op::kSum};
  finalize_block<11>(part, gridDim.x, ops, res);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 8; ++k) diag[k] = res[k];
    diag[3] = 0.5 * res[3];
    if (!kAngular) diag[5] = diag[6] = diag[7] = NAN;
    diag[9] = res[8];
    diag[10] = res[9];
    diag[11] = res[10];
    stats[2] += (unsigned long long)res[10];
    stats[3] += (unsigned long long)n;
    *counter = 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_diag(StateView s, int64_t n, double* diag,
                                                   double* part, unsigned int* counter) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double m = s.m[p], x = s.x[p], y = s.y[p], z = s.z[p];
    const double vx = s.vx[p], vy = s.vy[p], vz = s.vz[p];
    acc[0] += m * vx;
    acc[1] += m * vy;
    acc[2] += m * vz;
    acc[3] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    acc[4] += m * s.u[p];
    acc[5] += m * (y * vz - z * vy);
    acc[6] += m * (z * vx - x * vz);
    acc[7] += m * (x * vy - y * vx);
  }
  block_sums<8>(acc, part);
  if (!block_last(counter)) return;
  __threadfence();
  __shared__ double res[8];
  const Op ops[8] = {Op::kSum, Op::kSum, Op::kSum, Op::kSum,
                     Op::kSum, Op::kSum, Op::kSum, Op::kSum};
  finalize_block<8>(part, gridDim.x, ops, res);
  if (threadIdx.x < 8) diag[threadIdx.x] = res[threadIdx.x];
  if (threadIdx.x == 0) *counter = 0;
}

inline int red_blocks(int64_t n, int sm) {
  int64_t b = (n + kThreads - 1) / kThreads;
  int64_t cap = (int64_t)sm * 4;
  if (cap > kReduceBlocks) cap = kReduceBlocks;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_timestep(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n, double* dt_io,
                     cudaStream_t st) {
  k_timestep<<<red_blocks(n, ctx->sm_count), kThreads, 0, st>>>(
      s.h, o.c, s.u, o.du, n, ctx->prm.courant, ctx->prm.dt_growth, ctx->prm.energy_dt, dt_io,
      ctx->diag, ctx->red.part, ctx->red.counter + 1, ctx->err);
  ctx->launches += 1;
}

void launch_hfac_table(sph_ctx* ctx, cudaStream_t st) {
  k_hfac_table<<<(kHTab + 255) / 256, 256, 0, st>>>(ctx->hfac, ctx->prm.ng_target);
  ctx->hfac_ng = ctx->prm.ng_target;
  ctx->launches += 1;
}

void launch_update(sph_ctx* ctx, const StateView& s, const OutView& o, const StateView& dst,
                   int64_t n, const double* dt_io, cudaStream_t st) {
  (void)dt_io;
  if (ctx->hfac_ng != ctx->prm.ng_target) launch_hfac_table(ctx, st);
  auto kern = ctx->prm.angular_sums ? k_update<true> : k_update<false>;
  kern<<<red_blocks(n, ctx->sm_count), kThreads, 0, st>>>(
      s, o, dst, ctx->nn, n, ctx->prm, ctx->hfac, ctx->diag, ctx->red.part,
      ctx->red.counter + 2, ctx->stats);
  ctx->launches += 1;
}

void launch_diagnostics(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st) {
  k_diag<<<red_blocks(n, ctx->sm_count), kThreads, 0, st>>>(s, n, ctx->diag + 16, ctx->red.part,
                                                            ctx->red.counter + 3);
  ctx->launches += 1;
}

}  // namespace sph
