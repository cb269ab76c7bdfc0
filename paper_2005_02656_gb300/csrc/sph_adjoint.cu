// Differentiable rollout (sph_adjoint_* in include/sph.h): K FP64 steps of
// the section 4.1 pipeline with state checkpoints, and hand-written reverse
// kernels of one step, run from the last step to the first.
//
// Forward.  A recording step is sph_step itself with the context's sorted
// state, permutation, neighbour lists and grid redirected into a tape slot,
// and its density / EOS / IAD outputs written there: the tape then holds
// exactly what the step computed.  Steps outside the segment being recorded
// run into the context's own scratch.
//
// Reverse of one step (everything in the step's sorted order; b runs over the
// list of a, d = x_b - x_a with the minimum image, r^2 = d.d):
//   update      vh' = vh + D acc, x' = x + dt vh', v' = vh' + dt/2 acc,
//               u' = u + dt (k1 du - k2 du_prev), du_prev' = du
//               -> acc_bar = D (vh'_bar + v'_bar + dt x'_bar) + dt/2 v'_bar,
//                  du_bar = dt k1 u'_bar + du_prev'_bar (fused into the
//                  momentum kernel's prologue);
//   momentum    Eqs. 2-5 with A_a = W_a C_a d, A_b = W_b C_b d and the pair
//               viscosity Pi: every partial of one pair term is formed once,
//               by the thread of a; the partials that belong to b are written
//               to a pair buffer at the list entry's slot and summed by b over
//               its reverse list (the sorted set of (a, k) with b in a's list);
//   IAD         C = tau^{-1}: tau_bar = -C sym(C_bar) C, then
//               tau_a = sum_b (m_b/rho_b) W_a d d^T, gathered over the list
//               (for a) and over the reverse list (for b);
//   EOS         P = (gamma-1) rho u, c = sqrt(gamma P / rho), and with the
//               grad-h terms X = P / (Omega rho^2), Omega = -(2/(3 rho)) G,
//               G = sum_b m_b t dW/dt (t = r^2 / h_a^2);
//   density     Eq. 1 (and G's pair terms, whose r^2-derivative is
//               m_b (W' + t W'') / h_a^2), gathered over list and reverse
//               list as for IAD.
// Reverse lists are built per step from the tape's lists (count, scan,
// scatter, then each row sorted), so every sum runs in a fixed order and the
// gradient is bit-reproducible.  The viscosity switch x_ab . v_ab < 0 is
// decided from the recorded state exactly as the forward kernel decides it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_scan.cuh"
#include "sph_tile.cuh"

using sph::Grid;
using sph::scan::kScanItems;
using sph::StateView;

namespace {

constexpr int kThreads = 128;
constexpr int kRowSmem = 512;     // reverse-list rows sorted in shared memory up to this length
constexpr int kSortWarps = 4;
constexpr int kKBits = 12;        // reverse entry: (a << 12) | k with k < 4096 = max max_nb
constexpr int kAlphaBlocks = 1024;

// Adjoint of the 11 differentiated state fields, one array each.
struct Bar {
  double *x, *y, *z, *vx, *vy, *vz, *vxh, *vyh, *vzh, *u, *dup;
};

// Per-particle reverse scratch of one step.
struct Work {
  Bar z;         // adjoint of the step's input state, being assembled (sorted order)
  double* Xb;    // dL/dX, X = P / rho^2
  double* irb;   // dL/d(1/rho)
  double* cb;    // dL/dc
  double* Cb;    // 6 per particle: sym(dL/dC), then S = -C sym(dL/dC) C
  double* rhob;  // dL/drho
  double* Gb;    // dL/dG of the grad-h sum (0 without grad-h terms)
};

// One recorded step, sorted order.
struct Slot {
  StateView s;
  int32_t* perm;
  int32_t* nn;
  uint32_t* nbr;
  double *rho, *p, *c, *iad;
  double* omega;  // grad-h terms of the step (read when gradh)
  Grid* grid;
  double* dtp;  // device [dt, dt_prev]
};

struct Rev {
  int32_t* cnt;
  int64_t* start;  // n + 1
  uint64_t* list;  // (a << kKBits) | k, rows sorted ascending
};

// Per list entry (a, k), slot = k * stride + a: the 12 partials of the pair
// term that belong to the neighbour b (one 96-byte record), and W_a and
// dW_a/d(r^2) of the entry.
constexpr int kRec = 12;
struct PairBuf {
  double* rec;   // kRec doubles per slot
  double2* wk;   // (W_a, dW_a / d r^2) per slot
  int64_t stride;
};

// Per-particle factors of one step (sorted order): 1/h^2, B_n/h^3, 1/rho,
// P/rho^2, m/rho.
struct Prep {
  double *hinv2, *norm, *ir, *X, *vol;
};

struct Consts {
  double gamma, alpha, Bn;
  int sinc_n, max_nb;
  int gradh;
};

__device__ __forceinline__ void sepd(const Grid& g, double xa, double ya, double za, double xb,
                                     double yb, double zb, double& dx, double& dy, double& dz) {
  dx = sph::min_image(xb - xa, g.Lbox[0], g.halfL[0], g.periodic[0]);
  dy = sph::min_image(yb - ya, g.Lbox[1], g.halfL[1], g.periodic[1]);
  dz = sph::min_image(zb - za, g.Lbox[2], g.halfL[2], g.periodic[2]);
}

// y = C x for C stored as (xx, xy, xz, yy, yz, zz).
__device__ __forceinline__ void sym_mv(const double* C, double x0, double x1, double x2,
                                       double& y0, double& y1, double& y2) {
  y0 = C[0] * x0 + C[1] * x1 + C[2] * x2;
  y1 = C[1] * x0 + C[3] * x1 + C[4] * x2;
  y2 = C[2] * x0 + C[4] * x1 + C[5] * x2;
}

// ---------------------------------------------------------------------------
// Reverse lists
// ---------------------------------------------------------------------------
__global__ void k_rev_count(const int32_t* nn, const uint32_t* nbr, int mb, int64_t n,
                            int32_t* cnt) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int c = min(nn[a], mb);
    const uint32_t* row = nbr + a * mb;
    for (int k = 0; k < c; ++k) atomicAdd(&cnt[sph::entry_index(row[k])], 1);
  }
}

__global__ void k_rev_fill(const int32_t* nn, const uint32_t* nbr, int mb, int64_t n,
                           const int64_t* start, int32_t* fill, uint64_t* list) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int c = min(nn[a], mb);
    const uint32_t* row = nbr + a * mb;
    for (int k = 0; k < c; ++k) {
      const int b = sph::entry_index(row[k]);
      const int pos = atomicAdd(&fill[b], 1);
      list[start[b] + pos] = ((uint64_t)a << kKBits) | (uint64_t)k;
    }
  }
}

// Sorts every row ascending: a warp per row, rank of each entry among the
// row's (distinct) entries; rows longer than kRowSmem by one lane's
// insertion sort in place.
__global__ void __launch_bounds__(kSortWarps * 32) k_rev_sort(const int64_t* start, int64_t n,
                                                              uint64_t* list) {
  __shared__ uint64_t buf[kSortWarps][kRowSmem];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x * (int64_t)kSortWarps + w; b < n;
       b += (int64_t)gridDim.x * kSortWarps) {
    const int64_t s0 = start[b];
    const int L = (int)(start[b + 1] - s0);
    if (L <= 1) continue;
    uint64_t* row = list + s0;
    if (L <= kRowSmem) {
      for (int i = lane; i < L; i += 32) buf[w][i] = row[i];
      __syncwarp();
      for (int i = lane; i < L; i += 32) {
        const uint64_t e = buf[w][i];
        int rank = 0;
        for (int j = 0; j < L; ++j) rank += buf[w][j] < e;
        row[rank] = e;
      }
      __syncwarp();
    } else if (lane == 0) {
      for (int i = 1; i < L; ++i) {
        const uint64_t e = row[i];
        int j = i - 1;
        while (j >= 0 && row[j] > e) {
          row[j + 1] = row[j];
          --j;
        }
        row[j + 1] = e;
      }
    }
    __syncwarp();
  }
}

__global__ void k_adj_prep(Slot sl, Prep pr, int64_t n, double Bn, int gradh) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double h = sl.s.h[i];
    const double hinv2 = 1.0 / (h * h);
    const double ir = 1.0 / sl.rho[i];
    pr.hinv2[i] = hinv2;
    pr.norm[i] = Bn * hinv2 / h;
    pr.ir[i] = ir;
    pr.X[i] = gradh ? sl.p[i] * ir * ir / sl.omega[i] : sl.p[i] * ir * ir;
    pr.vol[i] = sl.s.m[i] * ir;
  }
}

// ---------------------------------------------------------------------------
// Reverse of update + momentum/energy, the target's side.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_adj_momentum_a(Slot sl, Prep pr, Bar q, Work w,
                                                             PairBuf pb, int64_t n, Consts kc,
                                                             double* apart) {
  const Grid g = *sl.grid;
  const double dt = sl.dtp[0], dt_prev = sl.dtp[1];
  const double delta = 0.5 * (dt + dt_prev);
  const double qr = dt_prev > 0.0 ? dt / (2.0 * dt_prev) : 0.0;
  const double k1 = dt_prev > 0.0 ? 1.0 + qr : 1.0;
  const double k2 = qr;
  const StateView& s = sl.s;
  const int mb = kc.max_nb;
  double alpha_bar = 0.0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    // update: adjoint of acc and du, and the pass-through fields
    const double vhbx = q.vxh[a] + q.vx[a] + dt * q.x[a];
    const double vhby = q.vyh[a] + q.vy[a] + dt * q.y[a];
    const double vhbz = q.vzh[a] + q.vz[a] + dt * q.z[a];
    const double gx = delta * vhbx + 0.5 * dt * q.vx[a];
    const double gy = delta * vhby + 0.5 * dt * q.vy[a];
    const double gz = delta * vhbz + 0.5 * dt * q.vz[a];
    const double e = dt * k1 * q.u[a] + q.dup[a];
    w.z.vxh[a] = vhbx;
    w.z.vyh[a] = vhby;
    w.z.vzh[a] = vhbz;
    w.z.u[a] = q.u[a];
    w.z.dup[a] = -dt * k2 * q.u[a];

    const double xa = s.x[a], ya = s.y[a], za = s.z[a];
    const double vxa = s.vx[a], vya = s.vy[a], vza = s.vz[a];
    const double hinv2a = pr.hinv2[a];
    const double norma = pr.norm[a];
    const double ira = pr.ir[a];
    const double Xa = pr.X[a];
    const double ca = sl.c[a];
    double Ca[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) Ca[i] = sl.iad[6 * a + i];
    double xbx = 0, xby = 0, xbz = 0, vbx = 0, vby = 0, vbz = 0;
    double Xbar = 0, irbar = 0, cbar = 0;
    double Cbar[6] = {0, 0, 0, 0, 0, 0};
    const int cnt = min(sl.nn[a], mb);
    const uint32_t* list = sl.nbr + a * mb;
    for (int k = 0; k < cnt; ++k) {
      const int64_t b = sph::entry_index(list[k]);
      double dx, dy, dz;
      sepd(g, xa, ya, za, s.x[b], s.y[b], s.z[b], dx, dy, dz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      double Wa, dWa;
      sph::kernel_w64_d(r2 * hinv2a, norma, kc.sinc_n, Wa, dWa);
      dWa *= hinv2a;  // dW_a / d r^2
      const double hinv2b = pr.hinv2[b];
      const double tb = r2 * hinv2b;
      double Wb = 0.0, dWb = 0.0;
      if (tb < 4.0) {
        sph::kernel_w64_d(tb, pr.norm[b], kc.sinc_n, Wb, dWb);
        dWb *= hinv2b;
      }
      double Cb[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) Cb[i] = sl.iad[6 * b + i];
      double cax, cay, caz, cbx, cby, cbz;
      sym_mv(Ca, dx, dy, dz, cax, cay, caz);
      sym_mv(Cb, dx, dy, dz, cbx, cby, cbz);
      const double Aax = Wa * cax, Aay = Wa * cay, Aaz = Wa * caz;
      const double Abx = Wb * cbx, Aby = Wb * cby, Abz = Wb * cbz;
      const double vabx = vxa - s.vx[b], vaby = vya - s.vy[b], vabz = vza - s.vz[b];
      const double xv = -(dx * vabx + dy * vaby + dz * vabz);
      const double irb = pr.ir[b];
      const double Xb = pr.X[b];
      const double cbv = sl.c[b];
      const bool on = xv < 0.0;
      double rinv = 0.0, wv = 0.0, vsig = 0.0, Pi = 0.0;
      if (on) {
        rinv = rsqrt(r2);
        wv = xv * rinv;
        vsig = ca + cbv - 3.0 * wv;
        Pi = -0.5 * kc.alpha * vsig * wv;
      }
      const double mb_ = s.m[b];
      const double fa1 = Xa + 0.5 * Pi * ira, fb1 = Xb + 0.5 * Pi * irb;
      const double fa2 = Xa + 0.25 * Pi * ira, fb2 = 0.25 * Pi * irb;
      const double gAa = gx * Aax + gy * Aay + gz * Aaz;
      const double gAb = gx * Abx + gy * Aby + gz * Abz;
      const double vAa = vabx * Aax + vaby * Aay + vabz * Aaz;
      const double vAb = vabx * Abx + vaby * Aby + vabz * Abz;
      // partials of L_pair = -m_b (fa1 g.A_a + fb1 g.A_b) + e m_b (fa2 v.A_a + fb2 v.A_b)
      const double fa1b = -mb_ * gAa, fb1b = -mb_ * gAb;
      const double fa2b = e * mb_ * vAa, fb2b = e * mb_ * vAb;
      const double Aabx = mb_ * (-fa1 * gx + e * fa2 * vabx);
      const double Aaby = mb_ * (-fa1 * gy + e * fa2 * vaby);
      const double Aabz = mb_ * (-fa1 * gz + e * fa2 * vabz);
      const double Abbx = mb_ * (-fb1 * gx + e * fb2 * vabx);
      const double Abby = mb_ * (-fb1 * gy + e * fb2 * vaby);
      const double Abbz = mb_ * (-fb1 * gz + e * fb2 * vabz);
      double vabbx = e * mb_ * (fa2 * Aax + fb2 * Abx);
      double vabby = e * mb_ * (fa2 * Aay + fb2 * Aby);
      double vabbz = e * mb_ * (fa2 * Aaz + fb2 * Abz);
      const double Pib = 0.5 * ira * fa1b + 0.5 * irb * fb1b + 0.25 * ira * fa2b + 0.25 * irb * fb2b;
      Xbar += fa1b + fa2b;
      irbar += Pi * (0.5 * fa1b + 0.25 * fa2b);
      const double Xbb = fb1b;
      const double irbb = Pi * (0.5 * fb1b + 0.25 * fb2b);
      // A_a = W_a C_a d and A_b = W_b C_b d
      const double Wab = Aabx * cax + Aaby * cay + Aabz * caz;
      const double Wbb = Abbx * cbx + Abby * cby + Abbz * cbz;
      Cbar[0] += Wa * Aabx * dx;
      Cbar[1] += 0.5 * Wa * (Aabx * dy + Aaby * dx);
      Cbar[2] += 0.5 * Wa * (Aabx * dz + Aabz * dx);
      Cbar[3] += Wa * Aaby * dy;
      Cbar[4] += 0.5 * Wa * (Aaby * dz + Aabz * dy);
      Cbar[5] += Wa * Aabz * dz;
      double t0, t1, t2, u0, u1, u2;
      sym_mv(Ca, Aabx, Aaby, Aabz, t0, t1, t2);
      sym_mv(Cb, Abbx, Abby, Abbz, u0, u1, u2);
      double dbx = Wa * t0 + Wb * u0;
      double dby = Wa * t1 + Wb * u1;
      double dbz = Wa * t2 + Wb * u2;
      double r2b = Wab * dWa + Wbb * dWb;
      double cpair = 0.0;
      if (on) {
        alpha_bar += Pib * (-0.5 * vsig * wv);
        cpair = Pib * (-0.5 * kc.alpha * wv);
        const double wb = Pib * (-0.5 * kc.alpha * (ca + cbv - 6.0 * wv));
        const double xvb = wb * rinv;
        r2b += -0.5 * wb * wv * rinv * rinv;
        dbx += -xvb * vabx;
        dby += -xvb * vaby;
        dbz += -xvb * vabz;
        vabbx += -xvb * dx;
        vabby += -xvb * dy;
        vabbz += -xvb * dz;
      }
      dbx += 2.0 * r2b * dx;
      dby += 2.0 * r2b * dy;
      dbz += 2.0 * r2b * dz;
      cbar += cpair;
      xbx -= dbx;
      xby -= dby;
      xbz -= dbz;
      vbx += vabbx;
      vby += vabby;
      vbz += vabbz;
      const int64_t slot = (int64_t)k * pb.stride + a;
      double2* rec = reinterpret_cast<double2*>(pb.rec + kRec * slot);
      rec[0] = make_double2(dbx, dby);
      rec[1] = make_double2(dbz, vabbx);
      rec[2] = make_double2(vabby, vabbz);
      rec[3] = make_double2(Xbb, irbb);
      rec[4] = make_double2(cpair, Wb * Abbx);
      rec[5] = make_double2(Wb * Abby, Wb * Abbz);
      pb.wk[slot] = make_double2(Wa, dWa);
    }
    w.z.x[a] = q.x[a] + xbx;
    w.z.y[a] = q.y[a] + xby;
    w.z.z[a] = q.z[a] + xbz;
    w.z.vx[a] = vbx;
    w.z.vy[a] = vby;
    w.z.vz[a] = vbz;
    w.Xb[a] = Xbar;
    w.irb[a] = irbar;
    w.cb[a] = cbar;
#pragma unroll
    for (int i = 0; i < 6; ++i) w.Cb[6 * a + i] = Cbar[i];
  }
  // block partial of dL/dalpha (summed in block order by k_alpha_sum)
  __shared__ double sh[kThreads / 32];
  alpha_bar = sph::warp_sum(alpha_bar);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = alpha_bar;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) t += sh[i];
    apart[blockIdx.x] = t;
  }
}

__global__ void k_alpha_sum(const double* apart, int nb, double* alpha_acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += apart[i];
    *alpha_acc += t;
  }
}

// ---------------------------------------------------------------------------
// Reverse of momentum/energy, the neighbour's side, then the IAD inverse and
// the EOS.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_adj_momentum_b(Slot sl, Work w, PairBuf pb, Rev rv,
                                                             int64_t n, Consts kc) {
  const Grid g = *sl.grid;
  const StateView& s = sl.s;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    const double xb = s.x[b], yb = s.y[b], zb = s.z[b];
    double dsx = 0, dsy = 0, dsz = 0, vsx = 0, vsy = 0, vsz = 0, Xs = 0, irs = 0, cs = 0;
    double Cs[6] = {0, 0, 0, 0, 0, 0};
    const int64_t e0 = rv.start[b], e1 = rv.start[b + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const uint64_t ent = rv.list[e];
      const int64_t a = (int64_t)(ent >> kKBits);
      const int64_t k = (int64_t)(ent & ((1u << kKBits) - 1u));
      const int64_t slot = k * pb.stride + a;
      const double2* rec = reinterpret_cast<const double2*>(pb.rec + kRec * slot);
      const double2 r0 = rec[0], r1 = rec[1], r2_ = rec[2], r3 = rec[3], r4 = rec[4], r5 = rec[5];
      dsx += r0.x;
      dsy += r0.y;
      dsz += r1.x;
      vsx += r1.y;
      vsy += r2_.x;
      vsz += r2_.y;
      Xs += r3.x;
      irs += r3.y;
      cs += r4.x;
      const double Ax = r4.y, Ay = r5.x, Az = r5.y;
      double dx, dy, dz;
      sepd(g, s.x[a], s.y[a], s.z[a], xb, yb, zb, dx, dy, dz);
      Cs[0] += Ax * dx;
      Cs[1] += 0.5 * (Ax * dy + Ay * dx);
      Cs[2] += 0.5 * (Ax * dz + Az * dx);
      Cs[3] += Ay * dy;
      Cs[4] += 0.5 * (Ay * dz + Az * dy);
      Cs[5] += Az * dz;
    }
    w.z.x[b] += dsx;
    w.z.y[b] += dsy;
    w.z.z[b] += dsz;
    w.z.vx[b] -= vsx;
    w.z.vy[b] -= vsy;
    w.z.vz[b] -= vsz;
    const double Xbar = w.Xb[b] + Xs;
    double irbar = w.irb[b] + irs;
    const double cbar = w.cb[b] + cs;
    double G[6], C[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      G[i] = w.Cb[6 * b + i] + Cs[i];
      C[i] = sl.iad[6 * b + i];
    }
    // S = -C G C (G and C symmetric): M = G C, then S = -C M
    double M[3][3];
    const double Gm[3][3] = {{G[0], G[1], G[2]}, {G[1], G[3], G[4]}, {G[2], G[4], G[5]}};
    const double Cm[3][3] = {{C[0], C[1], C[2]}, {C[1], C[3], C[4]}, {C[2], C[4], C[5]}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) M[i][j] = Gm[i][0] * Cm[0][j] + Gm[i][1] * Cm[1][j] + Gm[i][2] * Cm[2][j];
    double S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) S[i][j] = -(Cm[i][0] * M[0][j] + Cm[i][1] * M[1][j] + Cm[i][2] * M[2][j]);
    w.Cb[6 * b + 0] = S[0][0];
    w.Cb[6 * b + 1] = 0.5 * (S[0][1] + S[1][0]);
    w.Cb[6 * b + 2] = 0.5 * (S[0][2] + S[2][0]);
    w.Cb[6 * b + 3] = S[1][1];
    w.Cb[6 * b + 4] = 0.5 * (S[1][2] + S[2][1]);
    w.Cb[6 * b + 5] = S[2][2];
    // EOS and X = P / (Omega rho^2), 1/rho
    const double rho = sl.rho[b], p = sl.p[b], c = sl.c[b];
    const double ir = 1.0 / rho;
    const double om = kc.gradh ? sl.omega[b] : 1.0;
    const double pbar = Xbar * ir * ir / om + cbar * kc.gamma / (2.0 * c * rho);
    irbar += 2.0 * Xbar * p * ir / om;
    if (kc.gradh) {
      // Omega = -(2/3) (1/rho) G with G = -(3/2) Omega rho
      const double X = p * ir * ir / om;
      const double ombar = -Xbar * X / om;
      w.Gb[b] = -2.0 / 3.0 * ir * ombar;
      irbar += -2.0 / 3.0 * (-1.5 * om * rho) * ombar;
    } else {
      w.Gb[b] = 0.0;
    }
    w.rhob[b] = pbar * (kc.gamma - 1.0) * s.u[b] - cbar * c / (2.0 * rho);
    w.irb[b] = irbar;
    w.z.u[b] += pbar * (kc.gamma - 1.0) * rho;
  }
}

// ---------------------------------------------------------------------------
// Reverse of IAD's tau sums: tau_a = sum_b vol_b W_a d d^T, vol = m / rho.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_adj_iad(Slot sl, Prep pr, Work w, PairBuf pb, Rev rv,
                                                      int64_t n, Consts kc) {
  const Grid g = *sl.grid;
  const StateView& s = sl.s;
  const int mb = kc.max_nb;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double xp = s.x[p], yp = s.y[p], zp = s.z[p];
    double Sp[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) Sp[i] = w.Cb[6 * p + i];
    double xbx = 0, xby = 0, xbz = 0;
    // p's own sum: pairs (p, b)
    const int cnt = min(sl.nn[p], mb);
    const uint32_t* list = sl.nbr + p * mb;
    for (int k = 0; k < cnt; ++k) {
      const int64_t b = sph::entry_index(list[k]);
      double dx, dy, dz;
      sepd(g, xp, yp, zp, s.x[b], s.y[b], s.z[b], dx, dy, dz);
      const double2 wk = pb.wk[(int64_t)k * pb.stride + p];
      const double vol = pr.vol[b];
      double s0, s1, s2;
      sym_mv(Sp, dx, dy, dz, s0, s1, s2);
      const double wbar = dx * s0 + dy * s1 + dz * s2;
      const double ww = vol * wk.x;
      const double f = 2.0 * wbar * vol * wk.y;
      xbx -= 2.0 * ww * s0 + f * dx;
      xby -= 2.0 * ww * s1 + f * dy;
      xbz -= 2.0 * ww * s2 + f * dz;
    }
    // sums of the particles a whose list holds p: pairs (a, p)
    const double volp = pr.vol[p];
    double volbar = 0.0;
    const int64_t e0 = rv.start[p], e1 = rv.start[p + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const uint64_t ent = rv.list[e];
      const int64_t a = (int64_t)(ent >> kKBits);
      const int64_t k = (int64_t)(ent & ((1u << kKBits) - 1u));
      double dx, dy, dz;
      sepd(g, s.x[a], s.y[a], s.z[a], xp, yp, zp, dx, dy, dz);
      const double2 wk = pb.wk[k * pb.stride + a];
      double Sa[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) Sa[i] = w.Cb[6 * a + i];
      double s0, s1, s2;
      sym_mv(Sa, dx, dy, dz, s0, s1, s2);
      const double wbar = dx * s0 + dy * s1 + dz * s2;
      const double ww = volp * wk.x;
      const double f = 2.0 * wbar * volp * wk.y;
      xbx += 2.0 * ww * s0 + f * dx;
      xby += 2.0 * ww * s1 + f * dy;
      xbz += 2.0 * ww * s2 + f * dz;
      volbar += wbar * wk.x;
    }
    w.z.x[p] += xbx;
    w.z.y[p] += xby;
    w.z.z[p] += xbz;
    const double ir = pr.ir[p];
    const double irbar = w.irb[p] + s.m[p] * volbar;
    w.rhob[p] -= irbar * ir * ir;
  }
}

// ---------------------------------------------------------------------------
// Reverse of the density sums (Eq. 1), then the adjoint of the step's input
// written back through the sort permutation.  kCached: dW_a/d r^2 of every
// list entry is in the pair buffer (written by the momentum kernel);
// otherwise (the final density pass) it is evaluated here.
// ---------------------------------------------------------------------------
template <bool kCached>
__device__ __forceinline__ double dw_dr2(const PairBuf& pb, int64_t k, int64_t a, double r2,
                                         const Prep& pr, const Consts& kc) {
  if (kCached) return pb.wk[k * pb.stride + a].y;
  double W, dW;
  const double hinv2 = pr.hinv2[a];
  sph::kernel_w64_d(r2 * hinv2, pr.norm[a], kc.sinc_n, W, dW);
  return dW * hinv2;
}

// r^2-derivative of the grad-h pair term m_b t dW/dt of target a (t = r^2/h_a^2),
// without m_b.
__device__ __forceinline__ double dg_dr2(int64_t a, double r2, const Prep& pr, const Consts& kc) {
  const double hinv2 = pr.hinv2[a];
  return sph::kernel_tdw_dt64(r2 * hinv2, pr.norm[a], kc.sinc_n) * hinv2;
}

template <bool kCached, bool GRADH>
__global__ void __launch_bounds__(kThreads) k_adj_density(Slot sl, Prep pr, Work w, PairBuf pb,
                                                          Rev rv, Bar out, int64_t n, Consts kc) {
  const Grid g = *sl.grid;
  const StateView& s = sl.s;
  const int mb = kc.max_nb;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double xp = s.x[p], yp = s.y[p], zp = s.z[p];
    const double rbp = w.rhob[p];
    const double gbp = GRADH ? w.Gb[p] : 0.0;
    double xbx = 0, xby = 0, xbz = 0;
    const int cnt = min(sl.nn[p], mb);
    const uint32_t* list = sl.nbr + p * mb;
    for (int k = 0; k < cnt; ++k) {
      const int64_t b = sph::entry_index(list[k]);
      double dx, dy, dz;
      sepd(g, xp, yp, zp, s.x[b], s.y[b], s.z[b], dx, dy, dz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      double f = 2.0 * rbp * s.m[b] * dw_dr2<kCached>(pb, k, p, r2, pr, kc);
      if (GRADH) f += 2.0 * gbp * s.m[b] * dg_dr2(p, r2, pr, kc);
      xbx -= f * dx;
      xby -= f * dy;
      xbz -= f * dz;
    }
    const double mp = s.m[p];
    const int64_t e0 = rv.start[p], e1 = rv.start[p + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const uint64_t ent = rv.list[e];
      const int64_t a = (int64_t)(ent >> kKBits);
      const int64_t k = (int64_t)(ent & ((1u << kKBits) - 1u));
      double dx, dy, dz;
      sepd(g, s.x[a], s.y[a], s.z[a], xp, yp, zp, dx, dy, dz);
      const double r2 = dx * dx + dy * dy + dz * dz;
      double f = 2.0 * w.rhob[a] * mp * dw_dr2<kCached>(pb, k, a, r2, pr, kc);
      if (GRADH) f += 2.0 * w.Gb[a] * mp * dg_dr2(a, r2, pr, kc);
      xbx += f * dx;
      xby += f * dy;
      xbz += f * dz;
    }
    const int64_t o = sl.perm[p];
    out.x[o] = w.z.x[p] + xbx;
    out.y[o] = w.z.y[p] + xby;
    out.z[o] = w.z.z[p] + xbz;
    out.vx[o] = w.z.vx[p];
    out.vy[o] = w.z.vy[p];
    out.vz[o] = w.z.vz[p];
    out.vxh[o] = w.z.vxh[p];
    out.vyh[o] = w.z.vyh[p];
    out.vzh[o] = w.z.vzh[p];
    out.u[o] = w.z.u[p];
    out.dup[o] = w.z.dup[p];
  }
}

// Seed of the reverse pass: dL/d(final x, v, u, rho) from the caller's
// particle order into the sorted order of the final density pass.
__global__ void k_seed(const double* gf, const int64_t* id, int64_t n, Work w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = id[i];
    w.z.x[i] = gf[0 * n + j];
    w.z.y[i] = gf[1 * n + j];
    w.z.z[i] = gf[2 * n + j];
    w.z.vx[i] = gf[3 * n + j];
    w.z.vy[i] = gf[4 * n + j];
    w.z.vz[i] = gf[5 * n + j];
    w.z.u[i] = gf[6 * n + j];
    w.rhob[i] = gf[7 * n + j];
    w.z.vxh[i] = 0.0;
    w.z.vyh[i] = 0.0;
    w.z.vzh[i] = 0.0;
    w.z.dup[i] = 0.0;
  }
}

// Final state and density into the caller's particle order.
__global__ void k_final_out(StateView s, const double* rho, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = s.id[i];
    out[0 * n + j] = s.x[i];
    out[1 * n + j] = s.y[i];
    out[2 * n + j] = s.z[i];
    out[3 * n + j] = s.vx[i];
    out[4 * n + j] = s.vy[i];
    out[5 * n + j] = s.vz[i];
    out[6 * n + j] = s.u[i];
    out[7 * n + j] = rho[i];
  }
}

__global__ void k_iota(int64_t* id, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    id[i] = i;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct sph_adj {
  sph_ctx* ctx;
  sph_params prm;
  int64_t n_max;
  int steps, every, nseg;
  int64_t n;
  double alpha;
  int have_forward;
  int tape_seg;  // segment whose steps are in the tape, -1 none
  char last_error[512];
  int64_t bytes, launches, recomputed, backwards;
  int sm_count;
  // working state (caller order) and its output scratch
  double* wbuf;
  int64_t* wid;
  sph_state W;
  double* dt_dev;
  // checkpoints: nseg x (13 n_max doubles + n_max ids + 1 dt)
  double* cbuf;
  int64_t* cid;
  double* cdt;
  // tape: every + 1 slots (the last one is the final density pass)
  Slot* slot;
  double* tbuf;
  int64_t* tid;
  int32_t* tint;   // perm, nn per slot
  uint32_t* tnbr;
  Grid* tgrid;
  double* tdt;     // 2 per slot
  double* dts;     // dt of every step of the last forward
  // reverse
  double* bbuf;    // 2 x 11 n_max
  Bar q, pnext;
  double* kbuf;
  Work w;
  double* pbuf;
  double2* wkbuf;
  PairBuf pb;
  Prep pr;
  int32_t* rcnt;
  int64_t* rstart;
  uint64_t* rlist;
  int64_t* spart;
  double* apart;
  double* alpha_acc;
};

namespace {

int aerr(sph_adj* A, int code, const char* fmt, ...) {
  if (A) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(A->last_error, sizeof(A->last_error), fmt, ap);
    va_end(ap);
  }
  return code;
}

int acuda(sph_adj* A, cudaError_t e, const char* what) {
  return aerr(A, e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

template <typename T>
cudaError_t amalloc(sph_adj* A, T** p, size_t count) {
  size_t b = count * sizeof(T);
  if (b == 0) b = sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, b);
  if (e == cudaSuccess)
    A->bytes += (int64_t)b;
  else
    *p = nullptr;
  return e;
}

void free_adj(sph_adj* A) {
  void* ptrs[] = {A->wbuf, A->wid, A->dt_dev, A->cbuf, A->cid, A->cdt, A->tbuf, A->tid,
                  A->tint, A->tnbr, A->tgrid, A->tdt, A->dts, A->bbuf, A->kbuf, A->pbuf, A->wkbuf,
                  A->rcnt, A->rstart, A->rlist, A->spart, A->apart, A->alpha_acc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(A->slot);
  if (A->ctx) sph_destroy(A->ctx);
}

StateView view13(double* base, int64_t stride, int64_t* id) {
  StateView v;
  double** f[13] = {&v.x, &v.y, &v.z, &v.vx, &v.vy, &v.vz, &v.vxh, &v.vyh, &v.vzh, &v.h,
                    &v.m, &v.u, &v.du_prev};
  for (int k = 0; k < 13; ++k) *f[k] = base + (size_t)k * stride;
  v.id = id;
  return v;
}

Bar bar_of(double* base, int64_t stride) {
  Bar b;
  double** f[11] = {&b.x, &b.y, &b.z, &b.vx, &b.vy, &b.vz, &b.vxh, &b.vyh, &b.vzh, &b.u, &b.dup};
  for (int k = 0; k < 11; ++k) *f[k] = base + (size_t)k * stride;
  return b;
}

inline int grid_for(int64_t n, int sm, int threads, int per_sm) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sm * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Copies the 13 state arrays + ids between two stride layouts.
cudaError_t copy_state13(const StateView& dst, const StateView& src, int64_t n, cudaStream_t st) {
  double* d[13] = {dst.x, dst.y, dst.z, dst.vx, dst.vy, dst.vz, dst.vxh, dst.vyh, dst.vzh,
                   dst.h, dst.m, dst.u, dst.du_prev};
  const double* s[13] = {src.x, src.y, src.z, src.vx, src.vy, src.vz, src.vxh, src.vyh,
                         src.vzh, src.h, src.m, src.u, src.du_prev};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 13 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(d[k], s[k], sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && dst.id && src.id)
    e = cudaMemcpyAsync(dst.id, src.id, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                        st);
  return e;
}

sph_state state_of(const StateView& v, int64_t n) {
  sph_state s;
  memset(&s, 0, sizeof(s));
  s.x = v.x;
  s.y = v.y;
  s.z = v.z;
  s.vx = v.vx;
  s.vy = v.vy;
  s.vz = v.vz;
  s.vxh = v.vxh;
  s.vyh = v.vyh;
  s.vzh = v.vzh;
  s.h = v.h;
  s.m = v.m;
  s.u = v.u;
  s.du_prev = v.du_prev;
  s.id = v.id;
  s.n = n;
  return s;
}

struct Redirect {
  sph_ctx* c;
  StateView s;
  int32_t *perm, *nn;
  uint32_t* nbr;
  Grid* grid;
  Redirect(sph_ctx* ctx, const Slot& sl) : c(ctx) {
    s = c->s;
    perm = c->perm;
    nn = c->nn;
    nbr = c->nbr;
    grid = c->grid;
    c->s = sl.s;
    c->perm = sl.perm;
    c->nn = sl.nn;
    c->nbr = sl.nbr;
    c->grid = sl.grid;
  }
  ~Redirect() {
    c->s = s;
    c->perm = perm;
    c->nn = nn;
    c->nbr = nbr;
    c->grid = grid;
  }
};

// One forward step of the working state; recorded into slot j when j >= 0.
int run_step(sph_adj* A, int k, int j, cudaStream_t st) {
  sph_state s = A->W;
  int rc;
  if (j >= 0) {
    const Slot& sl = A->slot[j];
    s.rho = sl.rho;
    s.p = sl.p;
    s.c = sl.c;
    s.iad = sl.iad;
    s.omega = sl.omega;  // written by the density pass when params.gradh = 1
    Redirect r(A->ctx, sl);
    rc = sph_step(A->ctx, &s, A->dt_dev, st);
    if (rc != SPH_OK) return aerr(A, rc, "step %d: %s", k, sph_last_error(A->ctx));
    cudaError_t e = cudaMemcpyAsync(sl.dtp, A->ctx->diag + 8, sizeof(double),
                                    cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sl.dtp + 1, A->ctx->diag + 12, sizeof(double), cudaMemcpyDeviceToDevice,
                          st);
    if (e != cudaSuccess) return acuda(A, e, "tape dt");
  } else {
    rc = sph_step(A->ctx, &s, A->dt_dev, st);
    if (rc != SPH_OK) return aerr(A, rc, "step %d: %s", k, sph_last_error(A->ctx));
  }
  cudaError_t e = cudaMemcpyAsync(A->dts + k, A->ctx->diag + 8, sizeof(double),
                                  cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return acuda(A, e, "dt record");
  return SPH_OK;
}

int seg_len(const sph_adj* A, int seg) {
  const int first = seg * A->every;
  const int last = first + A->every < A->steps ? first + A->every : A->steps;
  return last - first;
}

// Restores checkpoint seg into the working state and records its steps.
int record_segment(sph_adj* A, int seg, cudaStream_t st) {
  const int64_t n = A->n;
  StateView wv = view13(A->wbuf, A->n_max, A->wid);
  StateView cv = view13(A->cbuf + (size_t)seg * 13 * A->n_max, A->n_max,
                        A->cid + (size_t)seg * A->n_max);
  cudaError_t e = copy_state13(wv, cv, n, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(A->dt_dev, A->cdt + seg, sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return acuda(A, e, "checkpoint restore");
  const int L = seg_len(A, seg);
  for (int j = 0; j < L; ++j) {
    int rc = run_step(A, seg * A->every + j, j, st);
    if (rc != SPH_OK) return rc;
  }
  A->tape_seg = seg;
  return SPH_OK;
}

int build_rev(sph_adj* A, const Slot& sl, cudaStream_t st) {
  const int64_t n = A->n;
  const int mb = A->prm.max_nb;
  cudaError_t e = cudaMemsetAsync(A->rcnt, 0, sizeof(int32_t) * (size_t)n, st);
  if (e != cudaSuccess) return acuda(A, e, "reverse lists");
  const int g = grid_for(n, A->sm_count, 256, 16);
  k_rev_count<<<g, 256, 0, st>>>(sl.nn, sl.nbr, mb, n, A->rcnt);
  sph::scan::exclusive_scan(A->rcnt, n, A->spart, A->rstart, st);
  e = cudaMemsetAsync(A->rcnt, 0, sizeof(int32_t) * (size_t)n, st);
  if (e != cudaSuccess) return acuda(A, e, "reverse lists");
  k_rev_fill<<<g, 256, 0, st>>>(sl.nn, sl.nbr, mb, n, A->rstart, A->rcnt, A->rlist);
  k_rev_sort<<<grid_for(n, A->sm_count, kSortWarps, 32), kSortWarps * 32, 0, st>>>(A->rstart, n,
                                                                                 A->rlist);
  A->launches += 7;
  e = cudaGetLastError();
  if (e != cudaSuccess) return acuda(A, e, "reverse-list launch");
  return SPH_OK;
}

Consts consts_of(const sph_adj* A) {
  Consts k;
  k.gamma = A->prm.gamma;
  k.alpha = A->alpha;
  k.Bn = sph_kernel_norm(A->ctx);
  k.sinc_n = (int)A->prm.sinc_n;
  k.max_nb = A->prm.max_nb;
  k.gradh = A->prm.gradh;
  return k;
}

Rev rev_of(sph_adj* A) {
  Rev r;
  r.cnt = A->rcnt;
  r.start = A->rstart;
  r.list = A->rlist;
  return r;
}

// Reverse of recorded step j: q (after the step) -> pnext (before it).
int reverse_step(sph_adj* A, int j, cudaStream_t st) {
  const Slot& sl = A->slot[j];
  int rc = build_rev(A, sl, st);
  if (rc != SPH_OK) return rc;
  const int64_t n = A->n;
  const Consts kc = consts_of(A);
  const int g = grid_for(n, A->sm_count, kThreads, 8);
  const int ga = g < kAlphaBlocks ? g : kAlphaBlocks;
  A->pb.stride = n;
  k_adj_prep<<<g, kThreads, 0, st>>>(sl, A->pr, n, kc.Bn, kc.gradh);
  k_adj_momentum_a<<<ga, kThreads, 0, st>>>(sl, A->pr, A->q, A->w, A->pb, n, kc, A->apart);
  k_alpha_sum<<<1, 32, 0, st>>>(A->apart, ga, A->alpha_acc);
  k_adj_momentum_b<<<g, kThreads, 0, st>>>(sl, A->w, A->pb, rev_of(A), n, kc);
  k_adj_iad<<<g, kThreads, 0, st>>>(sl, A->pr, A->w, A->pb, rev_of(A), n, kc);
  if (kc.gradh)
    k_adj_density<true, true><<<g, kThreads, 0, st>>>(sl, A->pr, A->w, A->pb, rev_of(A), A->pnext,
                                                      n, kc);
  else
    k_adj_density<true, false><<<g, kThreads, 0, st>>>(sl, A->pr, A->w, A->pb, rev_of(A),
                                                       A->pnext, n, kc);
  A->launches += 6;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return acuda(A, e, "reverse-step launch");
  const Bar t = A->q;
  A->q = A->pnext;
  A->pnext = t;
  return SPH_OK;
}

}  // namespace

extern "C" {

int sph_adjoint_init(const sph_params* params, int64_t n_max, int steps, int checkpoint_every,
                     sph_adj** out) {
  if (!out) return SPH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params || params->precision != SPH_FP64 || steps < 1 || checkpoint_every < 1 ||
      checkpoint_every > steps || n_max < 1 || n_max > sph::kMaxParticles)
    return SPH_ERR_INVALID_ARG;
  if (params->max_nb > (1 << kKBits)) return SPH_ERR_INVALID_ARG;
  // the reverse kernels differentiate the exact kernel (the table's is not built)
  if (params->kernel_mode != SPH_KERNEL_EXACT) return SPH_ERR_INVALID_ARG;
  sph_adj* A = (sph_adj*)calloc(1, sizeof(sph_adj));
  if (!A) return SPH_ERR_OOM;
  int rc = sph_init(params, n_max, &A->ctx);
  if (rc != SPH_OK) {
    free(A);
    return rc;
  }
  A->prm = *params;
  A->n_max = n_max;
  A->steps = steps;
  A->every = checkpoint_every;
  A->nseg = (steps + checkpoint_every - 1) / checkpoint_every;
  A->tape_seg = -1;
  A->sm_count = A->ctx->sm_count;
  const int nslot = checkpoint_every + 1;
  const size_t N = (size_t)n_max, mb = (size_t)params->max_nb;
  cudaError_t e = cudaSuccess;
#define AM(p, cnt) \
  if (e == cudaSuccess) e = amalloc(A, &(p), (size_t)(cnt))
  AM(A->wbuf, 26 * N);  // 13 state + rho p c + iad 6 + ax ay az du
  AM(A->wid, N);
  AM(A->dt_dev, 1);
  AM(A->cbuf, (size_t)A->nseg * 13 * N);
  AM(A->cid, (size_t)A->nseg * N);
  AM(A->cdt, A->nseg);
  AM(A->tbuf, (size_t)nslot * 23 * N);  // 13 sorted state + rho p c + iad 6 + omega
  AM(A->tid, (size_t)nslot * N);
  AM(A->tint, (size_t)nslot * 2 * N);
  AM(A->tnbr, (size_t)nslot * N * mb);
  AM(A->tgrid, nslot);
  AM(A->tdt, 2 * nslot);
  AM(A->dts, steps);
  AM(A->bbuf, 22 * N);
  AM(A->kbuf, 27 * N);  // Work: z 11 + X, ir, c + C 6 + rho = 21; Prep 5; G 1
  AM(A->pbuf, kRec * N * mb);
  AM(A->wkbuf, N * mb);
  AM(A->rcnt, N);
  AM(A->rstart, N + 1);
  AM(A->rlist, N * mb);
  AM(A->spart, (N + kScanItems - 1) / kScanItems + 1);
  AM(A->apart, kAlphaBlocks);
  AM(A->alpha_acc, 1);
#undef AM
  A->slot = (Slot*)calloc(nslot, sizeof(Slot));
  if (e != cudaSuccess || !A->slot) {
    rc = e != cudaSuccess ? acuda(A, e, "sph_adjoint_init") : SPH_ERR_OOM;
    free_adj(A);
    free(A);
    return rc == SPH_OK ? SPH_ERR_OOM : rc;
  }
  // working state
  StateView wv = view13(A->wbuf, N, A->wid);
  A->W = state_of(wv, 0);
  A->W.rho = A->wbuf + 13 * N;
  A->W.p = A->wbuf + 14 * N;
  A->W.c = A->wbuf + 15 * N;
  A->W.iad = A->wbuf + 16 * N;
  A->W.ax = A->wbuf + 22 * N;
  A->W.ay = A->wbuf + 23 * N;
  A->W.az = A->wbuf + 24 * N;
  A->W.du = A->wbuf + 25 * N;
  for (int j = 0; j < nslot; ++j) {
    Slot& sl = A->slot[j];
    double* base = A->tbuf + (size_t)j * 23 * N;
    sl.s = view13(base, N, A->tid + (size_t)j * N);
    sl.rho = base + 13 * N;
    sl.p = base + 14 * N;
    sl.c = base + 15 * N;
    sl.iad = base + 16 * N;
    sl.omega = base + 22 * N;
    sl.perm = A->tint + (size_t)j * 2 * N;
    sl.nn = A->tint + (size_t)j * 2 * N + N;
    sl.nbr = A->tnbr + (size_t)j * N * mb;
    sl.grid = A->tgrid + j;
    sl.dtp = A->tdt + 2 * j;
  }
  A->q = bar_of(A->bbuf, N);
  A->pnext = bar_of(A->bbuf + 11 * N, N);
  A->w.z = bar_of(A->kbuf, N);
  A->w.Xb = A->kbuf + 11 * N;
  A->w.irb = A->kbuf + 12 * N;
  A->w.cb = A->kbuf + 13 * N;
  A->w.Cb = A->kbuf + 14 * N;
  A->w.rhob = A->kbuf + 20 * N;
  A->pb.rec = A->pbuf;
  A->pb.wk = A->wkbuf;
  A->pb.stride = (int64_t)N;
  A->pr.hinv2 = A->kbuf + 21 * N;
  A->pr.norm = A->kbuf + 22 * N;
  A->pr.ir = A->kbuf + 23 * N;
  A->pr.X = A->kbuf + 24 * N;
  A->pr.vol = A->kbuf + 25 * N;
  A->w.Gb = A->kbuf + 26 * N;
  *out = A;
  return SPH_OK;
}

void sph_adjoint_destroy(sph_adj* A) {
  if (!A) return;
  cudaDeviceSynchronize();
  free_adj(A);
  free(A);
}

int sph_adjoint_forward(sph_adj* A, const sph_state* s0, double dt_prev0, double alpha,
                        double* final_out, sph_stream_t stream) {
  if (!A) return SPH_ERR_INVALID_ARG;
  if (!s0 || !final_out) return aerr(A, SPH_ERR_INVALID_ARG, "NULL argument");
  if (s0->n < 1 || s0->n > A->n_max)
    return aerr(A, SPH_ERR_INVALID_ARG, "n = %lld outside [1, n_max = %lld]", (long long)s0->n,
                (long long)A->n_max);
  const double* req[13] = {s0->x, s0->y, s0->z, s0->vx, s0->vy, s0->vz, s0->vxh, s0->vyh,
                           s0->vzh, s0->h, s0->m, s0->u, s0->du_prev};
  for (const double* p : req)
    if (!p) return aerr(A, SPH_ERR_INVALID_ARG, "a state array is NULL");
  if (!(alpha >= 0.0)) return aerr(A, SPH_ERR_INVALID_ARG, "alpha must be >= 0");
  if (!(dt_prev0 >= 0.0)) return aerr(A, SPH_ERR_INVALID_ARG, "dt_prev0 must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = s0->n;
  A->n = n;
  A->alpha = alpha;
  A->have_forward = 0;
  A->tape_seg = -1;
  sph_params prm = A->prm;
  prm.alpha = alpha;
  int rc = sph_set_params(A->ctx, &prm);
  if (rc != SPH_OK) return aerr(A, rc, "%s", sph_last_error(A->ctx));
  // working state <- s0 with ids 0..n-1
  StateView src;
  src.x = s0->x;
  src.y = s0->y;
  src.z = s0->z;
  src.vx = s0->vx;
  src.vy = s0->vy;
  src.vz = s0->vz;
  src.vxh = s0->vxh;
  src.vyh = s0->vyh;
  src.vzh = s0->vzh;
  src.h = s0->h;
  src.m = s0->m;
  src.u = s0->u;
  src.du_prev = s0->du_prev;
  src.id = nullptr;
  StateView wv = view13(A->wbuf, A->n_max, A->wid);
  cudaError_t e = copy_state13(wv, src, n, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(A->dt_dev, &dt_prev0, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return acuda(A, e, "forward set-up");
  k_iota<<<grid_for(n, A->sm_count, 256, 8), 256, 0, st>>>(A->wid, n);
  A->launches += 1;
  A->W.n = n;
  uint32_t flags = 0;
  rc = sph_error_word(A->ctx, &flags);  // clear stale flags
  if (rc != SPH_OK) return aerr(A, rc, "%s", sph_last_error(A->ctx));
  const int last = A->nseg - 1;
  for (int k = 0; k < A->steps; ++k) {
    const int seg = k / A->every;
    if (k % A->every == 0) {
      StateView cv = view13(A->cbuf + (size_t)seg * 13 * A->n_max, A->n_max,
                            A->cid + (size_t)seg * A->n_max);
      e = copy_state13(cv, wv, n, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(A->cdt + seg, A->dt_dev, sizeof(double), cudaMemcpyDeviceToDevice,
                            st);
      if (e != cudaSuccess) return acuda(A, e, "checkpoint");
    }
    rc = run_step(A, k, seg == last ? k - seg * A->every : -1, st);
    if (rc != SPH_OK) return rc;
  }
  A->tape_seg = last;
  // final density pass, recorded into the last slot
  {
    const Slot& sf = A->slot[A->every];
    Redirect r(A->ctx, sf);
    sph_state s = A->W;
    rc = sph_find_neighbors(A->ctx, &s, stream);
    if (rc == SPH_OK) {
      s.rho = sf.rho;
      s.p = sf.p;
      s.c = sf.c;
      rc = sph_density(A->ctx, &s, stream);
    }
    if (rc != SPH_OK) return aerr(A, rc, "final density: %s", sph_last_error(A->ctx));
    k_final_out<<<grid_for(n, A->sm_count, 256, 8), 256, 0, st>>>(sf.s, sf.rho, n, final_out);
    A->launches += 1;
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return acuda(A, e, "forward");
  rc = sph_error_word(A->ctx, &flags);
  if (rc != SPH_OK) return aerr(A, rc, "%s", sph_last_error(A->ctx));
  if (flags & SPH_FLAG_NB_OVERFLOW)
    return aerr(A, SPH_ERR_NB_OVERFLOW, "a neighbour list exceeded max_nb (flags 0x%x)", flags);
  if (flags & SPH_FLAG_SINGULAR_IAD)
    return aerr(A, SPH_ERR_SINGULAR_IAD, "singular IAD matrix (flags 0x%x)", flags);
  if (flags & SPH_FLAG_NONFINITE)
    return aerr(A, SPH_ERR_NONFINITE, "non-finite result (flags 0x%x)", flags);
  if (flags & (SPH_FLAG_BAD_BOX | SPH_FLAG_CELL_OVERFLOW))
    return aerr(A, SPH_ERR_INVALID_ARG, "box or cell occupancy out of range (flags 0x%x)", flags);
  A->have_forward = 1;
  return SPH_OK;
}

int sph_adjoint_backward(sph_adj* A, const double* g_final, double* g_init, double* g_alpha,
                         sph_stream_t stream) {
  if (!A) return SPH_ERR_INVALID_ARG;
  if (!g_final || !g_init || !g_alpha) return aerr(A, SPH_ERR_INVALID_ARG, "NULL argument");
  if (!A->have_forward) return aerr(A, SPH_ERR_ORDER, "call sph_adjoint_forward first");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = A->n;
  const Consts kc = consts_of(A);
  const int g = grid_for(n, A->sm_count, kThreads, 8);
  cudaError_t e = cudaMemsetAsync(A->alpha_acc, 0, sizeof(double), st);
  if (e != cudaSuccess) return acuda(A, e, "backward set-up");
  // final density pass: seed, reverse of Eq. 1, back to the order before it
  const Slot& sf = A->slot[A->every];
  int rc = build_rev(A, sf, st);
  if (rc != SPH_OK) return rc;
  A->pb.stride = n;
  k_seed<<<g, kThreads, 0, st>>>(g_final, sf.s.id, n, A->w);
  k_adj_prep<<<g, kThreads, 0, st>>>(sf, A->pr, n, kc.Bn, 0);
  k_adj_density<false, false><<<g, kThreads, 0, st>>>(sf, A->pr, A->w, A->pb, rev_of(A), A->q, n,
                                                      kc);
  A->launches += 3;
  for (int seg = A->nseg - 1; seg >= 0; --seg) {
    if (A->tape_seg != seg) {
      rc = record_segment(A, seg, st);
      if (rc != SPH_OK) return rc;
      A->recomputed += seg_len(A, seg);
    }
    for (int j = seg_len(A, seg) - 1; j >= 0; --j) {
      rc = reverse_step(A, j, st);
      if (rc != SPH_OK) return rc;
    }
  }
  double* dst[11] = {g_init, g_init + n, g_init + 2 * n, g_init + 3 * n, g_init + 4 * n,
                     g_init + 5 * n, g_init + 6 * n, g_init + 7 * n, g_init + 8 * n,
                     g_init + 9 * n, g_init + 10 * n};
  const double* srcb[11] = {A->q.x, A->q.y, A->q.z, A->q.vx, A->q.vy, A->q.vz,
                            A->q.vxh, A->q.vyh, A->q.vzh, A->q.u, A->q.dup};
  for (int k = 0; k < 11 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(dst[k], srcb[k], sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice,
                        st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g_alpha, A->alpha_acc, sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return acuda(A, e, "backward");
  A->backwards += 1;
  return SPH_OK;
}

int sph_adjoint_info(const sph_adj* A, int64_t* out) {
  if (!A || !out) return SPH_ERR_INVALID_ARG;
  out[0] = A->bytes;
  out[1] = A->launches + sph_launch_count(A->ctx);
  out[2] = A->recomputed;
  out[3] = A->backwards;
  return SPH_OK;
}

int sph_adjoint_time_steps(sph_adj* A, double* dt) {
  if (!A || !dt) return SPH_ERR_INVALID_ARG;
  if (!A->have_forward) return aerr(A, SPH_ERR_ORDER, "call sph_adjoint_forward first");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(dt, A->dts, sizeof(double) * (size_t)A->steps, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return acuda(A, e, "sph_adjoint_time_steps");
  return SPH_OK;
}

const char* sph_adjoint_last_error(const sph_adj* A) { return A ? A->last_error : "no context"; }

}  // extern "C"
