// FP32-mixed pair sums over cell-staged candidates (SPH_PAIRS_STAGED).
//
// findNeighbors (section 4.1: b runs over the particles inside the kernel
// support |x_a - x_b| < 2 h_a) and the three pair sums of the same section
// (Eq. 1 density, the IAD matrix, Eqs. 2-5 momentum and energy) work cell by
// cell on the uniform Morton-ordered grid (cells of side >= 2 h_max, so every
// neighbour of a target lies in the target cell's 3x3x3 stencil).
//
// Search (k_find_mask, one warp per occupied cell).  The stencil candidates
// within reach of the cell's targets are staged in stencil order, exactly as
// the list-writing search does (sph_find.cuh: FP32 prefilter with a proven
// error margin, the FP64 criterion without fused multiply-adds inside the
// margin).  Instead of appending neighbour indices to per-particle lists it
// writes, per occupied cell,
//   meta[cell]  = (slot_base, mask_base, a0, S << 16 | na)
//   sent[slot_base + j], j < S           list entry (sph_tile.cuh) of the j-th
//                                        staged candidate
//   masks[mask_base + blk * na + t]      bit 63 - q set when staged candidate
//                                        64 blk + q is a neighbour of target t
//                                        (the target itself excluded)
// and the exact neighbour count nn.  Space is taken from two device counters
// (upper bounds: the stencil's particle count P for the entries, na ceil(P/64)
// for the masks), so the layout depends on scheduling but the contents do not.
//
// Pair passes (k_cellpass, one CTA of kPT threads per occupied cell at a time).
// The cell's staged candidate records are copied once into shared memory,
// with their cell shift applied, so separations are FP32 differences of
// positions relative to the target cell.  Each target's hit masks are
// expanded into a list of staged slots in shared memory; the target's sum is
// split over nsub = kPT / (targets) threads, thread s taking entries s,
// s + nsub, ..., and the nsub partial sums are added in a fixed order, so the
// result does not depend on scheduling.  Cells whose staged set or target set
// exceeds the shared-memory window are processed in windows and rounds; a
// target with more than kLC hits in a window is expanded in several passes.
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_find.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

namespace sph {

namespace {

using find::FindWarpSmem;
using find::FindWarpSmemT;
using find::kFar;
using find::kFindThreads;
using find::kFindWarps;
using find::kFindWindow;
using find::kTop;
using find::pair_index;

// ------------------------------------------------------------------ search --

// A cell is staged (hit masks) when its stencil holds at most kStagedMaxP
// particles, so a target's mask row is at most kStagedMaxP / 64 words and the
// mask buffer (kMaskWords per particle) cannot overflow; larger stencils (a
// few particles with a much larger h than the rest make every cell large) get
// int32 lists, marked by mask_base = kListForm.
constexpr int kStagedMaxP = 64 * kMaskWords;
constexpr uint32_t kListForm = 0xffffffffu;

struct MaskOut {
  uint4* meta;                  // per occupied cell
  uint32_t* sent;               // staged candidate entries
  unsigned long long* masks;    // hit masks
  unsigned long long* alloc;    // [0] entries taken, [1] mask words taken
  unsigned long long sent_cap;  // capacities of sent and masks
  unsigned long long mask_cap;
};

template <bool WRAP, int WIN>
__device__ __forceinline__ void find_cell_masks(const Grid& g, uint32_t cell, uint32_t code,
                                                const StateView& s,
                                                const float4* __restrict__ pos32,
                                                const uint32_t* tbl_start,
                                                const uint32_t* tbl_count, int32_t* nn,
                                                uint32_t* nbr, int max_nb, const MaskOut& mo,
                                                uint32_t* err,
                                                FindWarpSmemT<WIN>& W, unsigned long long& tested,
                                                unsigned long long& exact) {
  const int lane = threadIdx.x & 31;
  Stencil& S = W.S;
  const float esum = g.err32[0] + g.err32[1] + g.err32[2];
  const float esq = g.err32[0] * g.err32[0] + g.err32[1] * g.err32[1] + g.err32[2] * g.err32[2];
  build_stencil_warp(g, code, tbl_start, tbl_count, S);
  const int P = S.off[S.ncell];
  const int a0 = S.a0, na = S.na;
  bool ok = P <= kStagedMaxP;
  unsigned long long sb = 0, mb = 0;
  if (ok) {
    const unsigned long long nblk_max = (unsigned long long)((P + 63) >> 6);
    if (lane == 0) {
      sb = atomicAdd(mo.alloc + 0, (unsigned long long)P);
      mb = atomicAdd(mo.alloc + 1, (unsigned long long)na * nblk_max);
    }
    sb = __shfl_sync(0xffffffffu, sb, 0);
    mb = __shfl_sync(0xffffffffu, mb, 0);
    // cannot fail (sum of P <= 27 n, sum of na ceil(P/64) <= kMaskWords n); kept
    // as a guard
    ok = sb + (unsigned long long)P <= mo.sent_cap &&
         mb + (unsigned long long)na * nblk_max <= mo.mask_cap;
  }
  if (!ok) {
    // list form: the list-writing search of sph_find.cuh for this cell
    __syncwarp();
    find::find_cell<WRAP, WIN>(g, code, s, pos32, tbl_start, tbl_count, nn, nbr, max_nb, err,
                               W, tested, exact);
    if (lane == 0) mo.meta[cell] = make_uint4(0u, kListForm, (uint32_t)a0, (uint32_t)na & 0xffffu);
    __syncwarp();
    return;
  }
  const uint32_t slot_base = (uint32_t)sb, mask_base = (uint32_t)mb;
  // bounding box of the targets (cell-relative FP32) and their largest h
  {
    float bl[3] = {kFar, kFar, kFar}, bh[3] = {-kFar, -kFar, -kFar}, hm = 0.0f;
    for (int t = lane; t < na; t += 32) {
      const float4 p = pos32[a0 + t];
      bl[0] = fminf(bl[0], p.x);
      bl[1] = fminf(bl[1], p.y);
      bl[2] = fminf(bl[2], p.z);
      bh[0] = fmaxf(bh[0], p.x);
      bh[1] = fmaxf(bh[1], p.y);
      bh[2] = fmaxf(bh[2], p.z);
      hm = fmaxf(hm, p.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      for (int ax = 0; ax < 3; ++ax) {
        bl[ax] = fminf(bl[ax], __shfl_xor_sync(0xffffffffu, bl[ax], o));
        bh[ax] = fmaxf(bh[ax], __shfl_xor_sync(0xffffffffu, bh[ax], o));
      }
      hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
    }
    // the reach of the list-writing search: 2 h in FP32 can be below 2 h_a
    // by 2^-23 relative, each coordinate carries at most err32 per axis
    const float reach = 2.0f * hm * 1.0001f + 4.0f * esum;
    if (lane == 0) {
      for (int ax = 0; ax < 3; ++ax) {
        S.box_lo[ax] = bl[ax];
        S.box_hi[ax] = bh[ax];
      }
      S.reach2 = reach * reach;
    }
    __syncwarp();
  }

  int wn = 0;          // slots in the window; window slot i is staged slot 64 gb + i
  uint32_t gb = 0;     // staged block of the window's first 64 slots
  int gself = -1;      // staged slot of the target cell's first particle
  bool first = true;
  int sc = 0, j0 = 0;  // next source: stencil cell and particle within it
  const uint32_t lt = (1u << lane) - 1u;
  for (;;) {
    while (sc < S.ncell && wn + 32 <= WIN) {
      const int cnt = S.off[sc + 1] - S.off[sc];
      const bool own = sc == S.self_cell;
      if (own && j0 == 0) gself = 64 * (int)gb + wn;
      const int st = S.start[sc];
      const int j = j0 + lane;
      bool keep = false;
      float cx = 0.f, cy = 0.f, cz = 0.f;
      if (j < cnt) {
        const float4 p = pos32[st + j];
        cx = p.x + S.shift[sc][0];
        cy = p.y + S.shift[sc][1];
        cz = p.z + S.shift[sc][2];
        if (WRAP || own) {
          keep = true;
        } else {
          const float dx = fmaxf(fmaxf(S.box_lo[0] - cx, cx - S.box_hi[0]), 0.0f);
          const float dy = fmaxf(fmaxf(S.box_lo[1] - cy, cy - S.box_hi[1]), 0.0f);
          const float dz = fmaxf(fmaxf(S.box_lo[2] - cz, cz - S.box_hi[2]), 0.0f);
          keep = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < S.reach2;
        }
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int q = wn + __popc(bal & lt);
        const int pq = pair_index(q);
        W.cx[pq] = cx;
        W.cy[pq] = cy;
        W.cz[pq] = cz;
        const uint32_t e = entry_make(S.scode[sc], st + j);
        W.entry[q] = e;
        mo.sent[slot_base + 64u * gb + (uint32_t)q] = e;
      }
      wn += __popc(bal);
      j0 += 32;
      if (j0 >= cnt) {
        ++sc;
        j0 = 0;
      }
    }
    const bool done = sc >= S.ncell;
    // full blocks now; the partial last block once the stencil is exhausted
    const int nblk = done ? (wn + 63) >> 6 : wn >> 6;
    if (done) {
      for (int i = wn + lane; i < 64 * nblk; i += 32) {
        const int q = pair_index(i);
        W.cx[q] = kFar;
        W.cy[q] = kFar;
        W.cz[q] = kFar;
      }
    }
    __syncwarp();
    const int nproc = done ? wn : 64 * nblk;  // real slots processed now
    for (int t0 = 0; t0 < na; t0 += 32) {
      const int t = t0 + lane;
      const bool active = t < na;
      const int a = a0 + (active ? t : 0);
      const float4 pa = pos32[a];
      const float two_h = 2.0f * pa.w;
      const float lim = two_h * two_h;
      const float margin = 2.0f * (2.0f * two_h * esum + esq + 4.76837158203125e-07f * lim);
      const float lo_lim = lim - margin, hi_lim = lim + margin;
      const float2 npx = make_float2(-pa.x, -pa.x), npy = make_float2(-pa.y, -pa.y),
                   npz = make_float2(-pa.z, -pa.z);
      const int gs = (active && gself >= 0) ? gself + t : -1;  // own staged slot
      int k = (first || !active) ? 0 : nn[a];
      for (int jb = 0; jb < nblk; ++jb) {
        uint64_t hit, unc;
        find::block_masks<WRAP>(g, W.cx + 64 * jb, W.cy + 64 * jb, W.cz + 64 * jb, npx, npy,
                                npz, lo_lim, hi_lim, hit, unc);
        while (unc) {  // inside the margin: the exact FP64 criterion
          const int q = __clzll((long long)unc);
          unc ^= kTop >> q;
          const int b = entry_index(W.entry[64 * jb + q]);
          if (exact_neighbor(g, s.x[a], s.y[a], s.z[a], s.h[a], s.x[b], s.y[b], s.z[b]))
            hit |= kTop >> q;
          ++exact;
        }
        const int gblk = (int)gb + jb;
        if (gs >= 0 && (gs >> 6) == gblk) hit &= ~(kTop >> (gs & 63));
        if (active) {
          mo.masks[mask_base + (uint32_t)gblk * (uint32_t)na + (uint32_t)t] = hit;
          k += __popcll(hit);
        }
      }
      if (active) {
        nn[a] = k;
        if (k > max_nb) raise_flag(err, SPH_FLAG_NB_OVERFLOW);
        const bool self_here = gs >= 0 && gs >= 64 * (int)gb && gs < 64 * (int)gb + nproc;
        tested += (unsigned long long)nproc - (self_here ? 1 : 0);
      }
    }
    __syncwarp();
    first = false;
    if (done) break;
    // carry the partial block (slots 64 nblk .. wn - 1) to the window's front
    const int rem = wn - 64 * nblk;
    if (rem > 0) {
      for (int i = lane; i < 64; i += 32) {
        W.cx[i] = W.cx[64 * nblk + i];
        W.cy[i] = W.cy[64 * nblk + i];
        W.cz[i] = W.cz[64 * nblk + i];
        W.entry[i] = W.entry[64 * nblk + i];
      }
    }
    gb += (uint32_t)nblk;
    wn = rem;
    __syncwarp();
  }
  if (lane == 0) {
    const uint32_t staged = 64u * gb + (uint32_t)wn;
    mo.meta[cell] = make_uint4(slot_base, mask_base, (uint32_t)a0,
                               (staged << 16) | ((uint32_t)na & 0xffffu));
  }
  __syncwarp();
}

// Capped at 128 registers so that four CTAs stay resident per SM.
template <bool WRAP>
__global__ void __launch_bounds__(kFindThreads, 4) k_find_mask(
    const Grid* gp, StateView s, const float4* __restrict__ pos32, const uint32_t* occ,
    const uint32_t* tbl_start, const uint32_t* tbl_count, int32_t* nn, uint32_t* nbr, int max_nb,
    MaskOut mo, uint32_t* err, unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  FindWarpSmem& W = reinterpret_cast<FindWarpSmem*>(smem_raw)[warp];
  const Grid g = *gp;
  if ((g.wrap32 != 0) != WRAP) return;
  unsigned long long tested = 0, exact = 0;
  const uint32_t gw = blockIdx.x * kFindWarps + warp, nw = gridDim.x * kFindWarps;
  for (uint32_t cell = gw; cell < g.n_occ; cell += nw)
    find_cell_masks<WRAP, kFindWindow>(g, cell, occ[cell], s, pos32, tbl_start, tbl_count, nn,
                                       nbr, max_nb, mo, err, W, tested, exact);
  for (int o = 16; o > 0; o >>= 1) {
    tested += __shfl_xor_sync(0xffffffffu, tested, o);
    exact += __shfl_xor_sync(0xffffffffu, exact, o);
  }
  if (lane == 0) {
    atomicAdd(stats + 0, tested);
    atomicAdd(stats + 1, exact);
  }
}

// ------------------------------------------------------------- pair passes --

constexpr int kPT = 256;        // threads per CTA (pair passes)
constexpr int kTR = 64;         // targets per round
constexpr int kLC = 128;        // list entries per target and expansion pass
constexpr int kLS = kLC + 2;    // list row stride (uint16): rows start in different banks
constexpr int kMaxSub = 32;     // threads sharing one target, at most

__device__ __forceinline__ float wrap32(float d, const Grid& g, int ax) {
  if (d > g.halfL32[ax])
    d -= g.L32[ax];
  else if (d < -g.halfL32[ax])
    d += g.L32[ax];
  return d;
}

// Separation b - a of two positions relative to the target's cell; the FP32
// minimum image is needed only on periodic axes with fewer than 3 cells.
__device__ __forceinline__ void sep(const Grid& g, float bx, float by, float bz, float ax_,
                                    float ay, float az, float& dx, float& dy, float& dz) {
  dx = bx - ax_;
  dy = by - ay;
  dz = bz - az;
  if (g.wrap32) {
    if (g.periodic[0]) dx = wrap32(dx, g, 0);
    if (g.periodic[1]) dy = wrap32(dy, g, 1);
    if (g.periodic[2]) dz = wrap32(dz, g, 2);
  }
}

// S(t)^n (t = v^2; the exact kernel's polynomial, or the table), B_n / h^3
// factored out of the sums.
__device__ __forceinline__ float s_pow(float t, int n, const float2* tab) {
  return tab ? kernel_w32_tab(t, 1.0f, tab) : kernel_w32(t, 1.0f, n);
}

// --- density + EOS (Eq. 1, self term included) ---
struct DensityPass {
  static constexpr int kWin = 1024;   // staged slots held in shared memory
  static constexpr int kRecBytes = 16;
  static constexpr int kV = 2;        // reduced values: sum m S^n, grad-h sum
  static constexpr int kMinBlocks = 4;
  static constexpr int kStageU = 4;   // staged records loaded per thread at once
  const float4* rec_d;   // (offset, m) per particle
  const float4* pos32;   // (offset, h)
  const double* u;
  OutView o;
  float4* rec_i;         // out: (offset, m / rho)
  float4* recA;          // out: (offset, 1 / h^2)
  float4* recQ;          // out: (B_n / h^3, X, c, 1 / rho)
  const float2* ktab;
  float Bn;
  int sinc_n;
  double gamma;
  int gradh;
  uint32_t* err;

  struct Target {
    float x, y, z, hinv2;
  };
  struct Rec {
    float4 r;  // position relative to the target's cell, m
  };
  __device__ Rec load(uint32_t e, const Grid& g) const {
    float sx, sy, sz;
    entry_shift(e, g, sx, sy, sz);
    const float4 r = rec_d[entry_index(e)];
    return {make_float4(r.x + sx, r.y + sy, r.z + sz, r.w)};
  }
  static __device__ void store(float4* rec, int j, const Rec& r) { rec[j] = r.r; }
  static __device__ Rec fetch(const float4* rec, int j) { return {rec[j]}; }
  __device__ void load_target(int64_t a, Target& T) const {
    const float4 p = pos32[a];
    T.x = p.x;
    T.y = p.y;
    T.z = p.z;
    T.hinv2 = 1.0f / (p.w * p.w);
  }
  __device__ void pair(const Target& T, const Rec& R, const Grid& g, float* acc) const {
    const float4 r = R.r;
    float dx, dy, dz;
    sep(g, r.x, r.y, r.z, T.x, T.y, T.z, dx, dy, dz);
    const float tt = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) * T.hinv2;
    acc[0] = fmaf(r.w, s_pow(tt, sinc_n, ktab), acc[0]);
    if (gradh) acc[1] = fmaf(r.w, kernel_tdw32(tt, 1.0f, sinc_n), acc[1]);
  }
  __device__ void finish(int64_t a, const float* acc) const {
    const float4 p = pos32[a];
    const float hinv2 = 1.0f / (p.w * p.w);
    const float norm = Bn * hinv2 / p.w;
    const float ma = rec_d[a].w;
    const float rho = norm * (ma + acc[0]);  // self term: S(0)^n = 1
    const double rho64 = (double)rho;
    const double pr = (gamma - 1.0) * rho64 * u[a];
    const double c = sqrt(gamma * pr / rho64);
    o.rho[a] = rho64;
    o.p[a] = pr;
    o.c[a] = c;
    const float inv_rho = 1.0f / rho;
    rec_i[a] = make_float4(p.x, p.y, p.z, ma * inv_rho);
    recA[a] = make_float4(p.x, p.y, p.z, hinv2);
    double X = pr / (rho64 * rho64);
    if (gradh) {
      const double omega = -2.0 * (double)(norm * acc[1]) / (3.0 * rho64);
      X /= omega;
      if (o.omega) o.omega[a] = omega;
    }
    recQ[a] = make_float4(norm, (float)X, (float)c, inv_rho);
    if (!isfinite(rho64) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
  }
};

// --- IAD: tau_a and C_a = tau_a^{-1} ---
struct IadPass {
  static constexpr int kWin = 1024;
  static constexpr int kRecBytes = 16;
  static constexpr int kV = 6;
  static constexpr int kMinBlocks = 4;
  static constexpr int kStageU = 4;
  const float4* rec_i;   // (offset, m / rho)
  const float4* recA;    // (offset, 1 / h^2)
  const float4* recQ;    // (B_n / h^3, ...)
  OutView o;
  float4* recC;          // out: (C00, C01, C02, C11)
  float2* recC2;         // out: (C12, C22)
  const float2* ktab;
  int sinc_n;
  uint32_t* err;

  struct Target {
    float x, y, z, hinv2, inv_h;
  };
  struct Rec {
    float4 r;  // position relative to the target's cell, m / rho
  };
  __device__ Rec load(uint32_t e, const Grid& g) const {
    float sx, sy, sz;
    entry_shift(e, g, sx, sy, sz);
    const float4 r = rec_i[entry_index(e)];
    return {make_float4(r.x + sx, r.y + sy, r.z + sz, r.w)};
  }
  static __device__ void store(float4* rec, int j, const Rec& r) { rec[j] = r.r; }
  static __device__ Rec fetch(const float4* rec, int j) { return {rec[j]}; }
  __device__ void load_target(int64_t a, Target& T) const {
    const float4 p = recA[a];
    T.x = p.x;
    T.y = p.y;
    T.z = p.z;
    T.hinv2 = p.w;
    T.inv_h = sqrtf(p.w);
  }
  __device__ void pair(const Target& T, const Rec& R, const Grid& g, float* acc) const {
    const float4 r = R.r;
    float dx, dy, dz;
    sep(g, r.x, r.y, r.z, T.x, T.y, T.z, dx, dy, dz);
    const float tt = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) * T.hinv2;
    // separation scaled by 1/h_a keeps tau of order one in FP32
    dx *= T.inv_h;
    dy *= T.inv_h;
    dz *= T.inv_h;
    const float w = r.w * s_pow(tt, sinc_n, ktab);
    const float wx = w * dx, wy = w * dy, wz = w * dz;
    acc[0] = fmaf(wx, dx, acc[0]);
    acc[1] = fmaf(wx, dy, acc[1]);
    acc[2] = fmaf(wx, dz, acc[2]);
    acc[3] = fmaf(wy, dy, acc[3]);
    acc[4] = fmaf(wy, dz, acc[4]);
    acc[5] = fmaf(wz, dz, acc[5]);
  }
  __device__ void finish(int64_t a, const float* acc) const {
    const float hinv2 = recA[a].w;
    const float norm = recQ[a].x;
    const float t00 = norm * acc[0], t01 = norm * acc[1], t02 = norm * acc[2];
    const float t11 = norm * acc[3], t12 = norm * acc[4], t22 = norm * acc[5];
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
    recC[a] = make_float4(Cm[0], Cm[1], Cm[2], Cm[3]);
    recC2[a] = make_float2(Cm[4], Cm[5]);
    double* out = o.iad + 6 * a;
    for (int q = 0; q < 6; ++q) out[q] = (double)Cm[q];
  }
};

// --- momentum and energy with artificial viscosity (Eqs. 2-5) ---
struct MomentumPass {
  static constexpr int kWin = 768;
  static constexpr int kRecBytes = 72;  // four float4 planes and one float2 plane
  static constexpr int kV = 4;
  static constexpr int kMinBlocks = 3;
  static constexpr int kStageU = 2;
  const float4* recA;    // (offset, 1 / h^2)
  const float4* recV;    // (v, m)
  const float4* recQ;    // (B_n / h^3, X = P / (Omega rho^2), c, 1 / rho)
  const float4* recC;    // (C00, C01, C02, C11)
  const float2* recC2;   // (C12, C22)
  OutView o;
  const float2* ktab;
  int sinc_n;
  float alpha;
  uint32_t* err;

  struct Target {
    float4 p, v, q;
    float c00, c01, c02, c11, c12, c22;
  };
  // shared-memory planes of a window: A, V, Q, C (float4) then C2 (float2)
  static __device__ __forceinline__ float4* plane(float4* rec, int k) { return rec + k * kWin; }
  static __device__ __forceinline__ float2* plane2(float4* rec) {
    return reinterpret_cast<float2*>(rec + 4 * kWin);
  }
  struct Rec {
    float4 p, v, q, c;  // (position relative to the target's cell, 1/h^2), (v, m), Q, C
    float2 c2;
  };
  __device__ Rec load(uint32_t e, const Grid& g) const {
    float sx, sy, sz;
    entry_shift(e, g, sx, sy, sz);
    const int b = entry_index(e);
    const float4 p = recA[b];
    return {make_float4(p.x + sx, p.y + sy, p.z + sz, p.w), recV[b], recQ[b], recC[b], recC2[b]};
  }
  static __device__ void store(float4* rec, int j, const Rec& r) {
    plane(rec, 0)[j] = r.p;
    plane(rec, 1)[j] = r.v;
    plane(rec, 2)[j] = r.q;
    plane(rec, 3)[j] = r.c;
    plane2(rec)[j] = r.c2;
  }
  static __device__ Rec fetch(float4* rec, int j) {
    return {plane(rec, 0)[j], plane(rec, 1)[j], plane(rec, 2)[j], plane(rec, 3)[j],
            plane2(rec)[j]};
  }
  __device__ void load_target(int64_t a, Target& T) const {
    T.p = recA[a];
    T.v = recV[a];
    T.q = recQ[a];
    const float4 c = recC[a];
    const float2 c2 = recC2[a];
    T.c00 = c.x;
    T.c01 = c.y;
    T.c02 = c.z;
    T.c11 = c.w;
    T.c12 = c2.x;
    T.c22 = c2.y;
  }
  __device__ void pair(const Target& T, const Rec& R, const Grid& g, float* acc) const {
    // one pair of Eqs. 2-5 (x_ab = -d, d = x_b - x_a)
    const float4 b0 = R.p;
    float dx, dy, dz;
    sep(g, b0.x, b0.y, b0.z, T.p.x, T.p.y, T.p.z, dx, dy, dz);
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float4 b2 = R.q;
    const float Wa = T.q.x * s_pow(r2 * T.p.w, sinc_n, ktab);
    const float Wb = b2.x * s_pow(r2 * b0.w, sinc_n, ktab);  // clamped at t = 4 (S = 0)
    const float Cadx = fmaf(T.c02, dz, fmaf(T.c01, dy, T.c00 * dx));
    const float Cady = fmaf(T.c12, dz, fmaf(T.c11, dy, T.c01 * dx));
    const float Cadz = fmaf(T.c22, dz, fmaf(T.c12, dy, T.c02 * dx));
    const float4 b3 = R.c;
    const float2 b4 = R.c2;
    const float Cbdx = fmaf(b3.z, dz, fmaf(b3.y, dy, b3.x * dx));
    const float Cbdy = fmaf(b4.x, dz, fmaf(b3.w, dy, b3.y * dx));
    const float Cbdz = fmaf(b4.y, dz, fmaf(b4.x, dy, b3.z * dx));
    const float4 vb = R.v;
    const float vabx = T.v.x - vb.x, vaby = T.v.y - vb.y, vabz = T.v.z - vb.z;
    const float xv = -fmaf(dz, vabz, fmaf(dy, vaby, dx * vabx));
    // Eq. 5 without a branch: w_ab = x_ab.v_ab / r, Pi = 0 unless approaching
    const float w = xv * rsqrtf(r2);
    const float vsig = T.q.z + b2.z - 3.0f * w;
    const float Pi = xv < 0.0f ? -0.5f * alpha * vsig * w : 0.0f;
    const float ira = T.q.w, irb = b2.w;
    const float mb = vb.w;
    const float fa = mb * Wa * fmaf(0.5f * Pi, ira, T.q.y);
    const float fb = mb * Wb * fmaf(0.5f * Pi, irb, b2.y);
    acc[0] -= fmaf(fa, Cadx, fb * Cbdx);
    acc[1] -= fmaf(fa, Cady, fb * Cbdy);
    acc[2] -= fmaf(fa, Cadz, fb * Cbdz);
    const float vCa = fmaf(vabz, Cadz, fmaf(vaby, Cady, vabx * Cadx));
    const float vCb = fmaf(vabz, Cbdz, fmaf(vaby, Cbdy, vabx * Cbdx));
    acc[3] = fmaf(mb, fmaf(Wa * fmaf(0.25f * Pi, ira, T.q.y), vCa, 0.25f * Pi * irb * Wb * vCb),
                  acc[3]);
  }
  __device__ void finish(int64_t a, const float* acc) const {
    o.ax[a] = acc[0];
    o.ay[a] = acc[1];
    o.az[a] = acc[2];
    o.du[a] = acc[3];
    if (!isfinite(acc[0]) || !isfinite(acc[1]) || !isfinite(acc[2]) || !isfinite(acc[3]))
      raise_flag(err, SPH_FLAG_NONFINITE);
  }
};

// Shared memory of a pass: the records of a window, the expanded lists (also
// the reduction's partial sums), per-(target, block) hit counts and the
// targets' totals.
template <class Pass>
struct PassSmem {
  static constexpr int kWB = Pass::kWin / 64;
  static constexpr size_t kRec = (size_t)Pass::kWin * Pass::kRecBytes;
  static constexpr size_t kLists = (size_t)kTR * kLS * sizeof(uint16_t);
  static constexpr size_t kPart = (size_t)kPT * Pass::kV * sizeof(float);
  static constexpr size_t kListsOrPart = kLists > kPart ? kLists : kPart;
  static constexpr size_t kCnt = (size_t)kTR * kWB * sizeof(int);
  static constexpr size_t kBytes = kRec + ((kListsOrPart + 15) & ~(size_t)15) + kCnt +
                                   (size_t)kTR * sizeof(int);
  static_assert(kRec % 16 == 0, "record planes keep 16-byte alignment");
};

// Neighbour source of one pass launch.
struct Src {
  const uint4* meta;                 // per occupied cell
  const uint32_t* sent;              // staged candidate entries
  const unsigned long long* masks;   // hit masks
  const int32_t* nn;                 // list-form cells: counts and int32 lists
  const uint32_t* nbr;
  int max_nb;
};

template <class Pass>
__global__ void __launch_bounds__(kPT, Pass::kMinBlocks) k_cellpass(Pass pass, const Grid* gp,
                                                                    Src src) {
  using SM = PassSmem<Pass>;
  constexpr int U = Pass::kStageU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* rec = reinterpret_cast<float4*>(smem_raw);
  uint16_t* lists = reinterpret_cast<uint16_t*>(smem_raw + SM::kRec);
  float* part = reinterpret_cast<float*>(smem_raw + SM::kRec);
  int* cnt = reinterpret_cast<int*>(smem_raw + SM::kRec + ((SM::kListsOrPart + 15) & ~(size_t)15));
  int* tot = cnt + kTR * SM::kWB;
  const Grid g = *gp;
  const uint32_t n_occ = g.n_occ;
  const int tid = threadIdx.x;
  uint4 md_next = blockIdx.x < n_occ ? __ldg(src.meta + blockIdx.x) : make_uint4(0, 0, 0, 0);
  for (uint32_t cell = blockIdx.x; cell < n_occ; cell += gridDim.x) {
    const uint4 md = md_next;
    if (cell + gridDim.x < n_occ) md_next = __ldg(src.meta + cell + gridDim.x);
    const uint32_t slot_base = md.x, mask_base = md.y, a0 = md.z;
    const int S = (int)(md.w >> 16), na = (int)(md.w & 0xffffu);
    const bool list_form = mask_base == kListForm;
    int staged_w0 = -1;
    for (int r0 = 0; r0 < na; r0 += kTR) {
      const int nr = min(kTR, na - r0);
      int nsub = kPT / nr;
      if (nsub > kMaxSub) nsub = kMaxSub;
      const int t = tid / nsub, sub = tid - t * nsub;
      const bool active = t < nr;
      typename Pass::Target T;
      float acc[Pass::kV];
#pragma unroll
      for (int v = 0; v < Pass::kV; ++v) acc[v] = 0.0f;
      if (active) pass.load_target((int64_t)a0 + r0 + t, T);
      if (list_form) {
        // a cell whose stencil exceeds the staged form's limits: int32 lists,
        // neighbour records read from global memory
        if (active) {
          const int64_t a = (int64_t)a0 + r0 + t;
          const int c = min(src.nn[a], src.max_nb);
          const uint32_t* row = src.nbr + a * src.max_nb;
          for (int k = sub; k < c; k += nsub) pass.pair(T, pass.load(__ldg(row + k), g), g, acc);
        }
      }
      for (int w0 = 0; !list_form && w0 < S; w0 += Pass::kWin) {
        const int wn = min(Pass::kWin, S - w0);
        const int wb = (wn + 63) >> 6;
        if (w0 != staged_w0) {
          __syncthreads();  // the previous window's readers are done
          const uint32_t* es = src.sent + slot_base + (uint32_t)w0;
          for (int j0 = 0; j0 < wn; j0 += U * kPT) {
            uint32_t e[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int j = j0 + u * kPT + tid;
              e[u] = j < wn ? __ldg(es + j) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (j0 + u * kPT + tid < wn) Pass::store(rec, j0 + u * kPT + tid, pass.load(e[u], g));
          }
          staged_w0 = w0;
        }
        const uint32_t mrow = mask_base + (uint32_t)(w0 >> 6) * (uint32_t)na + (uint32_t)r0;
        for (int ep = 0;; ++ep) {
          __syncthreads();  // records staged; lists free
          for (int i = tid; i < nr * wb; i += kPT) {
            const int tt = i % nr, jb = i / nr;
            cnt[jb * kTR + tt] = __popcll(__ldg(src.masks + mrow + (uint32_t)jb * na + tt));
          }
          __syncthreads();
          for (int i = tid; i < nr * wb; i += kPT) {
            const int tt = i % nr, jb = i / nr;
            int pos = -ep * kLC;
            for (int j = 0; j < jb; ++j) pos += cnt[j * kTR + tt];
            if (jb == 0) {
              int sum = 0;
              for (int j = 0; j < wb; ++j) sum += cnt[j * kTR + tt];
              tot[tt] = sum;
            }
            uint64_t w = __ldg(src.masks + mrow + (uint32_t)jb * na + tt);
            uint16_t* row = lists + tt * kLS;
            while (w && pos < kLC) {
              const int q = __clzll((long long)w);
              w ^= kTop >> q;
              if (pos >= 0) row[pos] = (uint16_t)(64 * jb + q);
              ++pos;
            }
          }
          __syncthreads();
          if (active) {
            const int nl = min(tot[t] - ep * kLC, kLC);
            const uint16_t* row = lists + t * kLS;
            for (int k = sub; k < nl; k += nsub) pass.pair(T, Pass::fetch(rec, row[k]), g, acc);
          }
          const int more = __syncthreads_or(active && sub == 0 && tot[t] > (ep + 1) * kLC);
          if (!more) break;
        }
      }
      // the nsub partial sums of each target, added in a fixed order
      __syncthreads();
#pragma unroll
      for (int v = 0; v < Pass::kV; ++v) part[v * kPT + tid] = acc[v];
      __syncthreads();
      if (tid < nr) {
        float sm[Pass::kV];
#pragma unroll
        for (int v = 0; v < Pass::kV; ++v) {
          float x = 0.0f;
          for (int q = 0; q < nsub; ++q) x += part[v * kPT + tid * nsub + q];
          sm[v] = x;
        }
        pass.finish((int64_t)a0 + r0 + tid, sm);
      }
    }
  }
}

template <class Pass>
int pass_blocks(sph_ctx* ctx, int* cache) {
  if (!*cache) {  // once per context, on its device
    using SM = PassSmem<Pass>;
    cudaFuncSetAttribute(k_cellpass<Pass>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SM::kBytes);
    cudaFuncSetAttribute(k_cellpass<Pass>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cellpass<Pass>, kPT, SM::kBytes);
    *cache = (per_sm > 0 ? per_sm : 1) * ctx->sm_count;
  }
  return *cache;
}

template <class Pass>
void launch_pass(sph_ctx* ctx, const Pass& p, int* cache, cudaStream_t st) {
  const int blocks = pass_blocks<Pass>(ctx, cache);
  Src src;
  src.meta = ctx->cmeta;
  src.sent = ctx->sent;
  src.masks = ctx->masks;
  src.nn = ctx->nn;
  src.nbr = ctx->nbr;
  src.max_nb = ctx->prm.max_nb;
  k_cellpass<Pass><<<blocks, kPT, PassSmem<Pass>::kBytes, st>>>(p, ctx->grid, src);
  ctx->launches += 1;
}

// ----------------------------------------------------------------- export --

// Per particle: the neighbours' ids from its hit masks, sorted ascending
// (insertion sort), at most max_nb of them; counts = the exact count.
__device__ __forceinline__ void insert_sorted(int64_t* row, int m, int64_t v) {
  int k = m - 1;
  while (k >= 0 && row[k] > v) {
    row[k + 1] = row[k];
    --k;
  }
  row[k + 1] = v;
}

__global__ void k_export_masks(int64_t n, const int32_t* nn, const uint32_t* cell_of,
                               const uint4* meta, const uint32_t* sent,
                               const unsigned long long* masks, const uint32_t* nbr, int max_nb,
                               const int64_t* id, int32_t* counts, int64_t* ids) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    counts[a] = nn[a];
    const uint4 md = meta[cell_of[a]];
    int64_t* row = ids + a * max_nb;
    if (md.y == kListForm) {  // a list-form cell: its int32 list
      const int c = min(nn[a], max_nb);
      for (int k = 0; k < c; ++k) insert_sorted(row, k, id[entry_index(nbr[a * max_nb + k])]);
      continue;
    }
    const int S = (int)(md.w >> 16), na = (int)(md.w & 0xffffu);
    const int t = (int)(a - (int64_t)md.z);
    int m = 0;
    for (int blk = 0; 64 * blk < S; ++blk) {
      uint64_t w = masks[md.y + (uint32_t)blk * na + t];
      while (w && m < max_nb) {
        const int q = __clzll((long long)w);
        w ^= kTop >> q;
        insert_sorted(row, m, id[entry_index(sent[md.x + 64u * blk + q])]);
        ++m;
      }
    }
  }
}

inline OutView outs_with_omega(const OutView& o, int gradh) {
  OutView r = o;
  if (!gradh) r.omega = nullptr;
  return r;
}

}  // namespace

void launch_find_masks(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st) {
  (void)n;
  const size_t smem = kFindWarps * sizeof(FindWarpSmem);
  if (!ctx->find_mask_blocks) {  // once per context, on its device
    int per_sm = 0;
    cudaFuncSetAttribute(k_find_mask<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_find_mask<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_find_mask<false>, kFindThreads,
                                                  smem);
    ctx->find_mask_blocks = (per_sm > 0 ? per_sm : 1) * ctx->sm_count;
  }
  MaskOut mo;
  mo.meta = ctx->cmeta;
  mo.sent = ctx->sent;
  mo.masks = ctx->masks;
  mo.alloc = ctx->salloc;
  mo.sent_cap = (unsigned long long)ctx->sent_cap;
  mo.mask_cap = (unsigned long long)ctx->mask_cap;
  cudaMemsetAsync(ctx->salloc, 0, 2 * sizeof(unsigned long long), st);
  k_find_mask<false><<<ctx->find_mask_blocks, kFindThreads, smem, st>>>(
      ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start, ctx->tbl_count, ctx->nn, ctx->nbr,
      ctx->prm.max_nb, mo, ctx->err, ctx->stats);
  k_find_mask<true><<<ctx->find_mask_blocks, kFindThreads, smem, st>>>(
      ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start, ctx->tbl_count, ctx->nn, ctx->nbr,
      ctx->prm.max_nb, mo, ctx->err, ctx->stats);
  ctx->launches += 2;
}

void launch_density_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                           cudaStream_t st) {
  (void)n;
  DensityPass p;
  p.rec_d = ctx->rec_d;
  p.pos32 = ctx->pos32;
  p.u = s.u;
  p.o = outs_with_omega(o, ctx->prm.gradh);
  p.rec_i = ctx->rec_i;
  p.recA = ctx->recA;
  p.recQ = ctx->recQ;
  p.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab32 : nullptr;
  p.Bn = (float)ctx->Bn;
  p.sinc_n = (int)ctx->prm.sinc_n;
  p.gamma = ctx->prm.gamma;
  p.gradh = ctx->prm.gradh;
  p.err = ctx->err;
  launch_pass(ctx, p, &ctx->pass_blocks[0], st);
}

void launch_iad_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                       cudaStream_t st) {
  (void)s;
  (void)n;
  IadPass p;
  p.rec_i = ctx->rec_i;
  p.recA = ctx->recA;
  p.recQ = ctx->recQ;
  p.o = o;
  p.recC = ctx->recC;
  p.recC2 = ctx->recC2;
  p.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab32 : nullptr;
  p.sinc_n = (int)ctx->prm.sinc_n;
  p.err = ctx->err;
  launch_pass(ctx, p, &ctx->pass_blocks[1], st);
}

void launch_momentum_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                            cudaStream_t st) {
  (void)s;
  (void)n;
  MomentumPass p;
  p.recA = ctx->recA;
  p.recV = ctx->recV;
  p.recQ = ctx->recQ;
  p.recC = ctx->recC;
  p.recC2 = ctx->recC2;
  p.o = o;
  p.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab32 : nullptr;
  p.sinc_n = (int)ctx->prm.sinc_n;
  p.alpha = (float)ctx->prm.alpha;
  p.err = ctx->err;
  launch_pass(ctx, p, &ctx->pass_blocks[2], st);
}

void launch_export_masks(sph_ctx* ctx, const StateView& s, int64_t n, int32_t* counts,
                         int64_t* ids, cudaStream_t st) {
  int64_t b = (n + 127) / 128;
  if (b > (int64_t)ctx->sm_count * 32) b = ctx->sm_count * 32;
  if (b < 1) b = 1;
  k_export_masks<<<(int)b, 128, 0, st>>>(n, ctx->nn, ctx->cell_of, ctx->cmeta, ctx->sent,
                                         ctx->masks, ctx->nbr, ctx->prm.max_nb, s.id, counts,
                                         ids);
  ctx->launches += 1;
}

}  // namespace sph
