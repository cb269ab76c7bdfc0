// The neighbour search of one occupied cell by one warp (findNeighbors,
// section 4.1: b runs over the particles inside the kernel support
// |x_a - x_b| < 2 h_a), shared by the single-box kernel (sph_neighbors.cu) and
// the ensemble's persistent kernel (sph_ensemble.cu).
//
// The cell's stencil particles are staged in the warp's shared-memory window
// as FP32 positions relative to the cell's origin (offset to their own cell +
// the stencil shift).  Only candidates within reach of some target are staged:
// the distance from the candidate to the bounding box of the cell's targets
// must be below the largest 2 h_a among them (plus the FP32 error bound), which
// every neighbour of every target satisfies.  With cells of side >= 2 h_max this
// keeps about three quarters of the 27-cell stencil where h is near h_max and
// about half where h is smaller; the staged candidates keep their stencil-slot
// order, so the lists are the same sequences as without the filter.
// Lane t owns target t of the cell (32 at a time) and
// walks the staged candidates in blocks of 64, all lanes reading the same
// candidate pair (broadcast loads, paired FP32 arithmetic on candidates j and
// j + 32 of the block):
//   1. FP32 prefilter: r2_32 against (2 h_a)^2 within a margin M_a that
//      bounds the FP32 rounding of the separation (Grid::err32) and of the
//      squares; outside the margin the FP32 decision is exact;
//   2. inside the margin, the exact FP64 criterion (exact_neighbor), so lists
//      are bit-identical to r^2 < (2h)^2 evaluated in FP64 without FMA;
//   3. each lane appends its hits of the block, in slot order, from a 64-bit
//      hit mask.
// Lists are uint32 entries (particle index + cell-shift code, sph_tile.cuh),
// row-major per particle: nbr[a * max_nb + k], in stencil-slot order.
#pragma once

#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

namespace sph {
namespace find {

constexpr int kFindWarps = 4;
constexpr int kFindThreads = 32 * kFindWarps;
constexpr int kFindWindow = 512;   // staged candidates per warp and pass (8 KB; the
                                   // ensemble also instantiates smaller windows)
constexpr float kFar = 1.0e18f;    // position of padding slots (never a neighbour)

__device__ __forceinline__ float wrap_axis(float d, const Grid& g, int ax) {
  if (d > g.halfL32[ax])
    d -= g.L32[ax];
  else if (d < -g.halfL32[ax])
    d += g.L32[ax];
  return d;
}

// Shared-memory layout of a window: per block of 64 slots, the x (y, z)
// coordinates as 32 float2 pairs (slot q, slot q + 32), so one 8-byte load
// gives the pair processed by one paired FP32 instruction.
__device__ __forceinline__ int pair_index(int i) {
  const int blk = i >> 6, r = i & 63;
  return (blk << 6) + ((r & 31) << 1) + (r >> 5);
}

template <int WIN>
struct FindWarpSmemT {
  static_assert(WIN % 64 == 0, "the window holds whole blocks of 64 slots");
  Stencil S;
  // 16-byte aligned: the candidate arrays are read as float2 pairs
  alignas(16) float cx[WIN];
  alignas(16) float cy[WIN];
  alignas(16) float cz[WIN];
  uint32_t entry[WIN];  // list entry of each staged slot (sph_tile.cuh)
};
using FindWarpSmem = FindWarpSmemT<kFindWindow>;
static_assert(sizeof(FindWarpSmemT<128>) % 16 == 0 && sizeof(FindWarpSmem) % 16 == 0,
              "per-warp window must keep 16-byte alignment");

// Hit and margin masks of one block of 64 staged candidates for one target.
// The decisions r2 < lo and r2 < hi are read from the sign bits of r2 - lo and
// r2 - hi, with the limit folded into the first fused multiply-add (the margin
// is twice the error bound, so a strict "< hi" is as safe as "<= hi").  Each
// sign bit is shifted into its mask by one funnel shift, so slot s of the
// block ends at bit 63 - s (kTop >> s).
template <bool WRAP>
__device__ __forceinline__ void block_masks(const Grid& g, const float* cx, const float* cy,
                                            const float* cz, float2 npx, float2 npy, float2 npz,
                                            float lo_lim, float hi_lim, uint64_t& hit,
                                            uint64_t& unc) {
  const float2* X = reinterpret_cast<const float2*>(cx);
  const float2* Y = reinterpret_cast<const float2*>(cy);
  const float2* Z = reinterpret_cast<const float2*>(cz);
  const float2 nlo = make_float2(-lo_lim, -lo_lim);
  const float2 dlh = make_float2(lo_lim - hi_lim, lo_lim - hi_lim);
  uint32_t hA = 0, hB = 0, uA = 0, uB = 0;
#pragma unroll 8
  for (int q = 0; q < 32; ++q) {  // slots q (.x) and q + 32 (.y)
    float2 dx = __fadd2_rn(X[q], npx);
    float2 dy = __fadd2_rn(Y[q], npy);
    float2 dz = __fadd2_rn(Z[q], npz);
    if (WRAP) {
      if (g.periodic[0]) dx = make_float2(wrap_axis(dx.x, g, 0), wrap_axis(dx.y, g, 0));
      if (g.periodic[1]) dy = make_float2(wrap_axis(dy.x, g, 1), wrap_axis(dy.y, g, 1));
      if (g.periodic[2]) dz = make_float2(wrap_axis(dz.x, g, 2), wrap_axis(dz.y, g, 2));
    }
    float2 t = __ffma2_rn(dx, dx, nlo);   // r2 - lo
    t = __ffma2_rn(dy, dy, t);
    t = __ffma2_rn(dz, dz, t);
    const float2 u = __fadd2_rn(t, dlh);   // r2 - hi
    hA = __funnelshift_l(__float_as_uint(t.x), hA, 1);
    hB = __funnelshift_l(__float_as_uint(t.y), hB, 1);
    uA = __funnelshift_l(__float_as_uint(u.x), uA, 1);
    uB = __funnelshift_l(__float_as_uint(u.y), uB, 1);
  }
  hit = ((uint64_t)hA << 32) | hB;
  unc = (((uint64_t)uA << 32) | uB) & ~hit;
}

constexpr uint64_t kTop = 1ull << 63;

// Builds the lists of every target of occupied cell `code` (one warp; the
// warp owns W, a window of WIN staged slots).  Counts tested candidates and
// exact FP64 tests.
template <bool WRAP, int WIN = kFindWindow>
__device__ __forceinline__ void find_cell(const Grid& g, uint32_t code, const StateView& s,
                                          const float4* __restrict__ pos32,
                                          const uint32_t* tbl_start, const uint32_t* tbl_count,
                                          int32_t* nn, uint32_t* nbr, int max_nb, uint32_t* err,
                                          FindWarpSmemT<WIN>& W, unsigned long long& tested,
                                          unsigned long long& exact) {
  const int lane = threadIdx.x & 31;
  Stencil& S = W.S;
  const float esum = g.err32[0] + g.err32[1] + g.err32[2];
  const float esq = g.err32[0] * g.err32[0] + g.err32[1] * g.err32[1] + g.err32[2] * g.err32[2];
  build_stencil_warp(g, code, tbl_start, tbl_count, S);
  const int P = S.off[S.ncell];
  const int a0 = S.a0, na = S.na;
  if (P > kMaxSlots || S.maxpop > kMaxCellPop) {
    for (int t = lane; t < na; t += 32) nn[a0 + t] = 0;
    if (lane == 0) raise_flag(err, SPH_FLAG_CELL_OVERFLOW);
    __syncwarp();
    return;
  }
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
    // generous: 2 h in FP32 can be below 2 h_a by 2^-23 relative, and each
    // candidate and target coordinate carries at most err32 per axis
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

  int wn = 0;           // slots staged in the current window
  int wbase = 0;        // staged slots before the current window
  int gself = -1;       // staged index of the target cell's first particle
  bool first = true;
  int sc = 0, j0 = 0;   // next source: stencil cell and particle within it
  const uint32_t lt = (1u << lane) - 1u;
  for (;;) {
    // stage candidates within reach, cell by cell in stencil order, until the
    // window cannot take another 32 or the stencil is exhausted (the targets'
    // box and the reach in registers for this pass, each cell's values read
    // once for all its batches of 32)
    const float blx = S.box_lo[0], bly = S.box_lo[1], blz = S.box_lo[2];
    const float bhx = S.box_hi[0], bhy = S.box_hi[1], bhz = S.box_hi[2];
    const float reach2 = S.reach2;
    while (sc < S.ncell && wn + 32 <= WIN) {
      const int cnt = S.off[sc + 1] - S.off[sc];
      const bool own = sc == S.self_cell;
      if (own && j0 == 0) gself = wbase + wn;
      const int st = S.start[sc];
      const float shx = S.shift[sc][0], shy = S.shift[sc][1], shz = S.shift[sc][2];
      const uint32_t ecode = entry_make(S.scode[sc], 0);
      do {
        const int j = j0 + lane;
        bool keep = false;
        float cx = 0.f, cy = 0.f, cz = 0.f;
        if (j < cnt) {
          const float4 p = pos32[st + j];
          cx = p.x + shx;
          cy = p.y + shy;
          cz = p.z + shz;
          if (WRAP || own) {
            keep = true;
          } else {
            const float dx = fmaxf(fmaxf(blx - cx, cx - bhx), 0.0f);
            const float dy = fmaxf(fmaxf(bly - cy, cy - bhy), 0.0f);
            const float dz = fmaxf(fmaxf(blz - cz, cz - bhz), 0.0f);
            keep = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < reach2;
          }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int q = wn + __popc(bal & lt);
          const int pq = pair_index(q);
          W.cx[pq] = cx;
          W.cy[pq] = cy;
          W.cz[pq] = cz;
          W.entry[q] = ecode | (uint32_t)(st + j);
        }
        wn += __popc(bal);
        j0 += 32;
      } while (j0 < cnt && wn + 32 <= WIN);
      if (j0 >= cnt) {
        ++sc;
        j0 = 0;
      }
    }
    // the targets of the cell against the staged window
    const int wpad = (wn + 63) & ~63;
    for (int i = wn + lane; i < wpad; i += 32) {
      const int q = pair_index(i);
      W.cx[q] = kFar;
      W.cy[q] = kFar;
      W.cz[q] = kFar;
    }
    __syncwarp();
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
      const int gs = gself >= 0 ? gself + t - wbase : -1;
      const int self = (active && gs >= 0 && gs < wn) ? gs : -1;
      int k = (first || !active) ? 0 : nn[a];
      for (int jb = 0; jb < wpad; jb += 64) {
        uint64_t hit, unc;
        block_masks<WRAP>(g, W.cx + jb, W.cy + jb, W.cz + jb, npx, npy, npz, lo_lim, hi_lim,
                          hit, unc);
        // candidates inside the margin: exact FP64 test
        while (unc) {
          const int q = __clzll((long long)unc);
          unc ^= kTop >> q;
          const int b = entry_index(W.entry[jb + q]);
          if (exact_neighbor(g, s.x[a], s.y[a], s.z[a], s.h[a], s.x[b], s.y[b], s.z[b]))
            hit |= kTop >> q;
          ++exact;
        }
        if (self >= jb && self < jb + 64) hit &= ~(kTop >> (self - jb));
        if (!active) hit = 0;
        uint32_t* row = nbr + (int64_t)a * max_nb;
        while (hit) {  // slot order
          const int q = __clzll((long long)hit);
          hit ^= kTop >> q;
          if (k < max_nb) row[k] = W.entry[jb + q];
          ++k;
        }
      }
      if (active) {
        nn[a] = k;
        if (k > max_nb) raise_flag(err, SPH_FLAG_NB_OVERFLOW);
        tested += (unsigned long long)wn - (self >= 0 ? 1 : 0);
      }
    }
    __syncwarp();
    first = false;
    if (sc >= S.ncell) break;
    wbase += wn;
    wn = 0;
  }
}

}  // namespace find
}  // namespace sph
