// Cell tiles: the neighbour search processes one occupied cell at a time.
// The cell's 3x3x3 stencil (distinct cells only) is laid out in a fixed
// order; slot j is the (j - off[s])-th particle of stencil cell s.
//
// A neighbour-list entry is a uint32: the neighbour's sorted particle index in
// the low kIndexBits bits and, above them, the code (sx+1) + 3(sy+1) + 9(sz+1)
// of the shift (-1, 0, +1 cell sides per axis) of the neighbour's cell
// relative to the target's cell.  A pair kernel thus gets both the particle
// and its FP32 position relative to the target's cell from the entry alone:
// (offset_b + shift * cell side) - offset_a, with no table lookup.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"

namespace sph {

constexpr int kMaxStencil = 27;
constexpr int kMaxSlots = 65535;       // stencil slots of one cell
constexpr int kIndexBits = 27;         // list entry: particle index (27 bits)
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
constexpr int64_t kMaxParticles = (int64_t)1 << kIndexBits;
constexpr int kMaxCellPop = kMaxSlots;

__host__ __device__ __forceinline__ int shift_code(int sx, int sy, int sz) {
  return (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
}
__host__ __device__ __forceinline__ uint32_t entry_make(int code, int particle) {
  return ((uint32_t)code << kIndexBits) | (uint32_t)particle;
}
__device__ __forceinline__ int entry_index(uint32_t e) { return (int)(e & kIndexMask); }
// FP32 shift of the entry's cell relative to the target's cell.
__device__ __forceinline__ void entry_shift(uint32_t e, const Grid& g, float& sx, float& sy,
                                            float& sz) {
  const int c = (int)(e >> kIndexBits);
  const int cz = c / 9, cy = (c - 9 * cz) / 3, cx = c - 9 * cz - 3 * cy;
  sx = (float)(cx - 1) * g.cs32[0];
  sy = (float)(cy - 1) * g.cs32[1];
  sz = (float)(cz - 1) * g.cs32[2];
}

struct alignas(16) Stencil {
  int ncell;
  int self_cell;                  // stencil index of the target cell
  int self_slot0;                 // slot of the target cell's first particle
  int a0, na;                     // target cell: first sorted index, population
  int start[kMaxStencil];         // first sorted index of each stencil cell
  int off[kMaxStencil + 1];       // slot prefix; off[ncell] = total slots
  float shift[kMaxStencil][3];    // stencil-cell origin minus target-cell origin (FP32)
  int scode[kMaxStencil];         // shift code of each stencil cell (list entries)
  int maxpop;                     // largest stencil-cell population
  float box_lo[3], box_hi[3];     // bounding box of the target cell's particles (FP32)
  float reach2;                   // squared staging reach (find_cell)
};

// Distinct stencil cells along one axis for a target cell at index ic: their
// number, and for the i-th one its cell index and shift (-1, 0, +1 cell
// sides).  Periodic axes wrap (a 2-cell axis has two distinct cells and a
// 1-cell axis one); open axes clip at the grid's ends.
__device__ __forceinline__ int axis_count(const Grid& g, int ax, int ic) {
  const int nc = g.nc[ax];
  if (g.periodic[ax]) return nc >= 3 ? 3 : nc;
  return 1 + (ic > 0 ? 1 : 0) + (ic + 1 < nc ? 1 : 0);
}

__device__ __forceinline__ void axis_cell(const Grid& g, int ax, int ic, int i, int& cell,
                                          int& shift) {
  const int nc = g.nc[ax];
  if (g.periodic[ax]) {
    if (nc >= 3) {
      shift = i - 1;
      const int c = ic + shift;
      cell = c < 0 ? c + nc : (c >= nc ? c - nc : c);
    } else if (nc == 2) {
      cell = i == 0 ? ic : 1 - ic;
      shift = i == 0 ? 0 : (ic == 0 ? 1 : -1);
    } else {
      cell = ic;
      shift = 0;
    }
  } else {
    const int first = ic > 0 ? ic - 1 : 0;
    cell = first + i;
    shift = cell - ic;
  }
}

__device__ __forceinline__ uint32_t compact3_bits(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}

// Builds the stencil of occupied cell `code` into the warp's shared-memory
// Stencil (warp-synchronous; no CTA barrier).
__device__ __forceinline__ void build_stencil_warp(const Grid& g, uint32_t code,
                                                   const uint32_t* tbl_start,
                                                   const uint32_t* tbl_count, Stencil& S) {
  const int lane = threadIdx.x & 31;
  const int ic[3] = {(int)compact3_bits(code), (int)compact3_bits(code >> 1),
                     (int)compact3_bits(code >> 2)};
  const int nx = axis_count(g, 0, ic[0]);
  const int ny = axis_count(g, 1, ic[1]);
  const int nz = axis_count(g, 2, ic[2]);
  const int ncell = nx * ny * nz;
  int cnt = 0;
  bool self = false;
  if (lane < ncell) {
    int cx, cy, cz, sx, sy, sz;
    axis_cell(g, 0, ic[0], lane % nx, cx, sx);
    axis_cell(g, 1, ic[1], (lane / nx) % ny, cy, sy);
    axis_cell(g, 2, ic[2], lane / (nx * ny), cz, sz);
    const uint32_t cc = morton3(cx, cy, cz);
    S.start[lane] = (int)tbl_start[cc];
    cnt = (int)tbl_count[cc];
    S.shift[lane][0] = sx * g.cs32[0];
    S.shift[lane][1] = sy * g.cs32[1];
    S.shift[lane][2] = sz * g.cs32[2];
    S.scode[lane] = shift_code(sx, sy, sz);
    self = sx == 0 && sy == 0 && sz == 0;
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane < ncell) S.off[lane] = incl - cnt;
  if (lane == ncell - 1) S.off[ncell] = incl;
  if (self) {
    S.self_cell = lane;
    S.self_slot0 = incl - cnt;
    S.a0 = S.start[lane];
    S.na = cnt;
  }
  int mp = cnt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mp = max(mp, __shfl_xor_sync(0xffffffffu, mp, o));
  if (lane == 0) {
    S.ncell = ncell;
    S.maxpop = mp;
  }
  __syncwarp();
}



}  // namespace sph
