// Cell tiles: the neighbour search and every pair kernel process one occupied
// cell at a time.  The cell's 3x3x3 stencil (distinct cells only) is laid out
// in a fixed order; slot j is the (j - off[s])-th particle of stencil cell s.
// A neighbour-list entry is the uint16 code (s << kOffBits) | (j - off[s]),
// so entries sorted by code are sorted by slot, and a kernel maps an entry to
// its particle start[s] + offset and to the stencil shift of cell s with one
// lookup in the cell's stencil.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"

namespace sph {

constexpr int kMaxStencil = 27;
constexpr int kMaxSlots = 65535;       // slots addressable by a window search
constexpr int kOffBits = 11;           // list entry: stencil cell (5 bits), offset (11 bits)
constexpr int kMaxCellPop = (1 << kOffBits) - 1;

__host__ __device__ __forceinline__ uint16_t entry_code(int cell, int off) {
  return (uint16_t)((cell << kOffBits) | off);
}

struct alignas(16) Stencil {
  int ncell;
  int self_slot0;                 // slot of the target cell's first particle
  int a0, na;                     // target cell: first sorted index, population
  int start[kMaxStencil];         // first sorted index of each stencil cell
  int off[kMaxStencil + 1];       // slot prefix; off[ncell] = total slots
  float shift[kMaxStencil][3];    // stencil-cell origin minus target-cell origin (FP32)
  int maxpop;                     // largest stencil-cell population
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

// Builds the stencil of occupied cell `code` into shared memory.  Must be
// called by the whole CTA (contains __syncthreads); warp 0 does the work.
__device__ __forceinline__ void build_stencil(const Grid& g, uint32_t code,
                                              const uint32_t* tbl_start,
                                              const uint32_t* tbl_count, Stencil& S) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
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
  }
  __syncthreads();
}

// Same as build_stencil for one warp that owns its Stencil (no CTA barrier).
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

// Particle index of list entry e.
__device__ __forceinline__ int entry_particle(const Stencil& S, uint32_t e) {
  return S.start[e >> kOffBits] + (int)(e & kMaxCellPop);
}

// Stencil cell holding slot j (binary search over off[0..ncell]).
__device__ __forceinline__ int slot_cell(const Stencil& S, int j) {
  int lo = 0, hi = S.ncell - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S.off[mid] <= j)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int slot_global(const Stencil& S, int j) {
  const int s = slot_cell(S, j);
  return S.start[s] + (j - S.off[s]);
}

// Threads per target for a cell of `na` targets on a CTA of `threads`:
// the largest power of two <= threads / na, at most kMaxTpp.
__device__ __forceinline__ int threads_per_target(int na, int threads, int max_tpp) {
  int t = 1;
  while (t < max_tpp && (t * 2) * na <= threads) t *= 2;
  return t;
}

}  // namespace sph
