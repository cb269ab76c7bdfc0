// findNeighbors (section 4.1: b runs over the neighbours of a, i.e. the
// particles inside the kernel support |x_a - x_b| < 2 h_a).
//
// One warp per occupied cell; each lane owns one target particle of the cell
// (32 at a time).  The warp walks the distinct cells of the 3x3x3 stencil and,
// for every candidate b (read once per warp and broadcast to all lanes), each
// lane decides b in N_a:
//   1. FP32 prefilter on cell-relative offsets: r2_32 is compared with
//      (2 h_a)^2 within a margin M_a that bounds the FP32 rounding error of
//      the separation (Grid::err32) and of the squares;
//   2. only candidates inside the margin are decided by the exact FP64
//      criterion (sph_device.cuh: exact_neighbor), so the lists are
//      bit-identical to r^2 < (2h)^2 evaluated in FP64 without FMA.
// Lists are stored transposed, nbr[k * stride + a], so that the per-particle
// pair kernels read them with coalesced loads.
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

struct AxisCells {
  int cell[3];
  int shift[3];
  int cnt;
};

__device__ __forceinline__ AxisCells axis_cells(const Grid& g, int ax, int ic) {
  AxisCells r;
  int nc = g.nc[ax];
  r.cnt = 0;
  if (g.periodic[ax]) {
    if (nc >= 3) {
      for (int d = -1; d <= 1; ++d) {
        int c = ic + d;
        c = c < 0 ? c + nc : (c >= nc ? c - nc : c);
        r.cell[r.cnt] = c;
        r.shift[r.cnt] = d;
        ++r.cnt;
      }
    } else if (nc == 2) {
      r.cell[0] = ic;
      r.shift[0] = 0;
      r.cell[1] = 1 - ic;
      r.shift[1] = ic == 0 ? 1 : -1;
      r.cnt = 2;
    } else {
      r.cell[0] = ic;
      r.shift[0] = 0;
      r.cnt = 1;
    }
  } else {
    for (int d = -1; d <= 1; ++d) {
      int c = ic + d;
      if (c < 0 || c >= nc) continue;
      r.cell[r.cnt] = c;
      r.shift[r.cnt] = d;
      ++r.cnt;
    }
  }
  return r;
}

__device__ __forceinline__ float wrap32(float d, const Grid& g, int ax) {
  if (g.periodic[ax]) {
    if (d > g.halfL32[ax])
      d -= g.L32[ax];
    else if (d < -g.halfL32[ax])
      d += g.L32[ax];
  }
  return d;
}

__global__ void __launch_bounds__(128) k_find(const Grid* gp, StateView s, const float4* pos32,
                                              const uint32_t* occ, const uint32_t* tbl_start,
                                              const uint32_t* tbl_count, int32_t* nn,
                                              int32_t* nbr, int64_t stride, int max_nb,
                                              uint32_t* err, unsigned long long* stats) {
  const Grid g = *gp;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < g.n_occ; k += warps) {
    const uint32_t code = occ[k];
    const uint32_t c0 = tbl_start[code], ccount = tbl_count[code];
    // cell coordinates from the Morton code
    int ic[3];
    {
      uint32_t v[3] = {code, code >> 1, code >> 2};
      for (int ax = 0; ax < 3; ++ax) {
        uint32_t t = v[ax] & 0x09249249u;
        t = (t | (t >> 2)) & 0x030c30c3u;
        t = (t | (t >> 4)) & 0x0300f00fu;
        t = (t | (t >> 8)) & 0x030000ffu;
        t = (t | (t >> 16)) & 0x000003ffu;
        ic[ax] = (int)t;
      }
    }
    const AxisCells AX = axis_cells(g, 0, ic[0]);
    const AxisCells AY = axis_cells(g, 1, ic[1]);
    const AxisCells AZ = axis_cells(g, 2, ic[2]);

    for (uint32_t t0 = 0; t0 < ccount; t0 += 32) {
      const bool active = t0 + lane < ccount;
      const int64_t a = (int64_t)c0 + t0 + (active ? lane : 0);
      const float4 pa = pos32[a];
      const double xa = s.x[a], ya = s.y[a], za = s.z[a], ha = s.h[a];
      const float two_h = 2.0f * pa.w;
      const float lim = two_h * two_h;
      const float esum = g.err32[0] + g.err32[1] + g.err32[2];
      const float esq = g.err32[0] * g.err32[0] + g.err32[1] * g.err32[1] +
                        g.err32[2] * g.err32[2];
      const float margin = 2.0f * (2.0f * two_h * esum + esq + 4.76837158203125e-07f * lim);
      const float lo_lim = lim - margin, hi_lim = lim + margin;
      int cnt = 0;
      uint32_t tested = 0, exact = 0;
      for (int iz = 0; iz < AZ.cnt; ++iz)
        for (int iy = 0; iy < AY.cnt; ++iy)
          for (int ix = 0; ix < AX.cnt; ++ix) {
            const uint32_t cc = morton3(AX.cell[ix], AY.cell[iy], AZ.cell[iz]);
            const uint32_t b0 = tbl_start[cc], bn = tbl_count[cc];
            const float sx = AX.shift[ix] * g.cs32[0];
            const float sy = AY.shift[iy] * g.cs32[1];
            const float sz = AZ.shift[iz] * g.cs32[2];
            tested += bn;
            for (uint32_t j = 0; j < bn; ++j) {
              const int64_t b = (int64_t)b0 + j;
              const float4 pb = pos32[b];
              float dx = wrap32((pb.x + sx) - pa.x, g, 0);
              float dy = wrap32((pb.y + sy) - pa.y, g, 1);
              float dz = wrap32((pb.z + sz) - pa.z, g, 2);
              float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              bool hit;
              if (r2 < lo_lim)
                hit = true;
              else if (r2 > hi_lim)
                hit = false;
              else {
                hit = exact_neighbor(g, xa, ya, za, ha, s.x[b], s.y[b], s.z[b]);
                exact += active ? 1u : 0u;
              }
              hit = hit && active && (b != a);
              if (hit) {
                if (cnt < max_nb) nbr[(int64_t)cnt * stride + a] = (int32_t)b;
                ++cnt;
              }
            }
          }
      if (active) {
        nn[a] = cnt;
        if (cnt > max_nb) raise_flag(err, SPH_FLAG_NB_OVERFLOW);
      }
      // counters: candidate tests of the active lanes and exact tests
      unsigned long long t = active ? tested : 0u, e = exact;
      for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
      }
      if (lane == 0) {
        atomicAdd(stats + 0, t);
        atomicAdd(stats + 1, e);
      }
    }
  }
}

// Export: ids of the neighbours of each particle, ascending (insertion sort).
__global__ void k_export(int64_t n, const int32_t* nn, const int32_t* nbr, int64_t stride,
                         int max_nb, const int64_t* id, int32_t* counts, int64_t* ids) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    int c = nn[p];
    counts[p] = c;
    int m = c < max_nb ? c : max_nb;
    int64_t* row = ids + p * max_nb;
    for (int k = 0; k < m; ++k) {
      int64_t v = id[nbr[(int64_t)k * stride + p]];
      int j = k - 1;
      while (j >= 0 && row[j] > v) {
        row[j + 1] = row[j];
        --j;
      }
      row[j + 1] = v;
    }
  }
}

}  // namespace

void launch_find_neighbors(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st) {
  (void)n;
  int blocks = ctx->sm_count * 16;
  k_find<<<blocks, 128, 0, st>>>(ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start,
                                 ctx->tbl_count, ctx->nn, ctx->nbr, ctx->n_max, ctx->prm.max_nb,
                                 ctx->err, ctx->stats);
  ctx->launches += 1;
}

void launch_export_neighbors(sph_ctx* ctx, const StateView& s, int64_t n, int32_t* counts,
                             int64_t* ids, cudaStream_t st) {
  int64_t b = (n + 127) / 128;
  if (b > ctx->sm_count * 32) b = ctx->sm_count * 32;
  if (b < 1) b = 1;
  k_export<<<(int)b, 128, 0, st>>>(n, ctx->nn, ctx->nbr, ctx->n_max, ctx->prm.max_nb, s.id,
                                   counts, ids);
  ctx->launches += 1;
}

}  // namespace sph
