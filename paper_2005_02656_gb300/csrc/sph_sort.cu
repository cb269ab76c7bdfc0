// Cell grid, Morton-order counting sort and state gather (section 4.3 of the
// paper keeps particles in the depth-first order of its octree, i.e. Morton
// order; here the cells of a uniform grid of side >= 2 h_max are ordered by
// Morton code and particles within a cell keep their previous relative order).
//
// Pipeline (all on the device, no host synchronisation):
//   k_grid_reduce  block min/max of x, y, z (open axes) and max h, on ordered
//                  integer keys; the last block derives the grid (Grid) and
//                  validates the periodic box
//   k_zero_table   clear the per-code particle counts
//   k_cell_count   Morton code per particle, arrival slot by atomicAdd
//   k_scan_*       exclusive scan of counts over codes -> cell start, and the
//                  list of occupied cells in Morton order
//   k_scatter      particle -> provisional sorted position
//   k_cell_order   per cell: rank members by source index (deterministic order)
//   k_gather_a     copy positions, h, m, u and id into sorted scratch, and
//                  build the FP32 cell-relative positions
//   k_gather_b     copy velocities and the integrator history (first read by
//                  the momentum pass)
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kRedThreads = 256;

// The extent and h_max reductions run on ordered integer keys (okey) in
// integer arithmetic: FP64 runs at 1/64 of the FP32 rate on this part.
__device__ __forceinline__ long long warp_min_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ long long warp_max_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Keys k[0..2] (minima of x, y, z), k[3..5] (maxima) and k[6] (max h, whose
// negative values are ignored as fmax from 0 would) of one block, reduced on
// the open axes only (periodic axes take the box and keep the neutral keys).
__global__ void k_grid_reduce(StateView in, int64_t n, sph_params prm, Grid* g, long long* part,
                              unsigned int* counter, uint32_t* err) {
  __shared__ long long sh[kRedThreads / 32][7];
  __shared__ bool last;
  const bool open[3] = {!prm.periodic[0], !prm.periodic[1], !prm.periodic[2]};
  long long v[7] = {kKeyInf, kKeyInf, kKeyInf, -kKeyInf, -kKeyInf, -kKeyInf, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double* xyz[3] = {in.x, in.y, in.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (!open[ax]) continue;
      const double q = xyz[ax][i];
      v[ax] = min(v[ax], okey(q, kKeyInf));
      v[3 + ax] = max(v[3 + ax], okey(q, -kKeyInf));
    }
    v[6] = max(v[6], okey(in.h[i], 0));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (!open[ax]) continue;
    v[ax] = warp_min_ll(v[ax]);
    v[3 + ax] = warp_max_ll(v[3 + ax]);
  }
  v[6] = warp_max_ll(v[6]);
  if (l == 0)
    for (int k = 0; k < 7; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) {
      for (int k = 0; k < 3; ++k) v[k] = min(v[k], sh[ww][k]);
      for (int k = 3; k < 7; ++k) v[k] = max(v[k], sh[ww][k]);
    }
    for (int k = 0; k < 7; ++k) part[blockIdx.x * 8 + k] = v[k];
    __threadfence();
    unsigned int done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // last block: every thread folds a strided subset of the block partials
  // (read from L2), then warp and block trees (min/max: order-free)
  __threadfence();
  long long r[7] = {kKeyInf, kKeyInf, kKeyInf, -kKeyInf, -kKeyInf, -kKeyInf, 0};
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const long long* pb = part + b * 8;
    for (int k = 0; k < 3; ++k) r[k] = min(r[k], __ldcg(pb + k));
    for (int k = 3; k < 7; ++k) r[k] = max(r[k], __ldcg(pb + k));
  }
  for (int k = 0; k < 3; ++k) r[k] = warp_min_ll(r[k]);
  for (int k = 3; k < 7; ++k) r[k] = warp_max_ll(r[k]);
  if (l == 0)
    for (int k = 0; k < 7; ++k) sh[w][k] = r[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) {
    for (int k = 0; k < 3; ++k) r[k] = min(r[k], sh[ww][k]);
    for (int k = 3; k < 7; ++k) r[k] = max(r[k], sh[ww][k]);
  }
  double rd[7];
  for (int k = 0; k < 7; ++k) rd[k] = from_okey(r[k]);
  *counter = 0;
  Grid G;
  double hmax = rd[6];
  G.hmax = hmax;
  int maxnc = 1;
  for (int ax = 0; ax < 3; ++ax) {
    int per = prm.periodic[ax] ? 1 : 0;
    double lo, L;
    if (per) {
      lo = prm.box_lo[ax];
      L = prm.box_hi[ax] - prm.box_lo[ax];
      if (!(2.0 * hmax < 0.5 * L)) raise_flag(err, SPH_FLAG_BAD_BOX);
    } else {
      lo = n > 0 ? rd[ax] : 0.0;
      L = n > 0 ? rd[3 + ax] - rd[ax] : 0.0;
    }
    int nc = 1;
    if (hmax > 0.0 && L > 0.0) {
      double q = floor(L / (2.0 * hmax * (1.0 + 1e-9)));
      nc = q < 1.0 ? 1 : (q > (double)(1 << kMaxCellBits) ? (1 << kMaxCellBits) : (int)q);
    }
    double cs = L > 0.0 ? L / nc : 0.0;
    G.lo[ax] = lo;
    G.cs[ax] = cs;
    G.inv_cs[ax] = cs > 0.0 ? 1.0 / cs : 0.0;
    G.Lbox[ax] = per ? L : 0.0;
    G.halfL[ax] = per ? 0.5 * L : 0.0;
    G.cs32[ax] = (float)cs;
    G.L32[ax] = (float)G.Lbox[ax];
    G.halfL32[ax] = (float)G.halfL[ax];
    G.err32[ax] = (float)(cs * 9.5367431640625e-07);  // 2^-20 cs
    G.nc[ax] = nc;
    G.periodic[ax] = per;
    maxnc = nc > maxnc ? nc : maxnc;
  }
  G.wrap32 = 0;
  for (int ax = 0; ax < 3; ++ax)
    if (G.periodic[ax] && G.nc[ax] < 3) G.wrap32 = 1;
  int bits = 0;
  while ((1 << bits) < maxnc) ++bits;
  G.bits = bits;
  G.tbl_size = 1u << (3 * bits);
  G.n_occ = 0;
  *g = G;
}

__global__ void k_zero_table(const Grid* g, uint32_t* count, double* org) {
  uint32_t size = g->tbl_size;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < size; i += gridDim.x * blockDim.x)
    count[i] = 0u;
  // cell origins lo + i cs, one table per axis (read by k_gather_a)
  constexpr int kRow = 1 << kMaxCellBits;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * kRow) {
    const int ax = i / kRow, c = i % kRow;
    if (c < g->nc[ax]) org[i] = g->lo[ax] + c * g->cs[ax];
  }
}

__device__ __forceinline__ void cell_coords(const Grid& g, double x, double y, double z, int& ix,
                                            int& iy, int& iz) {
  double p[3] = {x, y, z};
  int c[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    // floor((p - lo) / cs) clamped to [0, nc - 1]: the round-down conversion
    // saturates (NaN gives 0), so the clamp runs on integers
    const int v = __double2int_rd((p[ax] - g.lo[ax]) * g.inv_cs[ax]);
    c[ax] = v < 0 ? 0 : (v >= g.nc[ax] ? g.nc[ax] - 1 : v);
  }
  ix = c[0];
  iy = c[1];
  iz = c[2];
}

__global__ void k_cell_count(StateView in, int64_t n, const Grid* gp, uint32_t* count,
                             uint32_t* code, uint32_t* slot) {
  const Grid g = *gp;
  const int lane = threadIdx.x & 31;
  // the loop is warp-uniform (i - lane is the warp's first index); lanes past
  // n take no part but the shuffles
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - lane < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool valid = i < n;
    uint32_t c = 0xffffffffu;
    if (valid) {
      int ix, iy, iz;
      cell_coords(g, in.x[i], in.y[i], in.z[i], ix, iy, iz);
      c = morton3(ix, iy, iz);
      code[i] = c;
    }
    // one atomic per group of lanes with the same cell (the state is in the
    // previous step's cell order, so neighbouring lanes mostly share a cell);
    // the slot order inside a cell does not matter (k_cell_order ranks by
    // previous index)
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(same) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&count[c], (uint32_t)__popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) slot[i] = base + (uint32_t)__popc(same & ((1u << lane) - 1u));
  }
}

// Block-level exclusive scan helper for kScanItems entries with 1024 threads.
constexpr int kScanThreads = 1024;
constexpr int kPerThread = kScanItems / kScanThreads;

__global__ void k_scan_a(const Grid* g, const uint32_t* count, uint32_t* part) {
  uint32_t size = g->tbl_size;
  uint32_t base = blockIdx.x * kScanItems;
  if (base >= size) return;
  uint32_t s = 0, o = 0;
  for (int k = 0; k < kPerThread; ++k) {
    uint32_t i = base + threadIdx.x * kPerThread + k;
    if (i < size) {
      uint32_t c = count[i];
      s += c;
      o += c ? 1u : 0u;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
    o += __shfl_xor_sync(0xffffffffu, o, off);
  }
  __shared__ uint32_t ss[32], so[32];
  if ((threadIdx.x & 31) == 0) {
    ss[threadIdx.x >> 5] = s;
    so[threadIdx.x >> 5] = o;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ts = 0, to = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
      ts += ss[w];
      to += so[w];
    }
    part[2 * blockIdx.x] = ts;
    part[2 * blockIdx.x + 1] = to;
  }
}

// Inclusive block scan of one uint32 per thread (1024 threads).
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* sh32) {
  int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, off);
    if (l >= off) v += t;
  }
  if (l == 31) sh32[w] = v;
  __syncthreads();
  if (w == 0) {
    uint32_t t = sh32[l];
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t q = __shfl_up_sync(0xffffffffu, t, off);
      if (l >= off) t += q;
    }
    sh32[l] = t;
  }
  __syncthreads();
  if (w > 0) v += sh32[w - 1];
  __syncthreads();
  return v;
}

// Single block: exclusive scan of the per-block partials (<= 4096 blocks).
__global__ void k_scan_b(Grid* g, uint32_t* part) {
  uint32_t nblk = (g->tbl_size + kScanItems - 1) / kScanItems;
  __shared__ uint32_t sh32[32];
  __shared__ uint32_t carry_s, carry_o;
  if (threadIdx.x == 0) {
    carry_s = 0;
    carry_o = 0;
  }
  __syncthreads();
  for (uint32_t base = 0; base < nblk; base += kScanThreads) {
    uint32_t i = base + threadIdx.x;
    uint32_t s = i < nblk ? part[2 * i] : 0u;
    uint32_t o = i < nblk ? part[2 * i + 1] : 0u;
    uint32_t is = block_incl_scan(s, sh32);
    uint32_t io = block_incl_scan(o, sh32);
    uint32_t cs = carry_s, co = carry_o;
    if (i < nblk) {
      part[2 * i] = cs + is - s;
      part[2 * i + 1] = co + io - o;
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) {
      carry_s = cs + is;
      carry_o = co + io;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) g->n_occ = carry_o;
}

__global__ void k_scan_c(const Grid* g, const uint32_t* count, const uint32_t* part,
                         uint32_t* start, uint32_t* occ) {
  uint32_t size = g->tbl_size;
  uint32_t base = blockIdx.x * kScanItems;
  if (base >= size) return;
  __shared__ uint32_t sh32[32];
  uint32_t c[kPerThread];
  uint32_t s = 0, o = 0;
  for (int k = 0; k < kPerThread; ++k) {
    uint32_t i = base + threadIdx.x * kPerThread + k;
    c[k] = i < size ? count[i] : 0u;
    s += c[k];
    o += c[k] ? 1u : 0u;
  }
  uint32_t is = block_incl_scan(s, sh32);
  uint32_t io = block_incl_scan(o, sh32);
  uint32_t ps = part[2 * blockIdx.x] + is - s;
  uint32_t po = part[2 * blockIdx.x + 1] + io - o;
  for (int k = 0; k < kPerThread; ++k) {
    uint32_t i = base + threadIdx.x * kPerThread + k;
    if (i < size) {
      start[i] = ps;
      if (c[k]) occ[po++] = i;
      ps += c[k];
    }
  }
}

__global__ void k_scatter(int64_t n, const uint32_t* code, const uint32_t* slot,
                          const uint32_t* start, int32_t* perm_tmp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    perm_tmp[start[code[i]] + slot[i]] = (int32_t)i;
  }
}

// One warp per occupied cell: the members' final order is by source index.
__global__ void k_cell_order(const Grid* g, const uint32_t* occ, const uint32_t* start,
                             const uint32_t* count, const int32_t* perm_tmp, int32_t* perm,
                             uint32_t* cell_of) {
  const uint32_t n_occ = g->n_occ;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_occ; k += warps) {
    uint32_t code = occ[k];
    uint32_t s0 = start[code], cnt = count[code];
    for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
      uint32_t j = j0 + lane;
      int32_t v = j < cnt ? perm_tmp[s0 + j] : 0x7fffffff;
      uint32_t rank = 0;
      for (uint32_t l0 = 0; l0 < cnt; l0 += 32) {
        int32_t w = (l0 + lane < cnt) ? perm_tmp[s0 + l0 + lane] : 0x7fffffff;
        for (int q = 0; q < 32; ++q) {
          int32_t wq = __shfl_sync(0xffffffffu, w, q);
          rank += (l0 + q < cnt && wq < v) ? 1u : 0u;
        }
      }
      if (j < cnt) {
        perm[s0 + rank] = v;
        cell_of[s0 + j] = k;
      }
    }
  }
}

__device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}

// Gather, first part: what the search, density and IAD read (positions, h,
// m, u, id and the FP32 cell-relative positions).
// Every load of a particle (and the next particle's source index) is issued
// before its first store: the compiler cannot tell that the output arrays
// alias none of the inputs, so a load written after a store would wait for a
// memory round trip of its own.
__global__ void k_gather_a(StateView in, StateView out, int64_t n, const double* org,
                           const int32_t* perm, const uint32_t* code, float4* pos32,
                           int32_t* cell3, float4* rec_d) {
  constexpr int kRow = 1 << kMaxCellBits;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t s = p < n ? perm[p] : 0;
  for (; p < n; p += stride) {
    const double x = in.x[s], y = in.y[s], z = in.z[s], h = in.h[s];
    const double m = in.m[s], u = in.u[s];
    const int64_t id = in.id[s];
    const uint32_t c = code[s];
    const int64_t s_next = p + stride < n ? perm[p + stride] : 0;
    const int ix = compact3(c), iy = compact3(c >> 1), iz = compact3(c >> 2);
    const float ox = f32_rn(x - __ldg(org + ix));
    const float oy = f32_rn(y - __ldg(org + kRow + iy));
    const float oz = f32_rn(z - __ldg(org + 2 * kRow + iz));
    out.x[p] = x;
    out.y[p] = y;
    out.z[p] = z;
    out.h[p] = h;
    out.m[p] = m;
    out.u[p] = u;
    out.id[p] = id;
    pos32[p] = make_float4(ox, oy, oz, f32_rn(h));
    cell3[p] = pack_cell(ix, iy, iz);
    rec_d[p] = make_float4(ox, oy, oz, f32_rn(m));
    s = s_next;
  }
}

// Gather, second part: velocities and the integrator history, first read by
// the momentum pass (so a caller may still be copying them in while the
// search runs).  Loads before stores, as in k_gather_a.
__global__ void k_gather_b(StateView in, StateView out, int64_t n, const int32_t* perm,
                           float4* rec_m, float4* recV) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t s = p < n ? perm[p] : 0;
  for (; p < n; p += stride) {
    const double vx = in.vx[s], vy = in.vy[s], vz = in.vz[s];
    const double vxh = in.vxh[s], vyh = in.vyh[s], vzh = in.vzh[s];
    const double dup = in.du_prev[s];
    const double m = out.m[p];
    const int64_t s_next = p + stride < n ? perm[p + stride] : 0;
    out.vx[p] = vx;
    out.vy[p] = vy;
    out.vz[p] = vz;
    out.vxh[p] = vxh;
    out.vyh[p] = vyh;
    out.vzh[p] = vzh;
    out.du_prev[p] = dup;
    const float4 vm = make_float4(f32_rn(vx), f32_rn(vy), f32_rn(vz), f32_rn(m));
    if (recV)
      recV[p] = vm;  // the staged pair passes' velocity plane
    else
      rec_m[5 * p + 1] = vm;
    s = s_next;
  }
}

inline int grid_for(int64_t n, int threads, int sm) {
  int64_t b = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sm * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

void launch_grid(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st) {
  int blocks = grid_for(n, kRedThreads, ctx->sm_count);
  if (blocks > kReduceBlocks) blocks = kReduceBlocks;
  k_grid_reduce<<<blocks, kRedThreads, 0, st>>>(in, n, ctx->prm, ctx->grid,
                                                reinterpret_cast<long long*>(ctx->red.part),
                                                ctx->red.counter + 0, ctx->err);
  k_zero_table<<<ctx->sm_count * 8, 256, 0, st>>>(ctx->grid, ctx->tbl_count, ctx->cell_org);
  ctx->launches += 2;
}

void launch_sort(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st,
                 cudaEvent_t wait_gather) {
  int pb = grid_for(n, 256, ctx->sm_count);
  k_cell_count<<<pb, 256, 0, st>>>(in, n, ctx->grid, ctx->tbl_count, ctx->code, ctx->slot);
  const int scan_blocks = kMaxTable / kScanItems;
  k_scan_a<<<scan_blocks, kScanThreads, 0, st>>>(ctx->grid, ctx->tbl_count, ctx->scan_part);
  k_scan_b<<<1, kScanThreads, 0, st>>>(ctx->grid, ctx->scan_part);
  k_scan_c<<<scan_blocks, kScanThreads, 0, st>>>(ctx->grid, ctx->tbl_count, ctx->scan_part,
                                                  ctx->tbl_start, ctx->occ);
  k_scatter<<<pb, 256, 0, st>>>(n, ctx->code, ctx->slot, ctx->tbl_start, ctx->perm_tmp);
  k_cell_order<<<ctx->sm_count * 8, 256, 0, st>>>(ctx->grid, ctx->occ, ctx->tbl_start,
                                                  ctx->tbl_count, ctx->perm_tmp, ctx->perm,
                                                  ctx->cell_of);
  if (wait_gather) cudaStreamWaitEvent(st, wait_gather, 0);
  k_gather_a<<<pb, 256, 0, st>>>(in, ctx->s, n, ctx->cell_org, ctx->perm, ctx->code, ctx->pos32,
                                 ctx->cell3, ctx->rec_d);
  ctx->launches += 7;
}

void launch_gather_b(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st) {
  k_gather_b<<<grid_for(n, 256, ctx->sm_count), 256, 0, st>>>(
      in, ctx->s, n, ctx->perm, ctx->rec_m, staged_pairs(ctx) ? ctx->recV : nullptr);
  ctx->launches += 1;
}

void launch_sort_gather(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st) {
  launch_sort(ctx, in, n, st);
  launch_gather_b(ctx, in, n, st);
}

void launch_copy_state(const StateView& dst, const StateView& src, int64_t n, cudaStream_t st,
                       sph_ctx* ctx) {
  size_t b = (size_t)n * sizeof(double);
  double* d[13] = {dst.x, dst.y, dst.z, dst.vx, dst.vy, dst.vz, dst.vxh, dst.vyh, dst.vzh,
                   dst.h, dst.m, dst.u, dst.du_prev};
  double* s[13] = {src.x, src.y, src.z, src.vx, src.vy, src.vz, src.vxh, src.vyh, src.vzh,
                   src.h, src.m, src.u, src.du_prev};
  for (int k = 0; k < 13; ++k) cudaMemcpyAsync(d[k], s[k], b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(dst.id, src.id, (size_t)n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  (void)ctx;
}

}  // namespace sph
