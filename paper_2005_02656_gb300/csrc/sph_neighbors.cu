// findNeighbors (section 4.1: b runs over the neighbours of a, the particles
// inside the kernel support |x_a - x_b| < 2 h_a).
//
// One warp per occupied cell (warps of a CTA work independently, each with
// its own shared-memory window, so no CTA barrier is involved); the per-cell
// body is find::find_cell in sph_find.cuh.
#include <cuda_runtime.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_find.cuh"
#include "sph_tile.cuh"

namespace sph {

namespace {

using namespace find;

// Launched in both variants; the one whose WRAP does not match the grid (a
// periodic axis with fewer than 3 cells needs the FP32 wrap) returns at once.
// No register cap: at 108-122 registers (4 CTAs per SM) the search measured
// 1-2% faster than capped at 94 (5 CTAs) or 80 (6 CTAs); its unrolled mask
// loop gains more from registers than from resident warps.
template <bool WRAP>
__global__ void __launch_bounds__(kFindThreads, 1) k_find_tile(
    const Grid* gp, StateView s, const float4* __restrict__ pos32, const uint32_t* occ,
    const uint32_t* tbl_start, const uint32_t* tbl_count, int32_t* nn, uint32_t* nbr,
    int max_nb, uint32_t* err, unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  FindWarpSmem& W = reinterpret_cast<FindWarpSmem*>(smem_raw)[warp];
  const Grid g = *gp;
  if ((g.wrap32 != 0) != WRAP) return;
  unsigned long long tested = 0, exact = 0;
  const uint32_t gw = blockIdx.x * kFindWarps + warp, nw = gridDim.x * kFindWarps;
  for (uint32_t cell = gw; cell < g.n_occ; cell += nw)
    find_cell<WRAP>(g, occ[cell], s, pos32, tbl_start, tbl_count, nn, nbr, max_nb, err, W,
                    tested, exact);
  // counters: one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    tested += __shfl_xor_sync(0xffffffffu, tested, o);
    exact += __shfl_xor_sync(0xffffffffu, exact, o);
  }
  if (lane == 0) {
    atomicAdd(stats + 0, tested);
    atomicAdd(stats + 1, exact);
  }
}

// Export: per particle, the neighbours' ids sorted ascending (insertion sort).
__global__ void k_export(int64_t n, const int32_t* nn, const uint32_t* nbr, int max_nb,
                         const int64_t* id, int32_t* counts, int64_t* ids) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int c = nn[a];
    counts[a] = c;
    const int m = c < max_nb ? c : max_nb;
    int64_t* row = ids + a * max_nb;
    for (int k = 0; k < m; ++k) {
      const int64_t v = id[entry_index(nbr[a * max_nb + k])];
      int q = k - 1;
      while (q >= 0 && row[q] > v) {
        row[q + 1] = row[q];
        --q;
      }
      row[q + 1] = v;
    }
  }
}

}  // namespace

void launch_find_neighbors(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st) {
  (void)n;
  const size_t smem = kFindWarps * sizeof(FindWarpSmem);
  if (!ctx->find_blocks) {  // once per context, on its device
    int per_sm = 0;
    cudaFuncSetAttribute(k_find_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(k_find_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_find_tile<false>, kFindThreads,
                                                  smem);
    ctx->find_blocks = (per_sm > 0 ? per_sm : 1) * ctx->sm_count;
  }
  k_find_tile<false><<<ctx->find_blocks, kFindThreads, smem, st>>>(
      ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start, ctx->tbl_count, ctx->nn, ctx->nbr,
      ctx->prm.max_nb, ctx->err, ctx->stats);
  k_find_tile<true><<<ctx->find_blocks, kFindThreads, smem, st>>>(
      ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start, ctx->tbl_count, ctx->nn, ctx->nbr,
      ctx->prm.max_nb, ctx->err, ctx->stats);
  ctx->launches += 2;
}

void launch_export_neighbors(sph_ctx* ctx, const StateView& s, int64_t n, int32_t* counts,
                             int64_t* ids, cudaStream_t st) {
  int64_t b = (n + 127) / 128;
  if (b > (int64_t)ctx->sm_count * 32) b = ctx->sm_count * 32;
  if (b < 1) b = 1;
  k_export<<<(int)b, 128, 0, st>>>(n, ctx->nn, ctx->nbr, ctx->prm.max_nb, s.id, counts, ids);
  ctx->launches += 1;
}

}  // namespace sph
