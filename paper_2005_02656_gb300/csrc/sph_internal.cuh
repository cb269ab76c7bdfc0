// Internal declarations of libsph: the context, the device-side grid
// description and the kernel launchers of each translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kMaxCellBits = 8;                 // up to 256 cells per axis
constexpr uint32_t kMaxTable = 1u << (3 * kMaxCellBits);
constexpr int kReduceBlocks = 1024;             // partial slots of grid reductions
constexpr int kScanItems = 4096;                // cell-table entries per scan block
constexpr int kProfRing = 64;                   // step event sets kept before folding
constexpr int kHTab = 4097;                     // h factors tabulated for counts 0..4096
constexpr int kKernelTableN = 20000;            // kernel values of SPH_KERNEL_TABLE
constexpr int kMaskWords = 32;                  // hit-mask words per particle (staged pairs)
constexpr int kStats = 6;                       // cumulative device counters (sph_stats)

// Cell grid of the current step, computed on the device from the particles'
// extent and h_max, read by every later kernel of the step.
struct Grid {
  double lo[3];      // origin of cell (0,0,0)
  double cs[3];      // cell side per axis (>= 2 h_max)
  double inv_cs[3];
  double Lbox[3];    // period on periodic axes (box_hi - box_lo), 0 on open axes
  double halfL[3];   // 0.5 * Lbox
  float cs32[3];
  float L32[3];
  float halfL32[3];
  float err32[3];    // bound on the FP32 error of a cell-relative separation
  int wrap32;        // a periodic axis has < 3 cells: FP32 separations need a wrap
  int nc[3];
  int periodic[3];
  int bits;          // Morton bits per axis
  uint32_t tbl_size; // 2^(3 bits)
  uint32_t n_occ;    // occupied cells (written by the scan)
  double hmax;
};

// Sorted-state view passed to kernels by value.
struct StateView {
  double *x, *y, *z, *vx, *vy, *vz, *vxh, *vyh, *vzh, *h, *m, *u, *du_prev;
  int64_t* id;
};

struct OutView {
  double *rho, *p, *c, *iad, *ax, *ay, *az, *du;
  double* omega;  // grad-h terms (NULL: not written)
};

// Block-reduction partials (per block) and finalisation counters.
struct Reduce {
  double* part;          // kReduceBlocks * 16 doubles
  unsigned int* counter; // last-block-done counters (4)
};

}  // namespace sph

struct sph_ctx {
  sph_params prm;
  int64_t n_max;
  int device;
  double Bn;
  int sm_count;
  int64_t launches;
  int have_lists;     // lists valid for the current order
  int have_density;
  int have_iad;
  char last_error[512];

  // device scalars
  sph::Grid* grid;
  uint32_t* err;
  double* dt_dev;       // scratch dt (host-step path)
  double* diag;         // 16 doubles: [0..7] sums of the new state, [8] dt,
                        // [9] min nn, [10] max nn, [11] sum nn, [12] dt_prev
  double* hfac;         // kHTab: 0.5 (1 + cbrt(ng_target / max(k, 1))) for count k
  double2* ktab64;      // SPH_KERNEL_TABLE: (T_i, T_{i+1} - T_i), kKernelTableN entries
  float2* ktab32;       //   the same in FP32 (NULL when the mode is exact)
  double ktab_n;        // sinc_n the tables were built for (-1: none)
  int hfac_ng;          // ng_target the table was built for (-1: none)

  // sort
  uint32_t* code;       // Morton cell code per particle (input order)
  uint32_t* slot;       // arrival slot within the cell
  int32_t* perm_tmp;
  int32_t* perm;        // sorted position -> source index
  uint32_t* tbl_count;  // per Morton code
  uint32_t* tbl_start;
  uint32_t* occ;        // occupied cells in Morton order
  uint32_t* scan_part;  // per scan block: particle sum, occupied sum (2 x)
  uint32_t* cell_of;    // occupied-cell index of each sorted particle

  // sorted state scratch (FP64) + ids
  sph::StateView s;
  int64_t* s_id_buf;

  // per-particle FP32 cell-relative data (sorted order)
  double* cell_org;     // cell origins lo + i cs per axis (3 x 2^kMaxCellBits)
  float4* pos32;        // offset from the cell origin (x, y, z) and h
  int32_t* cell3;       // packed cell coordinates (10 bits per axis)

  // neighbour lists: nn[n], nbr[p * max_nb + k] = entry (sph_tile.cuh)
  int32_t* nn;
  uint32_t* nbr;

  // FP64 path: W_ab(h_a) of every list entry, written by the density pass and
  // read by IAD and momentum (nbr layout; allocated for SPH_FP64 contexts)
  double* wcache;

  // FP64 per-particle helpers: one block of 5 * n_max doubles
  double* vol;          // m / rho          (vol + 0 n_max)
  double* X;            // P / rho^2        (vol + 1 n_max)
  double* inv_rho;      // 1 / rho          (vol + 2 n_max)
                        // 1 / h^2          (vol + 3 n_max)
                        // B_n / h^3        (vol + 4 n_max)

  // FP32 mixed-path per-particle records (sorted order, sph_pairs_fp32.cu)
  float4* rec_d;        // offset x, y, z, m               (gather)
  float4* rec_i;        // offset x, y, z, m/rho           (density)
  float4* rec_m;        // 5 float4 per particle           (gather, density, IAD)

  // SPH_PAIRS_STAGED (sph_staged.cu): per occupied cell (slot_base,
  // mask_base, a0, S << 16 | na); staged candidate entries; hit masks
  // (mask_cap 64-bit words); two allocation counters.  Cells in list form
  // use nbr.
  uint4* cmeta;
  uint32_t* sent;
  unsigned long long* masks;
  unsigned long long* salloc;  // [0] entries, [1] mask words, cells of the lists of cells[]:
                               // [2] S <= 448, [3] the rest, [4] 448 < S <= 832
  uint32_t* cells;             // 3 n_max: cells staging at most 448 candidates (all pipelined
                               // passes), the others, cells staging 449..832 (pipelined
                               // density and IAD)
  int64_t sent_cap;
  int64_t mask_cap;
  // momentum records as planes: (offset, 1/h^2), (v, m),
  // (B_n/h^3, P/(Omega rho^2), c, 1/rho), (C00 C01 C02 C11), (C12 C22)
  float4* recA;
  float4* recV;
  float4* recQ;
  float4* recC;
  float2* recC2;
  int find_mask_blocks;   // persistent CTAs of the mask-writing search
  int pass_blocks[12];    // persistent CTAs of the density, IAD, momentum passes (general
                          // kernels, then pipelined ones at +3; the plain-configuration
                          // kernels at +6)

  // reductions
  sph::Reduce red;
  unsigned long long* stats;  // kStats cumulative counters (sph_stats)

  // per-stage timing (sph_profile): a ring of event sets, one per step
  int prof;
  int prof_slot;
  cudaEvent_t* prof_ev;   // kProfRing * (SPH_NSTAGE + 2)
  double prof_ms[SPH_NSTAGE];
  int64_t prof_steps;

  // self-gravity tree scratch (sph_gravity.cu), grown on demand
  void* grav_buf;
  size_t grav_bytes;

  // host-step mirrors
  int find_blocks;      // persistent CTAs of the neighbour search (occupancy x SMs)
  double* hm_buf;       // device mirror storage for sph_step_host
  cudaStream_t hs_stream;  // sph_step_host: second stream for the overlapped copies
  cudaEvent_t hs_ev[6];    // sph_step_host: start, inputs in (2), sorted, momentum done, copies done
  // set by sph_step_host around its sph_step call: wait for hook_wait_a
  // before the first gather part and hook_wait before the second; record
  // hook_sorted after the sort and hook_mom after the momentum pass
  cudaEvent_t hook_wait_a, hook_wait, hook_sorted, hook_mom;
  // set by sph_step_host when the caller's arrays are pinned: the update
  // writes the new state straight into them (m, id and du_prev NULL)
  const sph::StateView* hook_update_dst;
  int64_t* hm_id;
  int64_t hm_n;
};

namespace sph {

// --- error helpers (sph_api.cu) ---
int set_error(sph_ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(sph_ctx* ctx, cudaError_t e, const char* what);

// --- sph_sort.cu ---
// Grid from the particles' extent + h_max; zero the cell table.
void launch_grid(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st);
// Counting sort by Morton cell code, deterministic order within cells; gathers
// `in` into the sorted scratch ctx->s and builds pos32 / cell3 / cell_of.
// Sort and gather: launch_sort (cells, order, first gather part) then
// launch_gather_b (velocities, integrator history); launch_sort_gather does both.
// wait_gather (may be null): an event the first gather part waits for (the
// cell keys and order only read x, y, z and h)
void launch_sort(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st,
                 cudaEvent_t wait_gather = nullptr);
void launch_gather_b(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st);
void launch_sort_gather(sph_ctx* ctx, const StateView& in, int64_t n, cudaStream_t st);
// Recompute pos32 / cell3 for an already-sorted state (no permutation).
void launch_copy_state(const StateView& dst, const StateView& src, int64_t n, cudaStream_t st,
                       sph_ctx* ctx);

// --- sph_neighbors.cu ---
void launch_find_neighbors(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st);
void launch_export_neighbors(sph_ctx* ctx, const StateView& s, int64_t n, int32_t* counts,
                             int64_t* ids, cudaStream_t st);

// --- sph_pairs_fp64.cu ---
void launch_density_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st);
void launch_iad_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n, cudaStream_t st);
void launch_momentum_f64(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st);

// --- sph_staged.cu (SPH_FP32_MIXED with SPH_PAIRS_STAGED) ---
void launch_find_masks(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st);
void launch_density_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                           cudaStream_t st);
void launch_iad_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                       cudaStream_t st);
void launch_momentum_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                            cudaStream_t st);
void launch_export_masks(sph_ctx* ctx, const StateView& s, int64_t n, int32_t* counts,
                         int64_t* ids, cudaStream_t st);

// True when the context's pair sums run on cell-staged candidates.
inline bool staged_pairs(const sph_ctx* ctx) {
  return ctx->prm.precision == SPH_FP32_MIXED && ctx->prm.pair_mode == SPH_PAIRS_STAGED;
}

// --- sph_pairs_fp32.cu ---
void launch_density_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                        cudaStream_t st);
void launch_iad_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n, cudaStream_t st);
void launch_momentum_f32(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                         cudaStream_t st);

// --- sph_update.cu ---
void launch_timestep(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n, double* dt_io,
                     cudaStream_t st);
// Table of the smoothing-length factor per neighbour count (rebuilt when
// ng_target changes).
void launch_hfac_table(sph_ctx* ctx, cudaStream_t st);
// Update from the sorted scratch `s` into the caller's state `dst`.
void launch_update(sph_ctx* ctx, const StateView& s, const OutView& o, const StateView& dst,
                   int64_t n, const double* dt_io, cudaStream_t st);
void launch_diagnostics(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st);

}  // namespace sph
