// Batched ensemble: many independent SPH boxes (uneven sizes, their own
// viscosity alpha and time step) advanced together by ONE persistent
// cooperative kernel per call, for any number of steps; the launch can be
// captured in a CUDA graph (sph_ensemble_capture / sph_ensemble_replay).
//
// Every step runs the single-box pipeline phase by phase over ALL boxes at
// once: the work items of a phase (particles, occupied cells or boxes) of all
// boxes are spread over the whole persistent grid, so boxes of 512 and of
// 110,592 particles are load-balanced together.  Phases are separated by a
// software grid barrier whose spin is bounded: if a block waits longer than
// about two seconds it raises SPH_FLAG_TIMEOUT, sets an abort word and every
// block returns, so a fault never hangs the device.  The per-particle work
// uses the same device code as the single-box step (sph_find.cuh,
// sph_pairs32.cuh), in the FP32-mixed precision.
//
// Phases of one step (section numbers of the paper in parentheses):
//   reset -> extent (h_max, open-axis bounds) -> grid -> count -> scan
//   (cell start, occupied cells) -> cell items -> scatter -> in-cell order ->
//   gather -> findNeighbors (4.1) -> density + EOS + dt candidates (Eq. 1,
//   4.2) -> IAD -> momentum/energy (Eqs. 2-5) -> dt -> update (4.1).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sph_device.cuh"
#include "sph_find.cuh"
#include "sph_internal.cuh"
#include "sph_pairs32.cuh"
#include "sph_tile.cuh"

namespace sph {
namespace ens {

constexpr int kThreads = 32 * find::kFindWarps;  // 4 warps: one find window each
constexpr long long kSpinLimit = 20000000;        // x ~100 ns: about two seconds

struct Box {
  int64_t p0, n;        // particle range in the concatenated arrays
  Grid g;               // this step's grid
  int64_t tbl_off;      // offset of the box's cell table
  int cap_bits;         // table capacity: 2^(3 cap_bits) codes
  double lo[3], hi[3];  // box corners (periodic axes)
  int periodic[3];
  double alpha;
  double dt, dt_prev;
  double q;             // dt / (2 dt_prev), 0 on the first step (Adams-Bashforth weight)
  unsigned long long hmax_o, xmin_o[3], xmax_o[3];  // ordered-integer reductions
  unsigned long long qmin_o;                         // min h/c
  int64_t item0;        // first global cell item of the box
  int has_nonfinite;
};

constexpr int kPhases = 15;

struct Sync {
  unsigned int count;
  unsigned int gen;
  unsigned int abort;
  unsigned int pad;
  // phase timer: nanoseconds between the barrier completions seen by block 0
  // (the slowest block's time for each phase), and the number of steps
  unsigned long long ptime[kPhases];
  unsigned long long psteps;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Args {
  Box* boxes;
  int nbox;
  int64_t n;             // total particles
  const int32_t* box_of;
  StateView in;          // caller state (concatenated, permuted in place)
  OutView out;           // caller outputs
  StateView s;           // sorted scratch
  uint32_t* code;
  uint32_t* slot;
  int32_t* perm_tmp;
  int32_t* perm;
  uint32_t* tbl_count;
  uint32_t* tbl_start;
  uint32_t* occ;         // per box at [p0, p0 + n_occ)
  int64_t* item_off;     // nbox + 1: prefix of occupied cells
  float4* pos32;
  float4* rec_d;
  float4* rec_i;
  float4* rec_m;
  int32_t* nn;
  uint32_t* nbr;
  const double* hfac;    // kMaxSlots + 1: 0.5 (1 + cbrt(ng_target / max(k, 1))) for count k
  double* dt_io;         // per box: dt_{n-1} in, dt_n out
  uint32_t* err;
  Sync* sync;
  sph_params prm;
  float Bn;
  double cell_factor;    // cells of side >= cell_factor * 2 h_max
  int skip_block;        // test hook (sph_ens_config::test_skip_block)
  int tpp;               // threads per particle of the density and IAD phases (1, 2, 4)
  int tpm;               // threads per particle of the momentum phase (1, 2, 4)
};

// --- ordered-integer encodings of doubles for atomic min/max ---
__device__ __forceinline__ unsigned long long ord(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord(unsigned long long o) {
  const unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
  return __longlong_as_double((long long)b);
}

// Grid barrier with a bounded wait.  Returns false if the step must stop
// (this block timed out, or another block did).
__device__ bool grid_sync(Sync* sy, uint32_t* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &sy->gen;
    volatile unsigned int* vab = &sy->abort;
    const unsigned int g0 = *vgen;
    __threadfence();
    ok = 1;
    if (atomicAdd(&sy->count, 1u) == gridDim.x - 1) {
      sy->count = 0;
      __threadfence();
      atomicAdd(&sy->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g0) {
        if (*vab) {
          ok = 0;
          break;
        }
        if (++spins > kSpinLimit) {
          atomicExch(&sy->abort, 1u);
          atomicOr(err, (uint32_t)SPH_FLAG_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (*vab) ok = 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int box_of_item(const int64_t* item_off, int nbox, int64_t item) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (item_off[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- phases --
__device__ void ph_reset(const Args& A) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < A.nbox; b += gridDim.x * blockDim.x) {
    Box& B = A.boxes[b];
    B.hmax_o = ord(0.0);
    B.qmin_o = ord(INFINITY);
    for (int k = 0; k < 3; ++k) {
      B.xmin_o[k] = ord(INFINITY);
      B.xmax_o[k] = ord(-INFINITY);
    }
    B.dt_prev = A.dt_io[b];
  }
}

// h_max and open-axis bounds per box (warp-aggregated when a warp holds one box)
__device__ void ph_extent(const Args& A) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < A.n; base += stride) {
    const int64_t p = base + threadIdx.x;
    const bool on = p < A.n;
    const int b = on ? A.box_of[p] : -1;
    double h = on ? A.in.h[p] : 0.0;
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if (on) {
      v[0] = v[3] = A.in.x[p];
      v[1] = v[4] = A.in.y[p];
      v[2] = v[5] = A.in.z[p];
    }
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (__all_sync(0xffffffffu, b == b0 || b < 0) && b0 >= 0) {
      // one box for the whole warp: reduce only the open axes' extents (the
      // box decides, so the branches are uniform), on ordered integer keys
      // (FP64 min/max run at 1/64 of the FP32 rate on this part); NaN takes
      // the neutral key, as fmin/fmax would ignore it
      const Box& Bw = A.boxes[b0];
      long long kh = okey(h, 0);
      long long kv[6];
      for (int k = 0; k < 3; ++k) {
        kv[k] = okey(v[k], kKeyInf);
        kv[3 + k] = okey(v[3 + k], -kKeyInf);
      }
      for (int o = 16; o > 0; o >>= 1) {
        kh = max(kh, __shfl_xor_sync(0xffffffffu, kh, o));
        for (int k = 0; k < 3; ++k) {
          if (Bw.periodic[k]) continue;
          kv[k] = min(kv[k], __shfl_xor_sync(0xffffffffu, kv[k], o));
          kv[3 + k] = max(kv[3 + k], __shfl_xor_sync(0xffffffffu, kv[3 + k], o));
        }
      }
      if (lane == 0) {
        Box& B = A.boxes[b0];
        atomicMax(&B.hmax_o, ord(from_okey(kh)));
        for (int k = 0; k < 3; ++k) {  // the extent is needed on open axes only
          if (B.periodic[k]) continue;
          atomicMin(&B.xmin_o[k], ord(from_okey(kv[k])));
          atomicMax(&B.xmax_o[k], ord(from_okey(kv[3 + k])));
        }
      }
    } else if (on) {
      Box& B = A.boxes[b];
      atomicMax(&B.hmax_o, ord(h));
      for (int k = 0; k < 3; ++k) {
        if (B.periodic[k]) continue;
        atomicMin(&B.xmin_o[k], ord(v[k]));
        atomicMax(&B.xmax_o[k], ord(v[3 + k]));
      }
    }
  }
}

// Grid of each box (same rules as the single-box step, cells of side
// >= cell_factor * 2 h_max, at most 2^cap_bits per axis); zero its table.
__device__ void ph_grid(const Args& A) {
  for (int b = blockIdx.x; b < A.nbox; b += gridDim.x) {
    Box& B = A.boxes[b];
    __shared__ Grid G;
    if (threadIdx.x == 0) {
      const double hmax = unord(B.hmax_o);
      G.hmax = hmax;
      int maxnc = 1;
      for (int ax = 0; ax < 3; ++ax) {
        const int per = B.periodic[ax] ? 1 : 0;
        double lo, L;
        if (per) {
          lo = B.lo[ax];
          L = B.hi[ax] - B.lo[ax];
          if (!(2.0 * hmax < 0.5 * L)) atomicOr(A.err, (uint32_t)SPH_FLAG_BAD_BOX);
        } else {
          lo = unord(B.xmin_o[ax]);
          L = unord(B.xmax_o[ax]) - lo;
        }
        int nc = 1;
        if (hmax > 0.0 && L > 0.0) {
          const double q = floor(L / (A.cell_factor * 2.0 * hmax * (1.0 + 1e-9)));
          const double cap = (double)(1 << B.cap_bits);
          nc = q < 1.0 ? 1 : (q > cap ? (1 << B.cap_bits) : (int)q);
        }
        const double cs = L > 0.0 ? L / nc : 0.0;
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
      B.g = G;
    }
    __syncthreads();
    const uint32_t size = G.tbl_size;
    for (uint32_t i = threadIdx.x; i < size; i += blockDim.x) A.tbl_count[B.tbl_off + i] = 0u;
    __syncthreads();
  }
}

__device__ __forceinline__ void cell_of(const Grid& g, double x, double y, double z, int& ix,
                                        int& iy, int& iz) {
  const double p[3] = {x, y, z};
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

__device__ void ph_count(const Args& A) {
  const int lane = threadIdx.x & 31;
  // warp-uniform loop (p - lane is the warp's first particle)
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p - lane < A.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const bool valid = p < A.n;
    uint64_t key = ~0ull;
    uint32_t c = 0;
    int64_t off = 0;
    if (valid) {
      const Box& B = A.boxes[A.box_of[p]];
      int ix, iy, iz;
      cell_of(B.g, A.in.x[p], A.in.y[p], A.in.z[p], ix, iy, iz);
      c = morton3(ix, iy, iz);
      A.code[p] = c;
      off = B.tbl_off;
      key = ((uint64_t)off << 32) | c;
    }
    // one atomic per group of lanes with the same box and cell (the slot order
    // inside a cell does not matter: ph_order ranks by previous index)
    const unsigned same = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(same) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&A.tbl_count[off + c], (uint32_t)__popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) A.slot[p] = base + (uint32_t)__popc(same & ((1u << lane) - 1u));
  }
}

// Exclusive scan of a box's cell counts (one block per box) -> cell start
// (absolute particle index) and the box's occupied cells in Morton order.
__device__ void ph_scan(const Args& A) {
  __shared__ uint32_t sh_s[kThreads], sh_o[kThreads];
  for (int b = blockIdx.x; b < A.nbox; b += gridDim.x) {
    Box& B = A.boxes[b];
    const uint32_t size = B.g.tbl_size;
    const uint32_t seg = (size + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = threadIdx.x * seg, i1 = min(size, i0 + seg);
    const uint32_t* cnt = A.tbl_count + B.tbl_off;
    uint32_t s = 0, o = 0;
    for (uint32_t i = i0; i < i1; ++i) {
      s += cnt[i];
      o += cnt[i] ? 1u : 0u;
    }
    sh_s[threadIdx.x] = s;
    sh_o[threadIdx.x] = o;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t as = 0, ao = 0;
      for (int t = 0; t < (int)blockDim.x; ++t) {
        const uint32_t ts = sh_s[t], to = sh_o[t];
        sh_s[t] = as;
        sh_o[t] = ao;
        as += ts;
        ao += to;
      }
      B.g.n_occ = ao;
    }
    __syncthreads();
    uint32_t ps = sh_s[threadIdx.x], po = sh_o[threadIdx.x];
    uint32_t* start = A.tbl_start + B.tbl_off;
    for (uint32_t i = i0; i < i1; ++i) {
      start[i] = (uint32_t)(B.p0 + ps);
      if (cnt[i]) A.occ[B.p0 + po++] = i;
      ps += cnt[i];
    }
    __syncthreads();
  }
}

// Global numbering of occupied-cell work items (block 0).
__device__ void ph_items(const Args& A) {
  if (blockIdx.x != 0) return;
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int b = 0; b < A.nbox; ++b) {
      A.boxes[b].item0 = acc;
      A.item_off[b] = acc;
      acc += A.boxes[b].g.n_occ;
    }
    A.item_off[A.nbox] = acc;
  }
}

__device__ void ph_scatter(const Args& A) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < A.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Box& B = A.boxes[A.box_of[p]];
    A.perm_tmp[A.tbl_start[B.tbl_off + A.code[p]] + A.slot[p]] = (int32_t)p;
  }
}

// One warp per occupied cell: members ordered by previous position.
__device__ void ph_order(const Args& A) {
  const int lane = threadIdx.x & 31;
  const int64_t nitems = A.item_off[A.nbox];
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems;
       it += warps) {
    const int b = box_of_item(A.item_off, A.nbox, it);
    const Box& B = A.boxes[b];
    const uint32_t code = A.occ[B.p0 + (it - B.item0)];
    const uint32_t s0 = A.tbl_start[B.tbl_off + code], cnt = A.tbl_count[B.tbl_off + code];
    for (uint32_t j0 = 0; j0 < cnt; j0 += 32) {
      const uint32_t j = j0 + lane;
      const int32_t v = j < cnt ? A.perm_tmp[s0 + j] : 0x7fffffff;
      uint32_t rank = 0;
      for (uint32_t l0 = 0; l0 < cnt; l0 += 32) {
        const int32_t w = (l0 + lane < cnt) ? A.perm_tmp[s0 + l0 + lane] : 0x7fffffff;
        for (int q = 0; q < 32; ++q) {
          const int32_t wq = __shfl_sync(0xffffffffu, w, q);
          rank += (l0 + q < cnt && wq < v) ? 1u : 0u;
        }
      }
      if (j < cnt) A.perm[s0 + rank] = v;
    }
  }
}

__device__ void ph_gather(const Args& A) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < A.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Grid& g = A.boxes[A.box_of[p]].g;
    const int64_t s = A.perm[p];
    const double x = A.in.x[s], y = A.in.y[s], z = A.in.z[s], h = A.in.h[s];
    const double vx = A.in.vx[s], vy = A.in.vy[s], vz = A.in.vz[s], m = A.in.m[s];
    A.s.x[p] = x;
    A.s.y[p] = y;
    A.s.z[p] = z;
    A.s.h[p] = h;
    A.s.vx[p] = vx;
    A.s.vy[p] = vy;
    A.s.vz[p] = vz;
    A.s.vxh[p] = A.in.vxh[s];
    A.s.vyh[p] = A.in.vyh[s];
    A.s.vzh[p] = A.in.vzh[s];
    A.s.m[p] = m;
    A.s.u[p] = A.in.u[s];
    A.s.du_prev[p] = A.in.du_prev[s];
    A.s.id[p] = A.in.id[s];
    const uint32_t c = A.code[s];
    const int ix = compact3_bits(c), iy = compact3_bits(c >> 1), iz = compact3_bits(c >> 2);
    // f32_rn equals the FP64 conversion bit for bit, on the integer pipes
    const float ox = f32_rn(x - (g.lo[0] + ix * g.cs[0]));
    const float oy = f32_rn(y - (g.lo[1] + iy * g.cs[1]));
    const float oz = f32_rn(z - (g.lo[2] + iz * g.cs[2]));
    const float m32 = f32_rn(m);
    A.pos32[p] = make_float4(ox, oy, oz, f32_rn(h));
    A.rec_d[p] = make_float4(ox, oy, oz, m32);
    A.rec_m[5 * p + 1] = make_float4(f32_rn(vx), f32_rn(vy), f32_rn(vz), m32);
  }
}

template <int WIN>
__device__ void ph_find(const Args& A, find::FindWarpSmemT<WIN>& W) {
  const int64_t nitems = A.item_off[A.nbox];
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long tested = 0, exact = 0;
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems;
       it += warps) {
    const int b = box_of_item(A.item_off, A.nbox, it);
    const Box& B = A.boxes[b];
    const uint32_t code = A.occ[B.p0 + (it - B.item0)];
    const uint32_t* ts = A.tbl_start + B.tbl_off;
    const uint32_t* tc = A.tbl_count + B.tbl_off;
    if (B.g.wrap32)
      find::find_cell<true, WIN>(B.g, code, A.s, A.pos32, ts, tc, A.nn, A.nbr, A.prm.max_nb,
                                 A.err, W, tested, exact);
    else
      find::find_cell<false, WIN>(B.g, code, A.s, A.pos32, ts, tc, A.nn, A.nbr, A.prm.max_nb,
                                  A.err, W, tested, exact);
  }
}

__device__ __forceinline__ pairs32::F32 f32_of(const Args& A) {
  pairs32::F32 f;
  f.pos = A.pos32;
  f.rec_d = A.rec_d;
  f.rec_i = A.rec_i;
  f.rec_m = A.rec_m;
  f.ktab = nullptr;  // the ensemble runs the exact kernel
  return f;
}
__device__ __forceinline__ pairs32::Lists lists_of(const Args& A) {
  pairs32::Lists l;
  l.nn = A.nn;
  l.nbr = A.nbr;
  l.max_nb = A.prm.max_nb;
  return l;
}

// The pair phases run NSUB threads per particle (sph_ens_config::
// threads_per_particle): thread t of the grid-stride sweep works on particle
// t / NSUB as sub-lane t % NSUB, and every warp runs the loop uniformly (the
// group sums are warp shuffles).  The box's Grid is copied into registers,
// since the pair loop reads it for every pair.

// density + EOS, and the per-box minimum of h / c for the time step
// N > 0: the kernel exponent fixed at compile time (sinc_n = N, and for the
// density no grad-h terms); N = 0: both taken from the parameters.
template <int NSUB, int N>
__device__ void ph_density_t(const Args& A) {
  const pairs32::F32 f = f32_of(A);
  const pairs32::Lists L = lists_of(A);
  const int lane = threadIdx.x & 31, sub = threadIdx.x % NSUB;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, total = A.n * NSUB;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t t = base + threadIdx.x;
    const bool on = t < total;
    const int64_t p = on ? t / NSUB : 0;
    const int b = on ? A.box_of[p] : -1;
    const Grid g = A.boxes[on ? b : 0].g;
    pairs32::density_one<NSUB, N>(p, g, f, A.out, A.s.u, L, A.Bn, (int)A.prm.sinc_n,
                                  A.prm.gamma, A.err, on, sub, N == 0 && A.prm.gradh != 0);
    const bool own = on && sub == 0;
    const double q = own ? A.s.h[p] / A.out.c[p] : INFINITY;
    const int bq = own ? b : -1;
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (__all_sync(0xffffffffu, b == b0 || b < 0) && b0 >= 0) {
      // the warp's minimum on ordered integer keys (NaN ignored, as by fmin)
      long long km = okey(q, kKeyInf);
      for (int o = 16; o > 0; o >>= 1) km = min(km, __shfl_xor_sync(0xffffffffu, km, o));
      if (lane == 0) atomicMin(&A.boxes[b0].qmin_o, ord(from_okey(km)));
    } else if (bq >= 0) {
      atomicMin(&A.boxes[bq].qmin_o, ord(q));
    }
  }
}

template <int NSUB, int N>
__device__ void ph_iad_t(const Args& A) {
  const pairs32::F32 f = f32_of(A);
  const pairs32::Lists L = lists_of(A);
  const int sub = threadIdx.x % NSUB;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, total = A.n * NSUB;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t t = base + threadIdx.x;
    const bool on = t < total;
    const int64_t p = on ? t / NSUB : 0;
    const Grid g = A.boxes[on ? A.box_of[p] : 0].g;
    pairs32::iad_one<NSUB, N>(p, g, f, A.out, L, (int)A.prm.sinc_n, A.err, on, sub);
  }
}

template <int NSUB, int N>
__device__ void ph_momentum_t(const Args& A) {
  const pairs32::F32 f = f32_of(A);
  const pairs32::Lists L = lists_of(A);
  const int sub = threadIdx.x % NSUB;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, total = A.n * NSUB;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const int64_t t = base + threadIdx.x;
    const bool on = t < total;
    const int64_t p = on ? t / NSUB : 0;
    const Box& B = A.boxes[on ? A.box_of[p] : 0];
    const Grid g = B.g;
    pairs32::momentum_one<NSUB, N>(p, g, f, A.out, L, (int)A.prm.sinc_n, (float)B.alpha, A.err,
                                   on, sub);
  }
}

template <int N>
__device__ void ph_density_n(const Args& A) {
  if (A.tpp == 4)
    ph_density_t<4, N>(A);
  else if (A.tpp == 2)
    ph_density_t<2, N>(A);
  else
    ph_density_t<1, N>(A);
}
template <int N>
__device__ void ph_iad_n(const Args& A) {
  if (A.tpp == 4)
    ph_iad_t<4, N>(A);
  else if (A.tpp == 2)
    ph_iad_t<2, N>(A);
  else
    ph_iad_t<1, N>(A);
}
template <int N>
__device__ void ph_momentum_n(const Args& A) {
  if (A.tpm == 4)
    ph_momentum_t<4, N>(A);
  else if (A.tpm == 2)
    ph_momentum_t<2, N>(A);
  else
    ph_momentum_t<1, N>(A);
}
// density and IAD: the default kernel (n = 6, no grad-h terms) with its
// exponent fixed at compile time, any other with the parameters' values;
// momentum keeps the run-time exponent (its fixed-exponent body spilled at
// the kernel's 80-register cap)
__device__ void ph_density(const Args& A) {
  if (A.prm.sinc_n == 6.0 && !A.prm.gradh)
    ph_density_n<6>(A);
  else
    ph_density_n<0>(A);
}
__device__ void ph_iad(const Args& A) {
  if (A.prm.sinc_n == 6.0)
    ph_iad_n<6>(A);
  else
    ph_iad_n<0>(A);
}
__device__ void ph_momentum(const Args& A) { ph_momentum_n<0>(A); }

// dt_n = min(courant * min h/c, dt_growth * dt_{n-1}) per box (section 4.2)
__device__ void ph_dt(const Args& A) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < A.nbox; b += gridDim.x * blockDim.x) {
    Box& B = A.boxes[b];
    double dt = A.prm.courant * unord(B.qmin_o);
    if (B.dt_prev > 0.0) dt = fmin(dt, A.prm.dt_growth * B.dt_prev);
    if (!isfinite(dt) || !(dt > 0.0)) atomicOr(A.err, (uint32_t)SPH_FLAG_NONFINITE);
    B.dt = dt;
    B.q = B.dt_prev > 0.0 ? dt / (2.0 * B.dt_prev) : 0.0;
    A.dt_io[b] = dt;
  }
}

// Update of section 4.1 (leapfrog x, v; Adams-Bashforth u; h toward the
// target count), from the sorted scratch into the caller's arrays.
__device__ void ph_update(const Args& A) {
  const sph_params& prm = A.prm;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < A.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Box& B = A.boxes[A.box_of[p]];
    const double dt = B.dt, dt_prev = B.dt_prev;
    const double delta = 0.5 * (dt + dt_prev);
    const double q = B.q;
    const double a3[3] = {A.out.ax[p], A.out.ay[p], A.out.az[p]};
    const double x3[3] = {A.s.x[p], A.s.y[p], A.s.z[p]};
    const double vh3[3] = {A.s.vxh[p], A.s.vyh[p], A.s.vzh[p]};
    double xn[3], vn[3], vhn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      vhn[k] = vh3[k] + a3[k] * delta;
      double xk = x3[k] + dt * vhn[k];
      if (B.periodic[k]) {
        // the tests on ordered integer keys (a NaN position takes the key of
        // lo: no wrap, as in the FP comparison)
        const double L = B.hi[k] - B.lo[k];
        const long long klo = okey(B.lo[k], 0), kx = okey(xk, klo);
        if (kx >= okey(B.hi[k], 0))
          xk -= L;
        else if (kx < klo)
          xk += L;
      }
      xn[k] = xk;
      vn[k] = vhn[k] + 0.5 * dt * a3[k];
    }
    const double du = A.out.du[p];
    const double u = A.s.u[p];
    const double un = dt_prev > 0.0 ? u + dt * ((1.0 + q) * du - q * A.s.du_prev[p]) : u + dt * du;
    double h = A.s.h[p];
    // h (0.5 (1 + c)) equals (h 0.5) (1 + c) bit for bit (scaling by 0.5 is
    // exact), so the tabulated factor changes no result; counts are at most
    // kMaxSlots (a larger stencil is flagged and its counts are 0)
    if (prm.ng_target > 0) h = h * __ldg(A.hfac + min(max(A.nn[p], 0), kMaxSlots));
    A.in.x[p] = xn[0];
    A.in.y[p] = xn[1];
    A.in.z[p] = xn[2];
    A.in.vx[p] = vn[0];
    A.in.vy[p] = vn[1];
    A.in.vz[p] = vn[2];
    A.in.vxh[p] = vhn[0];
    A.in.vyh[p] = vhn[1];
    A.in.vzh[p] = vhn[2];
    A.in.u[p] = un;
    A.in.du_prev[p] = du;
    A.in.h[p] = h;
    A.in.m[p] = A.s.m[p];
    A.in.id[p] = A.s.id[p];
  }
}

// The h factors of the update for every possible count (the expression of
// the single-box table, over the counts a stencil can hold).
__global__ void k_ens_hfac(double* tab, int ng) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= kMaxSlots; k += gridDim.x * blockDim.x) {
    const int kk = k > 1 ? k : 1;
    tab[k] = 0.5 * (1.0 + cbrt((double)ng / (double)kk));
  }
}

template <int WIN>
__global__ void __launch_bounds__(kThreads, 6) k_ensemble(Args A, int steps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  find::FindWarpSmemT<WIN>& W =
      reinterpret_cast<find::FindWarpSmemT<WIN>*>(smem_raw)[threadIdx.x >> 5];
  if ((int)blockIdx.x == A.skip_block) return;  // test hook: the others' wait expires
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long t_last = timer ? global_ns() : 0ull;
  // runs one phase, the grid barrier after it, and the phase timer
#define SPH_PHASE(k, call)                                   \
  call;                                                      \
  if (!grid_sync(A.sync, A.err)) return;                     \
  if (timer) {                                               \
    const unsigned long long t = global_ns();                \
    A.sync->ptime[k] += t - t_last;                          \
    t_last = t;                                              \
  }
  for (int step = 0; step < steps; ++step) {
    SPH_PHASE(0, ph_reset(A))
    SPH_PHASE(1, ph_extent(A))
    SPH_PHASE(2, ph_grid(A))
    SPH_PHASE(3, ph_count(A))
    SPH_PHASE(4, ph_scan(A))
    SPH_PHASE(5, ph_items(A))
    SPH_PHASE(6, ph_scatter(A))
    SPH_PHASE(7, ph_order(A))
    SPH_PHASE(8, ph_gather(A))
    SPH_PHASE(9, ph_find<WIN>(A, W))
    SPH_PHASE(10, ph_density(A))
    SPH_PHASE(11, ph_iad(A))
    SPH_PHASE(12, ph_momentum(A))
    SPH_PHASE(13, ph_dt(A))
    SPH_PHASE(14, ph_update(A))
    if (timer) A.sync->psteps += 1;
  }
#undef SPH_PHASE
}

}  // namespace ens
}  // namespace sph

// ------------------------------------------------------------------ host --
using sph::ens::Args;
using sph::ens::Box;

struct sph_ens {
  sph_params prm;
  int nbox;
  int64_t n;
  int device, sm_count;
  double Bn;
  sph_ens_config cfg;
  Box* boxes;             // device
  Box* boxes_h;           // host copy of the static fields
  int32_t* box_of;
  int64_t* item_off;
  double* sbuf;
  int64_t* s_id;
  uint32_t *code, *slot;
  int32_t *perm_tmp, *perm;
  uint32_t *tbl_count, *tbl_start, *occ;
  int64_t tbl_total;
  float4 *pos32, *rec_d, *rec_i, *rec_m;
  int32_t* nn;
  uint32_t* nbr;
  double* hfac;
  uint32_t* err;
  sph::ens::Sync* sync;
  int blocks;
  cudaGraphExec_t graph;
  char last_error[256];
  int64_t launches;
};

namespace {

int ens_fail(sph_ens* e, int code, const char* fmt, ...) {
  if (e) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(e->last_error, sizeof(e->last_error), fmt, ap);
    va_end(ap);
  }
  return code;
}

double kernel_norm_host_ens(double n) {
  // same normalisation as the single-box context: composite Simpson, 2^16 panels
  const int N = 1 << 16;
  const double hs = 2.0 / N;
  double s = 0.0, comp = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double v = i * hs;
    double f = 0.0;
    if (v > 0.0) {
      const double x = 1.5707963267948966192 * v;
      f = pow(sin(x) / x, n) * v * v;
    }
    const double w = (i == 0 || i == N) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    const double y = w * f - comp;
    const double t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  return 1.0 / (4.0 * 3.14159265358979323846 * (s * hs / 3.0));
}

int cap_bits_for(int64_t n) {
  // room for cells down to a quarter of the initial cell volume per axis pair
  const double nc = 2.0 * cbrt((double)(n > 0 ? n : 1) / 16.0);
  int bits = 1;
  while ((1 << bits) < nc && bits < sph::kMaxCellBits) ++bits;
  return bits;
}

Args args_of(sph_ens* e, const sph_state* st, double* dt_dev) {
  Args A;
  memset(&A, 0, sizeof(A));
  A.boxes = e->boxes;
  A.nbox = e->nbox;
  A.n = e->n;
  A.box_of = e->box_of;
  A.in.x = st->x;
  A.in.y = st->y;
  A.in.z = st->z;
  A.in.vx = st->vx;
  A.in.vy = st->vy;
  A.in.vz = st->vz;
  A.in.vxh = st->vxh;
  A.in.vyh = st->vyh;
  A.in.vzh = st->vzh;
  A.in.h = st->h;
  A.in.m = st->m;
  A.in.u = st->u;
  A.in.du_prev = st->du_prev;
  A.in.id = st->id;
  A.out.rho = st->rho;
  A.out.p = st->p;
  A.out.c = st->c;
  A.out.iad = st->iad;
  A.out.ax = st->ax;
  A.out.ay = st->ay;
  A.out.az = st->az;
  A.out.du = st->du;
  A.out.omega = st->omega;
  double* f[13] = {};
  for (int k = 0; k < 13; ++k) f[k] = e->sbuf + (size_t)k * e->n;
  A.s.x = f[0];
  A.s.y = f[1];
  A.s.z = f[2];
  A.s.vx = f[3];
  A.s.vy = f[4];
  A.s.vz = f[5];
  A.s.vxh = f[6];
  A.s.vyh = f[7];
  A.s.vzh = f[8];
  A.s.h = f[9];
  A.s.m = f[10];
  A.s.u = f[11];
  A.s.du_prev = f[12];
  A.s.id = e->s_id;
  A.code = e->code;
  A.slot = e->slot;
  A.perm_tmp = e->perm_tmp;
  A.perm = e->perm;
  A.tbl_count = e->tbl_count;
  A.tbl_start = e->tbl_start;
  A.occ = e->occ;
  A.item_off = e->item_off;
  A.pos32 = e->pos32;
  A.rec_d = e->rec_d;
  A.rec_i = e->rec_i;
  A.rec_m = e->rec_m;
  A.nn = e->nn;
  A.nbr = e->nbr;
  A.hfac = e->hfac;
  A.dt_io = dt_dev;
  A.err = e->err;
  A.sync = e->sync;
  A.prm = e->prm;
  A.Bn = (float)e->Bn;
  A.cell_factor = e->cfg.cell_factor;
  A.skip_block = e->cfg.test_skip_block;
  A.tpp = e->cfg.threads_per_particle;
  A.tpm = e->cfg.momentum_threads;
  return A;
}

int check_ens_state(sph_ens* e, const sph_state* s, const double* dt) {
  if (!e) return SPH_ERR_INVALID_ARG;
  if (!s || !dt) return ens_fail(e, SPH_ERR_INVALID_ARG, "NULL state or dt");
  if (s->n != e->n) return ens_fail(e, SPH_ERR_INVALID_ARG, "state.n != ensemble size");
  const void* req[] = {s->x, s->y, s->z, s->vx, s->vy, s->vz, s->h, s->m, s->u, s->vxh, s->vyh,
                       s->vzh, s->du_prev, s->id, s->rho, s->p, s->c, s->iad, s->ax, s->ay,
                       s->az, s->du};
  for (const void* q : req)
    if (!q) return ens_fail(e, SPH_ERR_INVALID_ARG, "a state or output array is NULL");
  return SPH_OK;
}

// The kernel instance and its shared memory for a find window (tile shape).
template <int WIN>
size_t window_smem() {
  return sph::find::kFindWarps * sizeof(sph::find::FindWarpSmemT<WIN>);
}

int launch(sph_ens* e, const Args& A, int steps, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(e->blocks);
  cfg.blockDim = dim3(sph::ens::kThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err;
  switch (e->cfg.find_window) {
    case 128:
      cfg.dynamicSmemBytes = window_smem<128>();
      err = cudaLaunchKernelEx(&cfg, sph::ens::k_ensemble<128>, A, steps);
      break;
    case 256:
      cfg.dynamicSmemBytes = window_smem<256>();
      err = cudaLaunchKernelEx(&cfg, sph::ens::k_ensemble<256>, A, steps);
      break;
    default:
      cfg.dynamicSmemBytes = window_smem<512>();
      err = cudaLaunchKernelEx(&cfg, sph::ens::k_ensemble<512>, A, steps);
      break;
  }
  if (err != cudaSuccess)
    return ens_fail(e, SPH_ERR_CUDA, "ensemble launch: %s", cudaGetErrorString(err));
  e->launches += 1;
  return SPH_OK;
}

template <int WIN>
cudaError_t occupancy(int* per_sm) {
  const size_t smem = window_smem<WIN>();
  cudaError_t err = cudaFuncSetAttribute(sph::ens::k_ensemble<WIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sph::ens::k_ensemble<WIN>,
                                                        sph::ens::kThreads, smem);
  return err;
}

int configure(sph_ens* e) {
  int per_sm = 0;
  cudaError_t err = e->cfg.find_window == 128   ? occupancy<128>(&per_sm)
                    : e->cfg.find_window == 256 ? occupancy<256>(&per_sm)
                                                : occupancy<512>(&per_sm);
  if (err != cudaSuccess || per_sm < 1)
    return ens_fail(e, SPH_ERR_CUDA, "ensemble occupancy: %s", cudaGetErrorString(err));
  int want = e->cfg.blocks_per_sm > 0 ? e->cfg.blocks_per_sm : per_sm;
  if (want > per_sm) want = per_sm;  // co-residency is required for the grid barrier
  e->blocks = want * e->sm_count;
  return SPH_OK;
}

}  // namespace

extern "C" {

void sph_ens_default_config(sph_ens_config* c) {
  if (!c) return;
  c->cell_factor = 1.0;
  c->blocks_per_sm = 0;
  c->test_skip_block = -1;
  c->find_window = 512;
  c->threads_per_particle = 1;
  c->momentum_threads = 4;
}

int sph_ensemble_init(const sph_params* common, int n_boxes, const int64_t* box_n,
                      const double* box_lo, const double* box_hi, const int* box_periodic,
                      const double* box_alpha, sph_ens** out) {
  if (!out || !common || n_boxes < 1 || !box_n || !box_lo || !box_hi || !box_periodic ||
      !box_alpha)
    return SPH_ERR_INVALID_ARG;
  *out = nullptr;
  if (common->precision != SPH_FP32_MIXED || common->max_nb % 4 != 0 || common->max_nb < 4 ||
      !(common->sinc_n >= 1.0 && common->sinc_n <= 12.0) ||
      common->kernel_mode != SPH_KERNEL_EXACT || common->energy_dt != 0.0)
    return SPH_ERR_INVALID_ARG;
  sph_ens* e = (sph_ens*)calloc(1, sizeof(sph_ens));
  if (!e) return SPH_ERR_OOM;
  e->prm = *common;
  e->nbox = n_boxes;
  sph_ens_default_config(&e->cfg);
  cudaGetDevice(&e->device);
  cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, e->device);
  e->Bn = kernel_norm_host_ens(common->sinc_n);
  e->boxes_h = (Box*)calloc(n_boxes, sizeof(Box));
  int64_t n = 0, tbl = 0;
  for (int b = 0; b < n_boxes; ++b) {
    Box& B = e->boxes_h[b];
    if (box_n[b] < 1) {
      free(e->boxes_h);
      free(e);
      return SPH_ERR_INVALID_ARG;
    }
    B.p0 = n;
    B.n = box_n[b];
    n += box_n[b];
    B.cap_bits = cap_bits_for(box_n[b]);
    B.tbl_off = tbl;
    tbl += (int64_t)1 << (3 * B.cap_bits);
    for (int k = 0; k < 3; ++k) {
      B.lo[k] = box_lo[3 * b + k];
      B.hi[k] = box_hi[3 * b + k];
      B.periodic[k] = box_periodic[3 * b + k] ? 1 : 0;
    }
    B.alpha = box_alpha[b];
  }
  if (n > sph::kMaxParticles) {
    free(e->boxes_h);
    free(e);
    return SPH_ERR_INVALID_ARG;
  }
  e->n = n;
  e->tbl_total = tbl;
  cudaError_t err = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (err == cudaSuccess) err = cudaMalloc(p, bytes ? bytes : 8);
  };
  const size_t N = (size_t)n;
  A((void**)&e->boxes, sizeof(Box) * n_boxes);
  A((void**)&e->box_of, 4 * N);
  A((void**)&e->item_off, 8 * (size_t)(n_boxes + 1));
  A((void**)&e->sbuf, 8 * 13 * N);
  A((void**)&e->s_id, 8 * N);
  A((void**)&e->code, 4 * N);
  A((void**)&e->slot, 4 * N);
  A((void**)&e->perm_tmp, 4 * N);
  A((void**)&e->perm, 4 * N);
  A((void**)&e->tbl_count, 4 * (size_t)tbl);
  A((void**)&e->tbl_start, 4 * (size_t)tbl);
  A((void**)&e->occ, 4 * N);
  A((void**)&e->pos32, 16 * N);
  A((void**)&e->rec_d, 16 * N);
  A((void**)&e->rec_i, 16 * N);
  A((void**)&e->rec_m, 80 * N);
  A((void**)&e->nn, 4 * N);
  A((void**)&e->nbr, 4 * N * (size_t)common->max_nb);
  A((void**)&e->hfac, 8 * (size_t)(sph::kMaxSlots + 1));
  A((void**)&e->err, 4);
  A((void**)&e->sync, sizeof(sph::ens::Sync));
  if (err == cudaSuccess) {
    int32_t* bo = (int32_t*)malloc(4 * N);
    for (int b = 0; b < n_boxes; ++b)
      for (int64_t i = 0; i < box_n[b]; ++i) bo[e->boxes_h[b].p0 + i] = b;
    err = cudaMemcpy(e->box_of, bo, 4 * N, cudaMemcpyHostToDevice);
    free(bo);
  }
  if (err == cudaSuccess)
    err = cudaMemcpy(e->boxes, e->boxes_h, sizeof(Box) * n_boxes, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemset(e->err, 0, 4);
  if (err == cudaSuccess) {
    sph::ens::k_ens_hfac<<<64, 256>>>(e->hfac, common->ng_target > 0 ? common->ng_target : 1);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemset(e->sync, 0, sizeof(sph::ens::Sync));
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  int rc = err == cudaSuccess ? configure(e) : SPH_ERR_OOM;
  if (rc != SPH_OK) {
    sph_ensemble_destroy(e);
    return rc;
  }
  *out = e;
  return SPH_OK;
}

void sph_ensemble_destroy(sph_ens* e) {
  if (!e) return;
  cudaDeviceSynchronize();
  if (e->graph) cudaGraphExecDestroy(e->graph);
  void* ptrs[] = {e->boxes, e->box_of, e->item_off, e->sbuf, e->s_id, e->code, e->slot,
                  e->perm_tmp, e->perm, e->tbl_count, e->tbl_start, e->occ, e->pos32,
                  e->rec_d, e->rec_i, e->rec_m, e->nn, e->nbr, e->hfac, e->err, e->sync};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(e->boxes_h);
  free(e);
}

int sph_ensemble_set_config(sph_ens* e, const sph_ens_config* c) {
  if (!e || !c) return SPH_ERR_INVALID_ARG;
  if (!(c->cell_factor >= 1.0 && c->cell_factor <= 4.0) || c->blocks_per_sm < 0)
    return ens_fail(e, SPH_ERR_INVALID_ARG, "cell_factor must be in [1, 4]");
  if (c->find_window != 128 && c->find_window != 256 && c->find_window != 512)
    return ens_fail(e, SPH_ERR_INVALID_ARG, "find_window must be 128, 256 or 512");
  if (c->threads_per_particle != 1 && c->threads_per_particle != 2 &&
      c->threads_per_particle != 4)
    return ens_fail(e, SPH_ERR_INVALID_ARG, "threads_per_particle must be 1, 2 or 4");
  if (c->momentum_threads != 1 && c->momentum_threads != 2 && c->momentum_threads != 4)
    return ens_fail(e, SPH_ERR_INVALID_ARG, "momentum_threads must be 1, 2 or 4");
  e->cfg = *c;
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  return configure(e);
}

int sph_ensemble_step(sph_ens* e, sph_state* state, double* dt_dev, int steps,
                      sph_stream_t stream) {
  int rc = check_ens_state(e, state, dt_dev);
  if (rc != SPH_OK) return rc;
  if (steps < 1) return ens_fail(e, SPH_ERR_INVALID_ARG, "steps < 1");
  return launch(e, args_of(e, state, dt_dev), steps, (cudaStream_t)stream);
}

int sph_ensemble_capture(sph_ens* e, sph_state* state, double* dt_dev, int steps,
                         sph_stream_t stream) {
  int rc = check_ens_state(e, state, dt_dev);
  if (rc != SPH_OK) return rc;
  if (steps < 1) return ens_fail(e, SPH_ERR_INVALID_ARG, "steps < 1");
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return ens_fail(e, SPH_ERR_INVALID_ARG, "capture needs a non-default stream");
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (err != cudaSuccess) return ens_fail(e, SPH_ERR_CUDA, "capture: %s", cudaGetErrorString(err));
  rc = launch(e, args_of(e, state, dt_dev), steps, st);
  err = cudaStreamEndCapture(st, &g);
  if (rc != SPH_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (err != cudaSuccess) return ens_fail(e, SPH_ERR_CUDA, "capture: %s", cudaGetErrorString(err));
  e->launches -= 1;  // counted at replay
  return SPH_OK;
}

int sph_ensemble_replay(sph_ens* e, sph_stream_t stream) {
  if (!e) return SPH_ERR_INVALID_ARG;
  if (!e->graph) return ens_fail(e, SPH_ERR_ORDER, "no captured graph");
  cudaError_t err = cudaGraphLaunch(e->graph, (cudaStream_t)stream);
  if (err != cudaSuccess) return ens_fail(e, SPH_ERR_CUDA, "replay: %s", cudaGetErrorString(err));
  e->launches += 1;
  return SPH_OK;
}

int sph_ensemble_error_word(sph_ens* e, uint32_t* flags) {
  if (!e || !flags) return SPH_ERR_INVALID_ARG;
  cudaError_t err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = cudaMemcpy(flags, e->err, 4, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaMemset(e->err, 0, 4);
  if (err == cudaSuccess) err = cudaMemset(e->sync, 0, sizeof(sph::ens::Sync));
  if (err != cudaSuccess) return ens_fail(e, SPH_ERR_CUDA, "%s", cudaGetErrorString(err));
  return SPH_OK;
}

const char* sph_ensemble_last_error(const sph_ens* e) { return e ? e->last_error : "no context"; }

int sph_ensemble_phase_times(sph_ens* e, double* ms, int64_t* steps) {
  if (!e || !ms || !steps) return SPH_ERR_INVALID_ARG;
  sph::ens::Sync h;
  cudaError_t err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = cudaMemcpy(&h, e->sync, sizeof(h), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) {
    const size_t off = offsetof(sph::ens::Sync, ptime);
    err = cudaMemset((char*)e->sync + off, 0, sizeof(h) - off);
  }
  if (err != cudaSuccess) return ens_fail(e, SPH_ERR_CUDA, "sph_ensemble_phase_times: %s",
                                         cudaGetErrorString(err));
  for (int k = 0; k < sph::ens::kPhases; ++k) ms[k] = 1e-6 * (double)h.ptime[k];
  *steps = (int64_t)h.psteps;
  return SPH_OK;
}

int sph_ensemble_info(const sph_ens* e, int64_t* out) {
  if (!e || !out) return SPH_ERR_INVALID_ARG;
  out[0] = e->n;
  out[1] = e->nbox;
  out[2] = e->blocks;
  out[3] = e->launches;
  return SPH_OK;
}

}  // extern "C"
