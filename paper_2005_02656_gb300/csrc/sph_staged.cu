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
// positions relative to the target cell.  Each target's staged-slot list
// (written by the search from its hit masks) is copied into shared memory;
// the target's sum is split over nsub = kPT / (targets) threads, thread s
// taking entries s, s + nsub, ..., and the nsub partial sums are added in a
// fixed order, so the result does not depend on scheduling.  Cells whose
// staged set or target set exceeds the shared-memory window are processed in
// windows and rounds; a target with more than kLC entries is read in several
// list passes.
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

constexpr int kTR = 64;         // targets per round of the pair passes
constexpr int kLC = 128;        // list entries per target and list pass
constexpr int kPipeWin = 832;   // staged candidates of a cell the pipelined passes take
constexpr int kPipeWinM = 448;  // ... the pipelined momentum pass takes (64/72-byte records)

// A cell is staged (hit masks) when its stencil holds at most kStagedMaxP
// particles, so a target's mask row is at most kStagedMaxP / 64 words and the
// mask buffer (kMaskWords per particle) cannot overflow; larger stencils (a
// few particles with a much larger h than the rest make every cell large) get
// int32 lists, marked by mask_base = kListForm.
constexpr int kStagedMaxP = 64 * kMaskWords;
// per-warp buffer of one round's hit words of a one-window stencil
constexpr int kMaskBufWords = kFindWindow / 64 * 32;
constexpr uint32_t kListForm = 0xffffffffu;
constexpr uint32_t kNoCell = 0xffffffffu;  // past the end of a launch's cell list

// Targets of a cell (bit 15 of a staged cell's field is its pipelined-pass flag).
__device__ __forceinline__ int cell_na(uint4 md) {
  return (int)(md.w & (md.y == kListForm ? 0xffffu : 0x7fffu));
}
__device__ __forceinline__ int cell_S(uint4 md) { return (int)(md.w >> 16); }

struct MaskOut {
  uint4* meta;                  // per occupied cell
  uint32_t* sent;               // staged candidate entries
  unsigned long long* masks;    // hit masks
  unsigned long long* alloc;    // [0] entries taken, [1] mask words taken
  unsigned long long sent_cap;  // capacities of sent and masks
  unsigned long long mask_cap;
  uint16_t* slist;              // staged-slot lists (rows of max_nb entries)
  uint32_t* fcells;             // cells of every pipelined pass (alloc[2] of them)
  uint32_t* scells;             // the other cells (alloc[3])
  uint32_t* mcells;             // cells of the pipelined density and IAD passes only (alloc[4])
};

// Row of particle a in the staged-slot lists: max_nb uint16 entries inside the
// particle's int32 list row (a particle's cell is either staged or in list
// form, so the row serves one of the two).  16-byte aligned: max_nb is a
// multiple of 4.
__device__ __forceinline__ uint16_t* slot_row(uint16_t* slist, int64_t a, int max_nb) {
  return slist + 2 * a * max_nb;
}

// Staged-slot list of one target from its hit-mask words (word blk at
// words[32 blk], bit 63 - q for slot 64 blk + q): one loop over words and
// bits, slot indices packed into a 128-bit register eight at a time and each
// full group stored with one 16-byte store, the rest (up to max_nb entries)
// one by one.  Returns the number of hits.
__device__ __forceinline__ int write_slot_list(const unsigned long long* words, int nblk,
                                               uint16_t* row, int max_nb) {
  uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0;  // entries k-8..k-1 of the group being filled
  int k = 0;
  int blk = 0;
  uint64_t w = nblk > 0 ? words[0] : 0;
  for (;;) {
    if (!w) {
      if (++blk >= nblk) break;
      w = words[32 * blk];
      continue;
    }
    const int q = __clzll((long long)w);
    w ^= kTop >> q;
    const uint32_t e = (uint32_t)(64 * blk + q);
    b0 = __funnelshift_r(b0, b1, 16);
    b1 = __funnelshift_r(b1, b2, 16);
    b2 = __funnelshift_r(b2, b3, 16);
    b3 = (b3 >> 16) | (e << 16);
    ++k;
    if ((k & 7) == 0) {
      if (k <= max_nb) {
        *reinterpret_cast<uint4*>(row + (k - 8)) = make_uint4(b0, b1, b2, b3);
      } else if (k - 8 < max_nb) {  // a group across max_nb (max_nb = 4 mod 8)
        const uint32_t bb[4] = {b0, b1, b2, b3};
        for (int i = 0; k - 8 + i < max_nb; ++i)
          row[k - 8 + i] = (uint16_t)(bb[i >> 1] >> (16 * (i & 1)));
      }
    }
  }
  // the last, partial group (entries (k & ~7) .. k - 1, at the top of b)
  const int r = k & 7;
  const uint32_t bb[4] = {b0, b1, b2, b3};
  for (int i = 0; i < r; ++i) {
    const int pos = (k & ~7) + i, src = 8 - r + i;
    if (pos < max_nb) row[pos] = (uint16_t)(bb[src >> 1] >> (16 * (src & 1)));
  }
  return k;
}

template <bool WRAP, int WIN>
__device__ __forceinline__ void find_cell_masks(const Grid& g, uint32_t cell, uint32_t code,
                                                const StateView& s,
                                                const float4* __restrict__ pos32,
                                                const uint32_t* tbl_start,
                                                const uint32_t* tbl_count, int32_t* nn,
                                                uint32_t* nbr, int max_nb, const MaskOut& mo,
                                                uint32_t* err,
                                                FindWarpSmemT<WIN>& W, unsigned long long& tested,
                                                unsigned long long& exact,
                                                unsigned long long& slots,
                                                unsigned long long& words,
                                                unsigned long long* mbuf) {
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
    if (lane == 0) {
      mo.meta[cell] = make_uint4(0u, kListForm, (uint32_t)a0, (uint32_t)na & 0xffffu);
      mo.scells[atomicAdd(mo.alloc + 3, 1ull)] = cell;
    }
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
  // A stencil that fits one window (most cells): each round's hit words stay
  // in the warp's mask buffer (word jb of lane t at mbuf[32 jb + t]) and the
  // round's lists are written from there, so its masks never reach memory.
  bool direct = false;
  int kmax = 0;        // largest hit count of the cell's targets (direct cells)
  int sc = 0, j0 = 0;  // next source: stencil cell and particle within it
  const uint32_t lt = (1u << lane) - 1u;
  for (;;) {
    // the targets' box and the reach, in registers for this staging pass
    const float blx = S.box_lo[0], bly = S.box_lo[1], blz = S.box_lo[2];
    const float bhx = S.box_hi[0], bhy = S.box_hi[1], bhz = S.box_hi[2];
    const float reach2 = S.reach2;
    while (sc < S.ncell && wn + 32 <= WIN) {
      // this stencil cell's values, read once for all its batches of 32
      const int cnt = S.off[sc + 1] - S.off[sc];
      const bool own = sc == S.self_cell;
      if (own && j0 == 0) gself = 64 * (int)gb + wn;
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
          const uint32_t e = ecode | (uint32_t)(st + j);
          W.entry[q] = e;
          mo.sent[slot_base + 64u * gb + (uint32_t)q] = e;
        }
        wn += __popc(bal);
        j0 += 32;
      } while (j0 < cnt && wn + 32 <= WIN);
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
    direct = first && done;
    for (int t0 = 0; t0 < na; t0 += 32) {
      // a round of r targets; with r <= 16, G = 32 / r lanes share each target
      // and take its blocks round-robin (lane l: target l % r, blocks
      // jb = l / r, l / r + G, ...)
      const int r = min(32, na - t0);
      const int G = 32 / r;
      const int tl = lane % r, grp = lane / r;
      const bool active = grp < G;
      const int t = t0 + tl;
      const int a = a0 + t;
      const float4 pa = pos32[a];
      const float two_h = 2.0f * pa.w;
      const float lim = two_h * two_h;
      const float margin = 2.0f * (2.0f * two_h * esum + esq + 4.76837158203125e-07f * lim);
      const float lo_lim = lim - margin, hi_lim = lim + margin;
      const float2 npx = make_float2(-pa.x, -pa.x), npy = make_float2(-pa.y, -pa.y),
                   npz = make_float2(-pa.z, -pa.z);
      const int gs = gself >= 0 ? gself + t : -1;  // own staged slot
      int kp = 0;                                  // this lane's hits
      for (int jb = active ? grp : nblk; jb < nblk; jb += G) {
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
        if (direct)
          mbuf[32 * jb + tl] = hit;
        else
          mo.masks[mask_base + (uint32_t)gblk * (uint32_t)na + (uint32_t)t] = hit;
        kp += __popcll(hit);
      }
      // the target's hits over its G lanes (lanes tl, tl + r, ...)
      int k = kp;
      for (int gg = 1; gg < G; ++gg) k += __shfl_sync(0xffffffffu, kp, min(tl + gg * r, 31));
      const bool lead = grp == 0;  // the lane that owns the target's results
      if (direct) __syncwarp();    // the round's hit words are in mbuf
      if (!first && lead) k += nn[a];
      if (lead && direct) {
        write_slot_list(mbuf + tl, nblk, slot_row(mo.slist, (int64_t)a, max_nb), max_nb);
        kmax = max(kmax, k);
      }
      if (lead) {
        nn[a] = k;
        if (k > max_nb) raise_flag(err, SPH_FLAG_NB_OVERFLOW);
        const bool self_here = gs >= 0 && gs >= 64 * (int)gb && gs < 64 * (int)gb + nproc;
        tested += (unsigned long long)nproc - (self_here ? 1 : 0);
      }
      if (direct) __syncwarp();    // mbuf is free for the next round
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
  const uint32_t staged = 64u * gb + (uint32_t)wn;
  if (lane == 0) {
    slots += staged;
    words += (unsigned long long)na * ((staged + 63) >> 6);
  }
  // The staged-slot lists: lane t walks the hit masks it wrote for target t
  // (still in L2) in one loop over words and bits, packing slot indices into
  // a 128-bit register eight at a time and storing each full group with one
  // 16-byte store; the rest, up to max_nb entries, one by one.
  // The round's mask words are first copied (coalesced) into the window,
  // which is free now: nblk <= kStagedMaxP / 64 = 32 words per target.
  const int nblk = direct ? 0 : (int)((staged + 63) >> 6);
  static_assert(kStagedMaxP / 64 * 32 * 8 <= 4 * WIN * 4, "mask copy fits the window");
  unsigned long long* mcopy = reinterpret_cast<unsigned long long*>(W.cx);
  int kl = 0;  // this lane's count
  for (int t0 = 0; !direct && t0 < na; t0 += 32, kmax = max(kmax, kl), kl = 0) {
    const int t = t0 + lane;
    __syncwarp();
#pragma unroll 4
    for (int blk = 0; blk < nblk; ++blk)
      mcopy[blk * 32 + lane] =
          t < na ? mo.masks[mask_base + (uint32_t)blk * (uint32_t)na + (uint32_t)t] : 0ull;
    __syncwarp();
    if (t >= na) continue;
    kl = write_slot_list(mcopy + lane, nblk, slot_row(mo.slist, (int64_t)a0 + t, max_nb), max_nb);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  // cells the pipelined passes take whole: one round of at most kTR targets,
  // lists of at most kLC entries and one window of staged candidates (448
  // for momentum, 832 for the others)
  const int cls =
      na > kTR || kmax > kLC || (int)staged > kPipeWin ? 1 : ((int)staged <= kPipeWinM ? 0 : 2);
  if (lane == 0) {
    mo.meta[cell] = make_uint4(slot_base, (uint32_t)gself, (uint32_t)a0,
                               (staged << 16) | (cls != 1 ? 0x8000u : 0u) | (uint32_t)na);
    const unsigned long long q = atomicAdd(mo.alloc + 2 + cls, 1ull);
    (cls == 0 ? mo.fcells : (cls == 1 ? mo.scells : mo.mcells))[q] = cell;
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
  unsigned long long* mbuf = reinterpret_cast<unsigned long long*>(
                                 smem_raw + kFindWarps * sizeof(FindWarpSmem)) +
                             warp * kMaskBufWords;
  const Grid g = *gp;
  if ((g.wrap32 != 0) != WRAP) return;
  unsigned long long tested = 0, exact = 0, slots = 0, words = 0;
  const uint32_t gw = blockIdx.x * kFindWarps + warp, nw = gridDim.x * kFindWarps;
  for (uint32_t cell = gw; cell < g.n_occ; cell += nw)
    find_cell_masks<WRAP, kFindWindow>(g, cell, occ[cell], s, pos32, tbl_start, tbl_count, nn,
                                       nbr, max_nb, mo, err, W, tested, exact, slots, words, mbuf);
  for (int o = 16; o > 0; o >>= 1) {
    tested += __shfl_xor_sync(0xffffffffu, tested, o);
    exact += __shfl_xor_sync(0xffffffffu, exact, o);
  }
  if (lane == 0) {
    atomicAdd(stats + 0, tested);
    atomicAdd(stats + 1, exact);
    atomicAdd(stats + 4, slots);   // lane 0 alone counted its cells' slots and words
    atomicAdd(stats + 5, words);
  }
}

// ------------------------------------------------------------- pair passes --

constexpr int kPT = 256;        // threads per CTA (general pair passes)
constexpr int kLS = kLC + 8;    // list row stride (uint16): 16-byte aligned rows, in different banks
constexpr int kMaxSub = 32;     // threads sharing one target, at most

__device__ __forceinline__ float wrap32(float d, const Grid& g, int ax) {
  if (d > g.halfL32[ax])
    d -= g.L32[ax];
  else if (d < -g.halfL32[ax])
    d += g.L32[ax];
  return d;
}

// Pair-pass configurations.  kCfgAny decides at run time (per pair) whether
// separations take the FP32 minimum image, which kernel form is used and
// whether the grad-h sum is formed; kCfgPlain fixes the default case at
// compile time: no minimum image (every periodic axis has at least 3 cells),
// the series kernel with n = 6 and no grad-h terms.  The plain configuration
// also keeps 64-byte momentum records (1/h, c and 1/rho stored; 1/h^2, B_n/h^3
// and P/rho^2 formed per read), so the two agree to FP32 rounding, not bit for
// bit.  A plain launch runs only when the grid needs no minimum image
// (Grid::wrap32 = 0), so the launcher starts both and each returns at once
// unless the grid is its case.
constexpr int kCfgAny = 0;
constexpr int kCfgPlain = 1;

// Separation b - a of two positions relative to the target's cell; the FP32
// minimum image is needed only on periodic axes with fewer than 3 cells.
template <int CFG>
__device__ __forceinline__ void sep(const Grid& g, float bx, float by, float bz, float ax_,
                                    float ay, float az, float& dx, float& dy, float& dz) {
  dx = bx - ax_;
  dy = by - ay;
  dz = bz - az;
  if (CFG == kCfgAny && g.wrap32) {
    if (g.periodic[0]) dx = wrap32(dx, g, 0);
    if (g.periodic[1]) dy = wrap32(dy, g, 1);
    if (g.periodic[2]) dz = wrap32(dz, g, 2);
  }
}

// S(t)^n (t = v^2; the exact kernel's polynomial, or the table), B_n / h^3
// factored out of the sums.
template <int CFG>
__device__ __forceinline__ float s_pow(float t, int n, const float2* tab) {
  if (CFG == kCfgPlain) return kernel_w32(t, 1.0f, 6);
  return tab ? kernel_w32_tab(t, 1.0f, tab) : kernel_w32(t, 1.0f, n);
}

// L1 prefetch of the line holding p.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Paired FP32: two pairs per instruction (f32x2 arithmetic of sm_100+), each
// component rounded exactly as the scalar operation.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// s_pow for two arguments: the polynomial and the powers in paired FP32.
template <int CFG>
__device__ __forceinline__ float2 s_pow2(float2 t, int n, const float2* tab) {
  if (CFG == kCfgAny && tab)
    return make_float2(kernel_w32_tab(t.x, 1.0f, tab), kernel_w32_tab(t.y, 1.0f, tab));
  t = make_float2(fminf(t.x, 4.0f), fminf(t.y, 4.0f));
  constexpr SincCoefs<kSincTerms32> C{};
  float2 s = f2((float)C.c[kSincTerms32 - 1]);
#pragma unroll
  for (int k = kSincTerms32 - 2; k >= 0; --k) s = __ffma2_rn(s, t, f2((float)C.c[k]));
  if (CFG == kCfgPlain || n == 6) {
    const float2 s2 = __fmul2_rn(s, s);
    return __fmul2_rn(__fmul2_rn(s2, s2), s2);
  }
  return make_float2(ipow(s.x, n), ipow(s.y, n));
}

// Separations b - a of two neighbours (paired), with the FP32 minimum image
// on periodic axes of fewer than 3 cells.
template <int CFG>
__device__ __forceinline__ void sep2(const Grid& g, float4 b0, float4 b1, float ax_, float ay,
                                     float az, float2& dx, float2& dy, float2& dz) {
  dx = __fadd2_rn(f2(b0.x, b1.x), f2(-ax_));
  dy = __fadd2_rn(f2(b0.y, b1.y), f2(-ay));
  dz = __fadd2_rn(f2(b0.z, b1.z), f2(-az));
  if (CFG == kCfgAny && g.wrap32) {
    if (g.periodic[0]) dx = make_float2(wrap32(dx.x, g, 0), wrap32(dx.y, g, 0));
    if (g.periodic[1]) dy = make_float2(wrap32(dy.x, g, 1), wrap32(dy.y, g, 1));
    if (g.periodic[2]) dz = make_float2(wrap32(dz.x, g, 2), wrap32(dz.y, g, 2));
  }
}

// Asynchronous global -> shared copies (cp.async, no register staging): the
// pipelined passes copy the next cell's records and lists while the current
// cell is computed.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// --- density + EOS (Eq. 1, self term included) ---
template <int CFG>
struct DensityPassT {
  static constexpr int kWin = 1024;   // staged slots held in shared memory
  static constexpr int kRecBytes = 16;
  static constexpr int kV = 2;        // reduced values: sum m S^n, grad-h sum
  static constexpr int kMinBlocks = 4;
  static constexpr bool kPaired = true;  // two pairs per iteration in paired FP32
  static constexpr int kPipeThreads = 256;
  static constexpr int kPipeMinBlocks = 3;
  static constexpr int kPipeW = kPipeWin;  // its window (staged slots per buffer)
  static constexpr bool kPipeAll = true;   // cells of up to kPipeWin candidates
  static constexpr bool kSmemLists = true; // lists copied with the records
  static constexpr bool kTargetSmem = false;
  static constexpr bool kPipePaired = true;
  const float4* rec_d;   // (offset, m) per particle
  const float4* pos32;   // (offset, h)
  const double* u;
  OutView o;
  float4* rec_i;         // out: (offset, m / rho)
  float4* recA;          // out: (offset, 1 / h^2); plain configuration (offset, 1 / h)
  float4* recQ;          // out: (B_n / h^3, X, c, 1 / rho); plain configuration (c, 1 / rho, -, -)
  const float2* ktab;
  float Bn;
  int sinc_n;
  double gamma;
  int gradh;
  uint32_t* err;
  __device__ bool has_gradh() const { return CFG == kCfgAny && gradh; }
  // kCfgAny launched beside a kCfgPlain launch: runs only on grids that need
  // the minimum image
  int only_wrap;
  __device__ bool runs(const Grid& g) const {
    return CFG == kCfgPlain ? !g.wrap32 : (!only_wrap || g.wrap32);
  }

  struct Target {
    float x, y, z, hinv2;
  };
  struct Rec {
    float4 r;  // position relative to the target's cell, m
  };
  __device__ Rec load(uint32_t e, const float4* shtab) const {
    const float4 sh = shtab[e >> kIndexBits];
    const float4 r = rec_d[entry_index(e)];
    return {make_float4(r.x + sh.x, r.y + sh.y, r.z + sh.z, r.w)};
  }
  template <int W>
  static __device__ Rec fetch(const float4* rec, int j) { return {rec[j]}; }
  template <int W>
  static __device__ void target_from(float4*, int, Target&) {}
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
    sep<CFG>(g, r.x, r.y, r.z, T.x, T.y, T.z, dx, dy, dz);
    const float tt = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) * T.hinv2;
    acc[0] = fmaf(r.w, s_pow<CFG>(tt, sinc_n, ktab), acc[0]);
    if (has_gradh()) acc[1] = fmaf(r.w, kernel_tdw32(tt, 1.0f, sinc_n), acc[1]);
  }
  __device__ void pair2(const Target& T, const Rec& R0, const Rec& R1, const Grid& g,
                        float2* acc) const {
    float2 dx, dy, dz;
    sep2<CFG>(g, R0.r, R1.r, T.x, T.y, T.z, dx, dy, dz);
    const float2 tt =
        __fmul2_rn(__ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx))), f2(T.hinv2));
    const float2 m = f2(R0.r.w, R1.r.w);
    acc[0] = __ffma2_rn(m, s_pow2<CFG>(tt, sinc_n, ktab), acc[0]);
    if (has_gradh())
      acc[1] = __ffma2_rn(m, make_float2(kernel_tdw32(tt.x, 1.0f, sinc_n),
                                         kernel_tdw32(tt.y, 1.0f, sinc_n)), acc[1]);
  }
  template <int W>
  __device__ void copy_async(float4* rec, int j, int b) const { cp_async16(rec + j, rec_d + b); }
  struct FinishIn {
    float4 p;
    float m;
    double u;
  };
  __device__ FinishIn prefin(int64_t a) const { return {pos32[a], rec_d[a].w, u[a]}; }
  // L1 prefetch of prefin's lines, one iteration before prefin reads them
  __device__ void prefetch_fin(int64_t a) const {
    prefetch_l1(pos32 + a);
    prefetch_l1(rec_d + a);
    prefetch_l1(u + a);
  }
  __device__ void finish(int64_t a, const float* acc) const { finish2(a, acc, prefin(a)); }
  __device__ void finish2(int64_t a, const float* acc, const FinishIn& fin) const {
    const float4 p = fin.p;
    // the plain configuration keeps 1/h in the records and forms 1/h^2 and
    // B_n / h^3 from it as the momentum pass does
    const float hinv = CFG == kCfgPlain ? 1.0f / p.w : 0.0f;
    const float hinv2 = CFG == kCfgPlain ? hinv * hinv : 1.0f / (p.w * p.w);
    const float norm = CFG == kCfgPlain ? Bn * hinv * hinv2 : Bn * hinv2 / p.w;
    const float ma = fin.m;
    const float rho = norm * (ma + acc[0]);  // self term: S(0)^n = 1
    // the ideal-gas equation of state in FP32 (from the FP32 density; FP64
    // division and square root run at 1/64 of the FP32 rate on this part):
    // P = (gamma - 1) rho u, c = sqrt(gamma P / rho) = sqrt(gamma (gamma - 1) u),
    // X = P / rho^2 = (gamma - 1) u / rho
    const float uf = (float)fin.u, g1 = (float)(gamma - 1.0);
    const float pr = g1 * rho * uf;
    const float c = sqrtf((float)gamma * g1 * uf);
    const float inv_rho = 1.0f / rho;
    float X = g1 * uf * inv_rho;
    o.rho[a] = (double)rho;
    o.p[a] = (double)pr;
    o.c[a] = (double)c;
    rec_i[a] = make_float4(p.x, p.y, p.z, ma * inv_rho);
    recA[a] = make_float4(p.x, p.y, p.z, CFG == kCfgPlain ? hinv : hinv2);
    if (has_gradh()) {
      const float omega = -2.0f * norm * acc[1] * inv_rho * (1.0f / 3.0f);
      X /= omega;
      if (o.omega) o.omega[a] = (double)omega;
    }
    // (plain: X = P / rho^2 = c^2 / (gamma rho) is formed by the momentum pass;
    // the IAD pass writes C12 and C22 into the last two components)
    recQ[a] = CFG == kCfgPlain ? make_float4(c, inv_rho, 0.0f, 0.0f)
                               : make_float4(norm, X, c, inv_rho);
    if (!isfinite(rho) || !isfinite(c)) raise_flag(err, SPH_FLAG_NONFINITE);
  }
};

// --- IAD: tau_a and C_a = tau_a^{-1} ---
template <int CFG>
struct IadPassT {
  static constexpr int kWin = 1024;
  static constexpr int kRecBytes = 16;
  static constexpr int kV = 6;
  static constexpr int kMinBlocks = 3;  // general kernel (the few cells outside the pipelined
                                        // lists): no register spills at this bound
  static constexpr bool kPaired = true;
  static constexpr int kPipeThreads = 256;
  static constexpr int kPipeMinBlocks = 3;
  static constexpr int kPipeW = kPipeWin;
  static constexpr bool kPipeAll = true;
  static constexpr bool kSmemLists = true;
  static constexpr bool kTargetSmem = false;
  static constexpr bool kPipePaired = true;
  const float4* rec_i;   // (offset, m / rho)
  const float4* recA;    // (offset, 1 / h^2); plain configuration (offset, 1 / h)
  float4* recQ;          // (B_n / h^3, ...); plain configuration: out (-, -, C12, C22)
  OutView o;
  float4* recC;          // out: (C00, C01, C02, C11)
  float2* recC2;         // out: (C12, C22) (general configuration)
  const float2* ktab;
  float Bn;
  int sinc_n;
  uint32_t* err;
  // kCfgAny launched beside a kCfgPlain launch: runs only on grids that need
  // the minimum image
  int only_wrap;
  __device__ bool runs(const Grid& g) const {
    return CFG == kCfgPlain ? !g.wrap32 : (!only_wrap || g.wrap32);
  }

  struct Target {
    float x, y, z, hinv2;
  };
  struct Rec {
    float4 r;  // position relative to the target's cell, m / rho
  };
  __device__ Rec load(uint32_t e, const float4* shtab) const {
    const float4 sh = shtab[e >> kIndexBits];
    const float4 r = rec_i[entry_index(e)];
    return {make_float4(r.x + sh.x, r.y + sh.y, r.z + sh.z, r.w)};
  }
  template <int W>
  static __device__ Rec fetch(const float4* rec, int j) { return {rec[j]}; }
  template <int W>
  static __device__ void target_from(float4*, int, Target&) {}
  __device__ void load_target(int64_t a, Target& T) const {
    const float4 p = recA[a];
    T.x = p.x;
    T.y = p.y;
    T.z = p.z;
    T.hinv2 = CFG == kCfgPlain ? p.w * p.w : p.w;
  }
  __device__ void pair(const Target& T, const Rec& R, const Grid& g, float* acc) const {
    const float4 r = R.r;
    float dx, dy, dz;
    sep<CFG>(g, r.x, r.y, r.z, T.x, T.y, T.z, dx, dy, dz);
    const float tt = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) * T.hinv2;
    // the weight divided by h_a^2 (tau / h_a^2 is of order one in FP32)
    const float w = r.w * s_pow<CFG>(tt, sinc_n, ktab) * T.hinv2;
    const float wx = w * dx, wy = w * dy, wz = w * dz;
    acc[0] = fmaf(wx, dx, acc[0]);
    acc[1] = fmaf(wx, dy, acc[1]);
    acc[2] = fmaf(wx, dz, acc[2]);
    acc[3] = fmaf(wy, dy, acc[3]);
    acc[4] = fmaf(wy, dz, acc[4]);
    acc[5] = fmaf(wz, dz, acc[5]);
  }
  __device__ void pair2(const Target& T, const Rec& R0, const Rec& R1, const Grid& g,
                        float2* acc) const {
    float2 dx, dy, dz;
    sep2<CFG>(g, R0.r, R1.r, T.x, T.y, T.z, dx, dy, dz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const float2 tt = __fmul2_rn(r2, f2(T.hinv2));
    const float2 w = __fmul2_rn(__fmul2_rn(f2(R0.r.w, R1.r.w), s_pow2<CFG>(tt, sinc_n, ktab)),
                                f2(T.hinv2));
    const float2 wx = __fmul2_rn(w, dx), wy = __fmul2_rn(w, dy), wz = __fmul2_rn(w, dz);
    acc[0] = __ffma2_rn(wx, dx, acc[0]);
    acc[1] = __ffma2_rn(wx, dy, acc[1]);
    acc[2] = __ffma2_rn(wx, dz, acc[2]);
    acc[3] = __ffma2_rn(wy, dy, acc[3]);
    acc[4] = __ffma2_rn(wy, dz, acc[4]);
    acc[5] = __ffma2_rn(wz, dz, acc[5]);
  }
  template <int W>
  __device__ void copy_async(float4* rec, int j, int b) const { cp_async16(rec + j, rec_i + b); }
  struct FinishIn {
    float hinv2, norm;
  };
  __device__ void prefetch_fin(int64_t a) const {
    prefetch_l1(recA + a);
    if (CFG != kCfgPlain) prefetch_l1(recQ + a);
  }
  __device__ FinishIn prefin(int64_t a) const {
    if (CFG == kCfgPlain) {
      const float hinv = recA[a].w, hinv2 = hinv * hinv;
      return {hinv2, Bn * hinv * hinv2};
    }
    return {recA[a].w, recQ[a].x};
  }
  __device__ void finish(int64_t a, const float* acc) const { finish2(a, acc, prefin(a)); }
  __device__ void finish2(int64_t a, const float* acc, const FinishIn& fin) const {
    const float hinv2 = fin.hinv2;
    const float norm = fin.norm;
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
    if (CFG == kCfgPlain)
      reinterpret_cast<float2*>(recQ + a)[1] = make_float2(Cm[4], Cm[5]);
    else
      recC2[a] = make_float2(Cm[4], Cm[5]);
    double* out = o.iad + 6 * a;
    for (int q = 0; q < 6; ++q) out[q] = (double)Cm[q];
  }
};

// --- momentum and energy with artificial viscosity (Eqs. 2-5) ---
template <int CFG>
struct MomentumPassT {
  static constexpr int kWin = 768;  // staged slots (plane stride): three CTAs of <= 73 KB per SM
  // four float4 planes and one float2 plane; the plain configuration keeps
  // four float4 planes (1/h, c and 1/rho stored; 1/h^2, B_n / h^3 and X
  // formed per record read): 8 bytes fewer per pair from shared memory
  static constexpr int kRecBytes = CFG == kCfgPlain ? 64 : 72;
  static constexpr int kV = 4;
  static constexpr int kMinBlocks = 3;
  static constexpr bool kPaired = false;  // the paired body needs ~120 registers: scalar pairs
                                          // keep three CTAs per SM
  // pipelined kernel: cells of up to kPipeWinM candidates, a double buffer of
  // 2 x 32 KB, three CTAs per SM
  static constexpr int kPipeThreads = 256;
  static constexpr int kPipeMinBlocks = 3;
  static constexpr int kPipeW = kPipeWinM;
  static constexpr bool kPipeAll = false;    // the cells of 449..832 candidates: general kernel
  static constexpr bool kSmemLists = false;  // lists read through L1
  static constexpr bool kTargetSmem = true;  // target records from the staged window
  static constexpr bool kPipePaired = false;
  const float4* recA;    // (offset, 1 / h^2); plain configuration (offset, 1 / h)
  const float4* recV;    // (v, m)
  const float4* recQ;    // (B_n / h^3, X = P / (Omega rho^2), c, 1 / rho);
                         // plain configuration (c, 1 / rho, C12, C22)
  const float4* recC;    // (C00, C01, C02, C11)
  const float2* recC2;   // (C12, C22) (general configuration)
  OutView o;
  const float2* ktab;
  int sinc_n;
  float alpha;
  float Bn;              // kernel normalisation (plain configuration: B_n / h^3 from 1/h)
  float inv_gamma;       // 1 / gamma (plain configuration: X = c^2 / (gamma rho))
  uint32_t* err;
  // kCfgAny launched beside a kCfgPlain launch: runs only on grids that need
  // the minimum image
  int only_wrap;
  __device__ bool runs(const Grid& g) const {
    return CFG == kCfgPlain ? !g.wrap32 : (!only_wrap || g.wrap32);
  }

  struct Target {
    float4 p, v, q;
    float c00, c01, c02, c11, c12, c22;
  };
  // shared-memory planes of a window of W slots: A, V, Q, C (float4) then C2 (float2)
  template <int W>
  static __device__ __forceinline__ float4* plane(float4* rec, int k) { return rec + k * W; }
  template <int W>
  static __device__ __forceinline__ float2* plane2(float4* rec) {
    return reinterpret_cast<float2*>(rec + 4 * W);
  }
  struct Rec {
    float4 p, v, q, c;  // (position relative to the target's cell, 1/h^2), (v, m), Q, C
    float2 c2;
  };
  // a plain-configuration record (A: offset, 1/h; V; Q: c, 1/rho, C12, C22; C)
  // in the general form (A: offset, 1/h^2; Q: B_n / h^3, X, c, 1/rho; C2), with
  // X = P / rho^2 = c^2 / (gamma rho) for the ideal gas
  __device__ __forceinline__ Rec widen(float4 p, float4 v, float4 q, float4 c) const {
    const float hinv2 = p.w * p.w;
    const float norm = Bn * p.w * hinv2;
    const float X = q.x * q.x * (q.y * inv_gamma);
    return {make_float4(p.x, p.y, p.z, hinv2), v, make_float4(norm, X, q.x, q.y), c,
            make_float2(q.z, q.w)};
  }
  __device__ Rec load(uint32_t e, const float4* shtab) const {
    const float4 sh = shtab[e >> kIndexBits];
    const int b = entry_index(e);
    const float4 p = recA[b];
    const float4 ps = make_float4(p.x + sh.x, p.y + sh.y, p.z + sh.z, p.w);
    if (CFG == kCfgPlain) return widen(ps, recV[b], recQ[b], recC[b]);
    return {ps, recV[b], recQ[b], recC[b], recC2[b]};
  }
  template <int W>
  __device__ Rec fetch(float4* rec, int j) const {
    if (CFG == kCfgPlain)
      return widen(plane<W>(rec, 0)[j], plane<W>(rec, 1)[j], plane<W>(rec, 2)[j],
                   plane<W>(rec, 3)[j]);
    return {plane<W>(rec, 0)[j], plane<W>(rec, 1)[j], plane<W>(rec, 2)[j], plane<W>(rec, 3)[j],
            plane2<W>(rec)[j]};
  }
  static __device__ void to_target(const Rec& R, Target& T) {
    T.p = R.p;
    T.v = R.v;
    T.q = R.q;
    T.c00 = R.c.x;
    T.c01 = R.c.y;
    T.c02 = R.c.z;
    T.c11 = R.c.w;
    T.c12 = R.c2.x;
    T.c22 = R.c2.y;
  }
  __device__ void load_target(int64_t a, Target& T) const {
    if (CFG == kCfgPlain)
      to_target(widen(recA[a], recV[a], recQ[a], recC[a]), T);
    else
      to_target({recA[a], recV[a], recQ[a], recC[a], recC2[a]}, T);
  }
  __device__ void pair(const Target& T, const Rec& R, const Grid& g, float* acc) const {
    // one pair of Eqs. 2-5 (x_ab = -d, d = x_b - x_a)
    const float4 b0 = R.p;
    float dx, dy, dz;
    sep<CFG>(g, b0.x, b0.y, b0.z, T.p.x, T.p.y, T.p.z, dx, dy, dz);
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float4 b2 = R.q;
    // W_a and W_b together in paired FP32 (each component rounded as the
    // scalar operation), clamped at t = 4 (S = 0)
    const float2 Wab = __fmul2_rn(f2(T.q.x, b2.x),
                                  s_pow2<CFG>(__fmul2_rn(f2(r2), f2(T.p.w, b0.w)), sinc_n, ktab));
    const float Wa = Wab.x, Wb = Wab.y;
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
    // Eq. 5 without a branch: w_ab = x_ab.v_ab / r, Pi = 0 unless approaching;
    // hP = Pi / 2 and qP = Pi / 4 (exact: scalings by powers of two)
    const float w = xv * rsqrtf(r2);
    const float vsig = T.q.z + b2.z - 3.0f * w;
    const float hP = xv < 0.0f ? -0.25f * alpha * vsig * w : 0.0f;
    const float qP = 0.5f * hP;
    const float ira = T.q.w, irb = b2.w;
    const float mb = vb.w;
    const float fa = mb * Wa * fmaf(hP, ira, T.q.y);
    const float fb = mb * Wb * fmaf(hP, irb, b2.y);
    // a -= fa C_a d + fb C_b d as two fused steps
    acc[0] = fmaf(-fb, Cbdx, fmaf(-fa, Cadx, acc[0]));
    acc[1] = fmaf(-fb, Cbdy, fmaf(-fa, Cady, acc[1]));
    acc[2] = fmaf(-fb, Cbdz, fmaf(-fa, Cadz, acc[2]));
    const float vCa = fmaf(vabz, Cadz, fmaf(vaby, Cady, vabx * Cadx));
    const float vCb = fmaf(vabz, Cbdz, fmaf(vaby, Cbdy, vabx * Cbdx));
    acc[3] = fmaf(mb, fmaf(Wa * fmaf(qP, ira, T.q.y), vCa, qP * irb * Wb * vCb), acc[3]);
  }
  __device__ void pair2(const Target& T, const Rec& R0, const Rec& R1, const Grid& g,
                        float2* acc) const {
    // two pairs of Eqs. 2-5, the operations of pair() in paired FP32
    float2 dx, dy, dz;
    sep2<CFG>(g, R0.p, R1.p, T.p.x, T.p.y, T.p.z, dx, dy, dz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    const float2 Wa =
        __fmul2_rn(f2(T.q.x), s_pow2<CFG>(__fmul2_rn(r2, f2(T.p.w)), sinc_n, ktab));
    const float2 Wb = __fmul2_rn(f2(R0.q.x, R1.q.x),
                                 s_pow2<CFG>(__fmul2_rn(r2, f2(R0.p.w, R1.p.w)), sinc_n, ktab));
    const float2 Cadx = __ffma2_rn(f2(T.c02), dz, __ffma2_rn(f2(T.c01), dy, __fmul2_rn(f2(T.c00), dx)));
    const float2 Cady = __ffma2_rn(f2(T.c12), dz, __ffma2_rn(f2(T.c11), dy, __fmul2_rn(f2(T.c01), dx)));
    const float2 Cadz = __ffma2_rn(f2(T.c22), dz, __ffma2_rn(f2(T.c12), dy, __fmul2_rn(f2(T.c02), dx)));
    const float2 b00 = f2(R0.c.x, R1.c.x), b01 = f2(R0.c.y, R1.c.y), b02 = f2(R0.c.z, R1.c.z);
    const float2 b11 = f2(R0.c.w, R1.c.w), b12 = f2(R0.c2.x, R1.c2.x), b22 = f2(R0.c2.y, R1.c2.y);
    const float2 Cbdx = __ffma2_rn(b02, dz, __ffma2_rn(b01, dy, __fmul2_rn(b00, dx)));
    const float2 Cbdy = __ffma2_rn(b12, dz, __ffma2_rn(b11, dy, __fmul2_rn(b01, dx)));
    const float2 Cbdz = __ffma2_rn(b22, dz, __ffma2_rn(b12, dy, __fmul2_rn(b02, dx)));
    const float2 vabx = __fadd2_rn(f2(T.v.x), f2(-R0.v.x, -R1.v.x));
    const float2 vaby = __fadd2_rn(f2(T.v.y), f2(-R0.v.y, -R1.v.y));
    const float2 vabz = __fadd2_rn(f2(T.v.z), f2(-R0.v.z, -R1.v.z));
    const float2 xvn = __ffma2_rn(dz, vabz, __ffma2_rn(dy, vaby, __fmul2_rn(dx, vabx)));
    const float2 xv = make_float2(-xvn.x, -xvn.y);
    // Eq. 5 without a branch: w_ab = x_ab.v_ab / r, Pi = 0 unless approaching
    const float2 w = __fmul2_rn(xv, make_float2(rsqrtf(r2.x), rsqrtf(r2.y)));
    const float2 vsig = __fadd2_rn(__fadd2_rn(f2(T.q.z), f2(R0.q.z, R1.q.z)),
                                   __fmul2_rn(f2(-3.0f), w));
    const float2 pv = __fmul2_rn(__fmul2_rn(f2(-0.5f * alpha), vsig), w);
    const float2 Pi = make_float2(xv.x < 0.0f ? pv.x : 0.0f, xv.y < 0.0f ? pv.y : 0.0f);
    const float2 irb = f2(R0.q.w, R1.q.w);
    const float2 mb = f2(R0.v.w, R1.v.w);
    const float2 hP = __fmul2_rn(f2(0.5f), Pi), qP = __fmul2_rn(f2(0.25f), Pi);
    const float2 fa = __fmul2_rn(__fmul2_rn(mb, Wa), __ffma2_rn(hP, f2(T.q.w), f2(T.q.y)));
    const float2 fb = __fmul2_rn(__fmul2_rn(mb, Wb), __ffma2_rn(hP, irb, f2(R0.q.y, R1.q.y)));
    acc[0] = __ffma2_rn(f2(-1.0f), __ffma2_rn(fa, Cadx, __fmul2_rn(fb, Cbdx)), acc[0]);
    acc[1] = __ffma2_rn(f2(-1.0f), __ffma2_rn(fa, Cady, __fmul2_rn(fb, Cbdy)), acc[1]);
    acc[2] = __ffma2_rn(f2(-1.0f), __ffma2_rn(fa, Cadz, __fmul2_rn(fb, Cbdz)), acc[2]);
    const float2 vCa = __ffma2_rn(vabz, Cadz, __ffma2_rn(vaby, Cady, __fmul2_rn(vabx, Cadx)));
    const float2 vCb = __ffma2_rn(vabz, Cbdz, __ffma2_rn(vaby, Cbdy, __fmul2_rn(vabx, Cbdx)));
    const float2 i1 = __fmul2_rn(Wa, __ffma2_rn(qP, f2(T.q.w), f2(T.q.y)));
    const float2 i2 = __fmul2_rn(__fmul2_rn(__fmul2_rn(qP, irb), Wb), vCb);
    acc[3] = __ffma2_rn(mb, __ffma2_rn(i1, vCa, i2), acc[3]);
  }
  template <int W>
  __device__ void copy_async(float4* rec, int j, int b) const {
    cp_async16(plane<W>(rec, 0) + j, recA + b);
    cp_async16(plane<W>(rec, 1) + j, recV + b);
    cp_async16(plane<W>(rec, 2) + j, recQ + b);
    cp_async16(plane<W>(rec, 3) + j, recC + b);
    if (CFG != kCfgPlain) cp_async8(plane2<W>(rec) + j, recC2 + b);
  }
  // The target's data is its own staged record (its cell's shift is zero).
  template <int W>
  __device__ void target_from(float4* rec, int j, Target& T) const {
    to_target(fetch<W>(rec, j), T);
  }
  struct FinishIn {};
  __device__ FinishIn prefin(int64_t) const { return {}; }
  __device__ void prefetch_fin(int64_t) const {}
  __device__ void finish2(int64_t a, const float* acc, const FinishIn&) const { finish(a, acc); }
  __device__ void finish(int64_t a, const float* acc) const {
    o.ax[a] = acc[0];
    o.ay[a] = acc[1];
    o.az[a] = acc[2];
    o.du[a] = acc[3];
    if (!isfinite(acc[0]) || !isfinite(acc[1]) || !isfinite(acc[2]) || !isfinite(acc[3]))
      raise_flag(err, SPH_FLAG_NONFINITE);
  }
};

// Per-launch tables in shared memory: the FP32 shift of each of the 27
// stencil codes (entry_shift), nsub = min(PT / na, kMaxSub) for na <= 256 and
// 1/nsub in 16-bit fixed point, so that tid / nsub = (tid inv16) >> 16 (exact
// for tid < 256 and nsub <= 32: the error of the fixed-point reciprocal times
// tid stays below 1/nsub).
struct Tabs {
  static constexpr size_t kBytes = 27 * sizeof(float4) + 48 * sizeof(int) + 272;
  float4* shift;
  int* inv16;
  unsigned char* nsub;
  __device__ Tabs(unsigned char* base)
      : shift(reinterpret_cast<float4*>(base)),
        inv16(reinterpret_cast<int*>(base + 27 * sizeof(float4))),
        nsub(base + 27 * sizeof(float4) + 48 * sizeof(int)) {}
  // filled by the whole CTA; followed by a barrier
  template <int PT>
  __device__ void fill(const Grid& g) {
    const int tid = threadIdx.x;
    if (tid < 27) {
      float sx, sy, sz;
      entry_shift((uint32_t)tid << kIndexBits, g, sx, sy, sz);
      shift[tid] = make_float4(sx, sy, sz, 0.0f);
    }
    if (tid >= 1 && tid <= kMaxSub) inv16[tid] = (65536 + tid - 1) / tid;
    for (int na = tid; na <= PT; na += PT)
      nsub[na] = (unsigned char)(na > 0 ? min(PT / na, kMaxSub) : 1);
    __syncthreads();
  }
  __device__ int div(int tid, int ns) const { return (tid * inv16[ns]) >> 16; }
};

// Shared memory of a pass: the records of a window, the expanded lists (also
// the reduction's partial sums), per-(target, block) hit counts and the
// targets' totals, and the tables.
template <class Pass>
struct PassSmem {
  static constexpr size_t kRec = (size_t)Pass::kWin * Pass::kRecBytes;
  static constexpr size_t kLists = (size_t)kTR * kLS * sizeof(uint16_t);
  static constexpr size_t kPart = (size_t)kPT * Pass::kV * sizeof(float);
  static constexpr size_t kListsOrPart = kLists > kPart ? kLists : kPart;
  static constexpr size_t oTot = kRec + ((kListsOrPart + 15) & ~(size_t)15);
  static constexpr size_t oTab = oTot + (size_t)kTR * sizeof(int);
  static constexpr size_t kBytes = oTab + Tabs::kBytes;
  static_assert(kRec % 16 == 0 && oTab % 16 == 0, "16-byte aligned parts");
};

// Neighbour source of one pass launch.
struct Src {
  const uint4* meta;                 // per occupied cell
  const uint32_t* cells;             // the cells of this launch
  const unsigned long long* ncells;  // their number (device counter)
  const uint32_t* sent;              // staged candidate entries
  const int32_t* nn;                 // exact neighbour counts
  const uint32_t* nbr;               // list-form cells: int32 lists
  const uint16_t* slist;             // staged cells: staged-slot lists (same rows as nbr)
  int max_nb;
};

// Values of the next cell loaded while the current one is computed: the
// neighbour counts of its first targets and the staged entries of its first
// window (slots tid + i kPT, i < J).
template <int J>
struct Prefetch {
  int nn;          // thread tid < kTR: count of target tid of the first round
  uint32_t e[J];
};

// staged slots per thread in a window of the general kernel
template <class Pass>
constexpr int window_slots() {
  return (Pass::kWin + kPT - 1) / kPT;
}

template <class Pass>
__device__ __forceinline__ void prefetch_cell(const Src& src, uint4 md,
                                              Prefetch<window_slots<Pass>()>& pf) {
  const int tid = threadIdx.x;
  const int S = cell_S(md), na = cell_na(md);
  const bool staged = md.y != kListForm;
  pf.nn = (staged && tid < kTR && tid < na) ? __ldg(src.nn + md.z + tid) : 0;
  const int wn = min(Pass::kWin, S);
#pragma unroll
  for (int i = 0; i < window_slots<Pass>(); ++i) {
    const int j = tid + i * kPT;
    pf.e[i] = (staged && j < wn) ? __ldg(src.sent + md.x + (uint32_t)j) : 0u;
  }
}

template <class Pass>
__global__ void __launch_bounds__(kPT, Pass::kMinBlocks) k_cellpass(Pass pass, const Grid* gp,
                                                                    Src src) {
  using SM = PassSmem<Pass>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* rec = reinterpret_cast<float4*>(smem_raw);
  uint16_t* lists = reinterpret_cast<uint16_t*>(smem_raw + SM::kRec);
  float* part = reinterpret_cast<float*>(smem_raw + SM::kRec);
  int* tot = reinterpret_cast<int*>(smem_raw + SM::oTot);
  const Grid g = *gp;
  if (!pass.runs(g)) return;
  Tabs tb(smem_raw + SM::oTab);
  tb.fill<kPT>(g);
  const uint32_t n_cells = (uint32_t)*src.ncells;
  const uint32_t G = gridDim.x;
  const int tid = threadIdx.x;
  const uint4 zero4 = make_uint4(0u, kListForm, 0u, 0u);
  auto meta_of = [&](uint32_t q) { return q < n_cells ? __ldg(src.meta + src.cells[q]) : zero4; };
  auto cell_at = [&](uint32_t q) { return q < n_cells ? __ldg(src.cells + q) : kNoCell; };
  auto meta_at = [&](uint32_t c) { return c != kNoCell ? __ldg(src.meta + c) : zero4; };
  uint4 md_next = meta_of(blockIdx.x);
  uint4 md_after = meta_of(blockIdx.x + G);
  uint32_t c_ahead = cell_at(blockIdx.x + 2 * G);  // meta loaded one cell later
  constexpr int NJ = window_slots<Pass>();
  Prefetch<NJ> pf;
  prefetch_cell<Pass>(src, md_next, pf);
  for (uint32_t q = blockIdx.x; q < n_cells; q += G) {
    const uint4 md = md_next;
    const Prefetch<NJ> cur = pf;
    md_next = md_after;
    md_after = meta_at(c_ahead);
    c_ahead = cell_at(q + 3 * G);
    prefetch_cell<Pass>(src, md_next, pf);  // lands while this cell is computed
    const uint32_t slot_base = md.x, a0 = md.z;
    const int S = cell_S(md), na = cell_na(md);
    const bool list_form = md.y == kListForm;
    int staged_w0 = -1;
    for (int r0 = 0; r0 < na; r0 += kTR) {
      const int nr = min(kTR, na - r0);
      const int nsub = tb.nsub[nr];
      const int t = tb.div(tid, nsub), sub = tid - t * nsub;
      const bool active = t < nr;
      const int64_t a = (int64_t)a0 + r0 + (active ? t : 0);
      typename Pass::Target T;
      float acc[Pass::kV];
      float2 acc2[Pass::kV];  // paired partial sums, folded into acc at the end
#pragma unroll
      for (int v = 0; v < Pass::kV; ++v) {
        acc[v] = 0.0f;
        acc2[v] = make_float2(0.0f, 0.0f);
      }
      if (active) pass.load_target(a, T);
      if (list_form) {
        // a cell whose stencil exceeds the staged form's limits: int32 lists,
        // neighbour records read from global memory
        const int c = active ? min(__ldg(src.nn + a), src.max_nb) : 0;
        const uint32_t* row = src.nbr + a * src.max_nb;
        for (int k = sub; k < c; k += nsub)
          pass.pair(T, pass.load(__ldg(row + k), tb.shift), g, acc);
      } else {
        // the targets' staged-slot lists (ascending slots), kLC entries per
        // target at a time in shared memory, walked window by window
        if (tid < nr)
          tot[tid] = min(r0 == 0 ? cur.nn : __ldg(src.nn + a0 + r0 + tid), src.max_nb);
        for (int lp = 0;; ++lp) {
          __syncthreads();  // tot written; the previous readers are done
          for (int i = tid; i < nr * (kLC / 4); i += kPT) {
            const int tt = i / (kLC / 4), k4 = 4 * (i - tt * (kLC / 4));
            const int kk = lp * kLC + k4;
            if (kk < tot[tt])  // 8-byte chunks: max_nb and kLC are multiples of 4
              cp_async8(lists + tt * kLS + k4,
                        slot_row(const_cast<uint16_t*>(src.slist), (int64_t)a0 + r0 + tt,
                                 src.max_nb) + kk);
          }
          cp_async_commit();
          const int nl = active ? min(tot[t] - lp * kLC, kLC) : 0;
          int k = sub;
          for (int w0 = 0; w0 < S; w0 += Pass::kWin) {
            const int wn = min(Pass::kWin, S - w0);
            if (w0 != staged_w0) {
              if (w0 > 0) __syncthreads();  // the previous window's readers are done
              const uint32_t* es = src.sent + slot_base + (uint32_t)w0;
              const bool pre = w0 == 0 && r0 == 0 && lp == 0;  // entries already loaded
              // the window's records by cp.async (no register staging, one round
              // trip), then the cell shifts added to the records this thread copied
              uint32_t e[NJ];
#pragma unroll
              for (int i = 0; i < NJ; ++i) {
                const int j = i * kPT + tid;
                e[i] = pre ? cur.e[i] : (j < wn ? __ldg(es + j) : 0u);
              }
              // the entries' shift codes (5 bits each) kept packed across the wait
              static_assert(NJ <= 6, "shift codes packed into one register");
              uint32_t codes = 0;
#pragma unroll
              for (int i = 0; i < NJ; ++i) {
                const int j = i * kPT + tid;
                if (j < wn) pass.template copy_async<Pass::kWin>(rec, j, entry_index(e[i]));
                codes |= (e[i] >> kIndexBits) << (5 * i);
              }
              cp_async_commit();
              cp_async_wait_all();
#pragma unroll
              for (int i = 0; i < NJ; ++i) {
                const int j = i * kPT + tid;
                if (j < wn) {
                  const float4 sh = tb.shift[(codes >> (5 * i)) & 31u];
                  float4 r = rec[j];
                  r.x += sh.x;
                  r.y += sh.y;
                  r.z += sh.z;
                  rec[j] = r;
                }
              }
              staged_w0 = w0;
            }
            cp_async_wait_all();  // the list chunks have landed
            __syncthreads();      // lists copied, records staged
            const uint16_t* row = lists + t * kLS;
            const int wend = w0 + wn;
            for (; Pass::kPaired && k + nsub < nl; k += 2 * nsub) {  // two entries at a time
              const int s0 = row[k], s1 = row[k + nsub];
              if (s1 >= wend) break;                 // ascending: s0 < s1
              pass.pair2(T, pass.template fetch<Pass::kWin>(rec, s0 - w0),
                         pass.template fetch<Pass::kWin>(rec, s1 - w0), g, acc2);
            }
            for (; k < nl; k += nsub) {
              const int slot = row[k];
              if (slot >= wend) break;
              pass.pair(T, pass.template fetch<Pass::kWin>(rec, slot - w0), g, acc);
            }
          }
          // a cell of a pipelined list has no list longer than kLC: one pass
          if (md.w & 0x8000u) break;
          const int more = __syncthreads_or(active && sub == 0 && tot[t] > (lp + 1) * kLC);
          if (!more) break;
        }
      }
      // the nsub partial sums of each target, added in a fixed order
      __syncthreads();
#pragma unroll
      for (int v = 0; v < Pass::kV; ++v) part[v * kPT + tid] = acc[v] + (acc2[v].x + acc2[v].y);
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

// ------------------------------------------------- pipelined pair passes --
//
// Cells staging at most kPipeW candidates are processed by a two-stage
// software pipeline: while a CTA computes cell i from one half of a double
// buffer, the records of cell i + 1 arrive in the other half by cp.async, the
// staged entries of cell i + 2 and the meta of cell i + 3 by plain loads into
// registers.  Each thread adds the cell shifts (a 27-entry table) to the
// records it copied itself once they have landed, so one barrier per cell
// publishes the records and one more the per-target partial sums.
//
// Thread (t, s) of target t takes entries s, s + nsub, ... of t's staged-slot
// list, so the threads of a warp step through their lists in lockstep.  The
// lists come from shared memory (passes with 16-byte records: the next cell's
// lists are copied by cp.async with its records) or from global memory
// through L1 (momentum, whose 64/72-byte records leave no room for list buffers:
// the next cell's list rows are prefetched into L1).

template <class Pass>
struct PipeSmem {
  static constexpr int PT = Pass::kPipeThreads;
  static constexpr int W = Pass::kPipeW;
  static constexpr bool L = Pass::kSmemLists;
  static constexpr size_t kRec = (size_t)W * Pass::kRecBytes;  // one buffer
  static constexpr size_t kList = L ? (size_t)kTR * kLS * sizeof(uint16_t) : 0;
  static constexpr size_t kCnt = L ? (size_t)kTR * sizeof(int) : 0;
  static constexpr size_t kPart = (size_t)PT * Pass::kV * sizeof(float);
  static constexpr size_t kTab = Tabs::kBytes;
  static constexpr size_t oList = 2 * kRec;
  static constexpr size_t oCnt = oList + 2 * kList;
  static constexpr size_t oPart = oCnt + 3 * kCnt;
  static constexpr size_t oTab = oPart + 2 * kPart;
  static constexpr size_t kBytes = oTab + kTab;
  static_assert(kRec % 16 == 0 && kList % 16 == 0 && kCnt % 16 == 0 && kPart % 16 == 0,
                "16-byte aligned parts");
  static_assert(PT <= 256, "nsub table sized for at most 256 targets");
};

// Cells of a pipelined launch: list 0 then list 1 (optional).
struct PipeSrc {
  const uint4* meta;
  const uint32_t* cells0;
  const unsigned long long* n0;
  const uint32_t* cells1;
  const unsigned long long* n1;
  const uint32_t* sent;
  const int32_t* nn;
  const uint16_t* slist;
  int max_nb;
};

// This thread's share of a cell's targets: target t (-1: none), its lane sub
// of nsub and the length of t's list (global-list passes).
struct Share {
  int t, sub, nsub, cnt;
};


template <class Pass>
__global__ void __launch_bounds__(Pass::kPipeThreads, Pass::kPipeMinBlocks) k_cellpipe(
    Pass pass, const Grid* gp, PipeSrc src) {
  using SM = PipeSmem<Pass>;
  constexpr int PT = SM::PT;
  constexpr int W = SM::W;
  constexpr bool kLists = SM::L;
  constexpr int U = (W + PT - 1) / PT;  // staged slots per thread
  constexpr int kV = Pass::kV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto rbuf = [&](int h) { return reinterpret_cast<float4*>(smem_raw + h * SM::kRec); };
  auto lbuf = [&](int h) {
    return reinterpret_cast<uint16_t*>(smem_raw + SM::oList + h * SM::kList);
  };
  auto tcnt = [&](int h) { return reinterpret_cast<int*>(smem_raw + SM::oCnt) + h * kTR; };
  auto part = [&](int h) {
    return reinterpret_cast<float*>(smem_raw + SM::oPart + h * SM::kPart);
  };
  const Grid g = *gp;
  if (!pass.runs(g)) return;
  const int tid = threadIdx.x;
  Tabs tb(smem_raw + SM::oTab);
  tb.fill<PT>(g);
  const float4* shtab = tb.shift;
  const uint32_t n0 = (uint32_t)*src.n0;
  const uint32_t n_cells = n0 + (src.cells1 ? (uint32_t)*src.n1 : 0u);
  const uint32_t G = gridDim.x;
  uint32_t q = blockIdx.x;
  if (q >= n_cells) return;
  const uint4 none = make_uint4(0u, kListForm, 0u, 0u);
  auto cell_at = [&](uint32_t qq) {
    return qq < n0 ? __ldg(src.cells0 + qq)
                   : (qq < n_cells ? __ldg(src.cells1 + (qq - n0)) : kNoCell);
  };
  auto meta_at = [&](uint32_t c) { return c != kNoCell ? __ldg(src.meta + c) : none; };
  auto present = [&](uint4 md) { return md.y != kListForm; };
  // staged entries of a cell's slots tid + u PT
  auto load_entries = [&](uint4 md, uint32_t* e) {
    const int S = present(md) ? cell_S(md) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = tid + u * PT;
      e[u] = j < S ? __ldg(src.sent + md.x + (uint32_t)j) : 0u;
    }
  };
  auto issue_records = [&](uint4 md, const uint32_t* e, float4* rec) {
    const int S = cell_S(md);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = tid + u * PT;
      if (j < S) pass.template copy_async<W>(rec, j, entry_index(e[u]));
    }
  };
  // the next cell's lists (shared-memory lists): 16-byte chunks of each row
  // this thread's target in a cell (nsub threads per target)
  auto target_of = [&](uint4 md, int& t, int& sub, int& nsub) {
    const int na = present(md) ? cell_na(md) : 0;
    nsub = tb.nsub[min(na, PT)];
    t = tb.div(tid, nsub);
    sub = tid - t * nsub;
    if (t >= na) t = -1;
  };
  // shared-memory lists: the count of target tid; global lists: of this
  // thread's target
  auto count_of = [&](uint4 md) {
    if (kLists) {
      const int na = present(md) ? cell_na(md) : 0;
      return tid < na ? min(__ldg(src.nn + md.z + tid), src.max_nb) : 0;
    }
    int t, sub, nsub;
    target_of(md, t, sub, nsub);
    return t >= 0 ? min(__ldg(src.nn + md.z + t), src.max_nb) : 0;
  };
  auto share_of = [&](uint4 md, int cnt) {
    Share sh;
    target_of(md, sh.t, sh.sub, sh.nsub);
    sh.cnt = sh.t >= 0 ? cnt : 0;
    return sh;
  };
  // the 128-byte lines of a cell's list rows (the first 2 max_nb bytes of each)
  const int lines = (2 * src.max_nb + 127) >> 7;
  auto prefetch_rows = [&](uint4 md) {
    const int na = present(md) ? cell_na(md) : 0;
    for (int i = tid; i < na * lines; i += PT) {
      const int t = i / lines;
      prefetch_l1(reinterpret_cast<const unsigned char*>(slot_row(
                      const_cast<uint16_t*>(src.slist), (int64_t)md.z + t, src.max_nb)) +
                  128 * (i - t * lines));
    }
  };
  // the next cell's lists (shared-memory lists): thread (t, s) copies the
  // 16-byte chunks s, s + nsub, ... of target t's row that hold entries
  auto issue_lists = [&](uint4 md, const Share& sh, const int* cnt, uint16_t* lst) {
    if (sh.t < 0) return;
    const int c = cnt[sh.t];
    const uint16_t* row =
        slot_row(const_cast<uint16_t*>(src.slist), (int64_t)md.z + sh.t, src.max_nb);
    uint16_t* dst = lst + sh.t * kLS;
    for (int k8 = 8 * sh.sub; k8 < c; k8 += 8 * sh.nsub) {
      if (k8 + 8 <= src.max_nb)
        cp_async16(dst + k8, row + k8);
      else  // the last 4 entries of a row of max_nb = 4 mod 8
        cp_async8(dst + k8, row + k8);
    }
  };
  // prologue: the first cell's copies, registers of the next two cells
  uint4 md_cur = meta_at(cell_at(q)), md_nxt = meta_at(cell_at(q + G));
  uint4 md_nn = meta_at(cell_at(q + 2 * G));
  uint32_t c_nnn = cell_at(q + 3 * G);
  uint32_t e_cur[U], e_nxt[U];
  load_entries(md_cur, e_cur);
  const int c_cur0 = count_of(md_cur);
  issue_records(md_cur, e_cur, rbuf(0));
  Share sh_cur = share_of(md_cur, c_cur0);
  if (kLists) {
    if (tid < kTR) tcnt(0)[tid] = c_cur0;
    __syncthreads();
    issue_lists(md_cur, sh_cur, tcnt(0), lbuf(0));
  } else {
    prefetch_rows(md_cur);
  }
  cp_async_commit();
  load_entries(md_nxt, e_nxt);
  int cnt_nxt = count_of(md_nxt);
  typename Pass::Target T_cur, T_nxt;
  if (!Pass::kTargetSmem && sh_cur.t >= 0) pass.load_target((int64_t)md_cur.z + sh_cur.t, T_cur);
  // the previous cell, whose per-target sums are added after this iteration's
  // barrier (its partial sums are in the other half of the partial buffer)
  int na_prv = 0, nsub_prv = 1;
  uint32_t a0_prv = 0;
  // the per-target reduction and finish of the previous cell: thread tid < na
  // adds the nsub partial sums of target tid in a fixed order
  auto finish_prev = [&](int ph, const typename Pass::FinishIn& fin) {
    if (tid < na_prv) {
      const float* pp = part(ph);
      float sm[kV];
#pragma unroll
      for (int v = 0; v < kV; ++v) {
        float x = 0.0f;
        for (int qq = 0; qq < nsub_prv; ++qq) x += pp[v * PT + tid * nsub_prv + qq];
        sm[v] = x;
      }
      pass.finish2((int64_t)a0_prv + tid, sm, fin);
    }
  };
  int buf = 0, cb = 0;  // record/list/partial half, count third
  for (;;) {
    typename Pass::FinishIn fin_prv;
    if (tid < na_prv) fin_prv = pass.prefin((int64_t)a0_prv + tid);
    // this cell's records have landed (the copies this thread made): add the
    // cell shifts to the records this thread copied
    cp_async_wait_all();
    {
      const int S = cell_S(md_cur);
      float4* rec = rbuf(buf);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = tid + u * PT;
        if (j < S) {
          const float4 sh = shtab[e_cur[u] >> kIndexBits];
          float4 r = rec[j];
          r.x += sh.x;
          r.y += sh.y;
          r.z += sh.z;
          rec[j] = r;
        }
      }
    }
    const bool has_nxt = q + G < n_cells;
    const int cb_nxt = cb == 2 ? 0 : cb + 1;
    // (the counts' third of two cells ago: read by no thread any more)
    if (kLists && has_nxt && tid < kTR) tcnt(cb_nxt)[tid] = cnt_nxt;
    __syncthreads();  // this cell's data published; the previous cell computed
    finish_prev(buf ^ 1, fin_prv);
    // the next cell's thread shares: needed here by the list copies, after the
    // next loads otherwise
    Share sh_nxt;
    if (kLists) sh_nxt = share_of(md_nxt, cnt_nxt);
    if (has_nxt) {
      issue_records(md_nxt, e_nxt, rbuf(buf ^ 1));
      if (kLists) issue_lists(md_nxt, sh_nxt, tcnt(cb_nxt), lbuf(buf ^ 1));
    }
    cp_async_commit();
    // registers for the next cells
    uint32_t e_nn[U];
    load_entries(md_nn, e_nn);
    const int cnt_nn = count_of(md_nn);
    const uint4 md_nnn = meta_at(c_nnn);
    c_nnn = cell_at(q + 4 * G);
    if (!kLists) {
      sh_nxt = share_of(md_nxt, cnt_nxt);
      prefetch_rows(md_nxt);
    }
    if (!Pass::kTargetSmem && sh_nxt.t >= 0)
      pass.load_target((int64_t)md_nxt.z + sh_nxt.t, T_nxt);
    // compute this cell
    const int na = cell_na(md_cur);
    const uint32_t a0 = md_cur.z;
    if (tid < na) pass.prefetch_fin((int64_t)a0 + tid);  // read by its finish next iteration
    float acc[kV];
    float2 acc2[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      acc[v] = 0.0f;
      acc2[v] = make_float2(0.0f, 0.0f);
    }
    if (sh_cur.t >= 0) {
      float4* rec = rbuf(buf);
      if (Pass::kTargetSmem)
        pass.template target_from<W>(rec, (int)md_cur.y + sh_cur.t, T_cur);
      const int ns = sh_cur.nsub;
      int k = sh_cur.sub;
      if (kLists) {
        const uint16_t* row = lbuf(buf) + sh_cur.t * kLS;
        const int c = tcnt(cb)[sh_cur.t];
        if (Pass::kPipePaired)
          for (; k + ns < c; k += 2 * ns)
            pass.pair2(T_cur, pass.template fetch<W>(rec, row[k]),
                       pass.template fetch<W>(rec, row[k + ns]), g, acc2);
        for (; k < c; k += ns) pass.pair(T_cur, pass.template fetch<W>(rec, row[k]), g, acc);
      } else {
        const uint16_t* row =
            slot_row(const_cast<uint16_t*>(src.slist), (int64_t)a0 + sh_cur.t, src.max_nb);
        const int c = sh_cur.cnt;
        if (Pass::kPipePaired)
          for (; k + ns < c; k += 2 * ns)
            pass.pair2(T_cur, pass.template fetch<W>(rec, __ldg(row + k)),
                       pass.template fetch<W>(rec, __ldg(row + k + ns)), g, acc2);
        // the next entry's slot is loaded (through L1) while this pair is summed
        int slot = k < c ? __ldg(row + k) : 0;
        for (; k < c; k += ns) {
          const int nxt = k + ns < c ? __ldg(row + k + ns) : 0;
          pass.pair(T_cur, pass.template fetch<W>(rec, slot), g, acc);
          slot = nxt;
        }
      }
    }
    {
      float* pp = part(buf);
#pragma unroll
      for (int v = 0; v < kV; ++v) pp[v * PT + tid] = acc[v] + (acc2[v].x + acc2[v].y);
    }
    na_prv = na;
    a0_prv = a0;
    nsub_prv = sh_cur.nsub;
    q += G;
    if (q >= n_cells) {
      // the last cell's sums
      typename Pass::FinishIn fin_last;
      if (tid < na_prv) fin_last = pass.prefin((int64_t)a0_prv + tid);
      __syncthreads();
      finish_prev(buf, fin_last);
      break;
    }
    md_cur = md_nxt;
    md_nxt = md_nn;
    md_nn = md_nnn;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      e_cur[u] = e_nxt[u];
      e_nxt[u] = e_nn[u];
    }
    sh_cur = sh_nxt;
    cnt_nxt = cnt_nn;
    if (!Pass::kTargetSmem) T_cur = T_nxt;
    buf ^= 1;
    cb = cb_nxt;
  }
}

template <class Pass>
int pipe_blocks(sph_ctx* ctx, int* cache) {
  if (!*cache) {  // once per context, on its device
    using SM = PipeSmem<Pass>;
    cudaFuncSetAttribute(k_cellpipe<Pass>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SM::kBytes);
    cudaFuncSetAttribute(k_cellpipe<Pass>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cellpipe<Pass>, SM::PT,
                                                  SM::kBytes);
    *cache = (per_sm > 0 ? per_sm : 1) * ctx->sm_count;
  }
  return *cache;
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
  // the pipelined kernel: cells of at most 448 staged candidates, and for the
  // passes with 16-byte records also those of 449..832
  PipeSrc ps;
  ps.meta = ctx->cmeta;
  ps.cells0 = ctx->cells;
  ps.n0 = ctx->salloc + 2;
  ps.cells1 = Pass::kPipeAll ? ctx->cells + 2 * ctx->n_max : nullptr;
  ps.n1 = ctx->salloc + 4;
  ps.sent = ctx->sent;
  ps.nn = ctx->nn;
  ps.slist = reinterpret_cast<uint16_t*>(ctx->nbr);
  ps.max_nb = ctx->prm.max_nb;
  k_cellpipe<Pass><<<pipe_blocks<Pass>(ctx, cache + 3), Pass::kPipeThreads,
                     PipeSmem<Pass>::kBytes, st>>>(p, ctx->grid, ps);
  // the general kernel: the other cells (for momentum also those of 449..832)
  Src src;
  src.meta = ctx->cmeta;
  src.sent = ctx->sent;
  src.nn = ctx->nn;
  src.nbr = ctx->nbr;
  src.slist = reinterpret_cast<uint16_t*>(ctx->nbr);
  src.max_nb = ctx->prm.max_nb;
  src.cells = ctx->cells + ctx->n_max;
  src.ncells = ctx->salloc + 3;
  k_cellpass<Pass><<<pass_blocks<Pass>(ctx, cache), kPT, PassSmem<Pass>::kBytes, st>>>(
      p, ctx->grid, src);
  ctx->launches += 2;
  if (!Pass::kPipeAll) {
    src.cells = ctx->cells + 2 * ctx->n_max;
    src.ncells = ctx->salloc + 4;
    k_cellpass<Pass><<<pass_blocks<Pass>(ctx, cache), kPT, PassSmem<Pass>::kBytes, st>>>(
        p, ctx->grid, src);
    ctx->launches += 1;
  }
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

// The lists of a particle as sorted ids: staged cells from the staged-slot
// list (slot -> staged entry -> particle), list-form cells from the int32 list.
__global__ void k_export_lists(int64_t n, const int32_t* nn, const uint32_t* cell_of,
                               const uint4* meta, const uint32_t* sent, const uint16_t* slist,
                               const uint32_t* nbr, int max_nb, const int64_t* id,
                               int32_t* counts, int64_t* ids) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    counts[a] = nn[a];
    const uint4 md = meta[cell_of[a]];
    int64_t* row = ids + a * max_nb;
    const int c = min(nn[a], max_nb);
    if (md.y == kListForm) {
      for (int k = 0; k < c; ++k) insert_sorted(row, k, id[entry_index(nbr[a * max_nb + k])]);
    } else {
      const uint16_t* srow = slist + 2 * a * max_nb;
      for (int k = 0; k < c; ++k) insert_sorted(row, k, id[entry_index(sent[md.x + srow[k]])]);
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
  const size_t smem = kFindWarps * (sizeof(FindWarpSmem) + kMaskBufWords * sizeof(unsigned long long));
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
  mo.slist = reinterpret_cast<uint16_t*>(ctx->nbr);
  mo.fcells = ctx->cells;
  mo.scells = ctx->cells + ctx->n_max;
  mo.mcells = ctx->cells + 2 * ctx->n_max;
  cudaMemsetAsync(ctx->salloc, 0, 5 * sizeof(unsigned long long), st);
  k_find_mask<false><<<ctx->find_mask_blocks, kFindThreads, smem, st>>>(
      ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start, ctx->tbl_count, ctx->nn, ctx->nbr,
      ctx->prm.max_nb, mo, ctx->err, ctx->stats);
  k_find_mask<true><<<ctx->find_mask_blocks, kFindThreads, smem, st>>>(
      ctx->grid, s, ctx->pos32, ctx->occ, ctx->tbl_start, ctx->tbl_count, ctx->nn, ctx->nbr,
      ctx->prm.max_nb, mo, ctx->err, ctx->stats);
  ctx->launches += 2;
}

// The pair passes run in the plain configuration (kCfgPlain) when the
// parameters allow it: the exact kernel with n = 6 and no grad-h terms.  The
// three passes take the same configuration, since the plain one also lays out
// the momentum records differently.  The general kernels are launched too and
// take over on grids that need the FP32 minimum image; one of the two returns
// at once.
inline bool plain_kernel(const sph_ctx* ctx) {
  return ctx->prm.kernel_mode == SPH_KERNEL_EXACT && ctx->prm.sinc_n == 6.0;
}

template <template <int> class PassT, class Fill>
void launch_cfg(sph_ctx* ctx, bool plain, int slot, Fill fill, cudaStream_t st) {
  if (plain) {
    PassT<kCfgPlain> q;
    fill(q);
    q.only_wrap = 0;
    launch_pass(ctx, q, &ctx->pass_blocks[6 + slot], st);
  }
  PassT<kCfgAny> p;
  fill(p);
  p.only_wrap = plain ? 1 : 0;
  launch_pass(ctx, p, &ctx->pass_blocks[slot], st);
}

void launch_density_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                           cudaStream_t st) {
  (void)n;
  auto fill = [&](auto& p) {
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
  };
  launch_cfg<DensityPassT>(ctx, plain_kernel(ctx) && !ctx->prm.gradh, 0, fill, st);
}

void launch_iad_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                       cudaStream_t st) {
  (void)s;
  (void)n;
  auto fill = [&](auto& p) {
    p.rec_i = ctx->rec_i;
    p.recA = ctx->recA;
    p.recQ = ctx->recQ;
    p.o = o;
    p.recC = ctx->recC;
    p.recC2 = ctx->recC2;
    p.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab32 : nullptr;
    p.Bn = (float)ctx->Bn;
    p.sinc_n = (int)ctx->prm.sinc_n;
    p.err = ctx->err;
  };
  launch_cfg<IadPassT>(ctx, plain_kernel(ctx) && !ctx->prm.gradh, 1, fill, st);
}

void launch_momentum_staged(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                            cudaStream_t st) {
  (void)s;
  (void)n;
  auto fill = [&](auto& p) {
    p.recA = ctx->recA;
    p.recV = ctx->recV;
    p.recQ = ctx->recQ;
    p.recC = ctx->recC;
    p.recC2 = ctx->recC2;
    p.o = o;
    p.ktab = ctx->prm.kernel_mode == SPH_KERNEL_TABLE ? ctx->ktab32 : nullptr;
    p.sinc_n = (int)ctx->prm.sinc_n;
    p.alpha = (float)ctx->prm.alpha;
    p.Bn = (float)ctx->Bn;
    p.inv_gamma = (float)(1.0 / ctx->prm.gamma);
    p.err = ctx->err;
  };
  launch_cfg<MomentumPassT>(ctx, plain_kernel(ctx) && !ctx->prm.gradh, 2, fill, st);
}

void launch_export_masks(sph_ctx* ctx, const StateView& s, int64_t n, int32_t* counts,
                         int64_t* ids, cudaStream_t st) {
  int64_t b = (n + 127) / 128;
  if (b > (int64_t)ctx->sm_count * 32) b = ctx->sm_count * 32;
  if (b < 1) b = 1;
  k_export_lists<<<(int)b, 128, 0, st>>>(n, ctx->nn, ctx->cell_of, ctx->cmeta, ctx->sent,
                                         reinterpret_cast<const uint16_t*>(ctx->nbr), ctx->nbr,
                                         ctx->prm.max_nb, s.id, counts, ids);
  ctx->launches += 1;
}

}  // namespace sph
