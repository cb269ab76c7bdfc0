// Self-gravity (sph_gravity in include/sph.h): section 4.1 evaluates it by a
// multipolar expansion on the tree used to find neighbours.  Here the tree's
// leaves are the occupied cells of the neighbour grid (side >= 2 h_max, in
// Morton order after the library's sort) and a node of level l groups the
// cells that share the top 3 l bits of their Morton code.
//
//   build     leaves from the occupied-cell list; each upper level by a flag
//             per run of equal parent codes (code >> 3) and an exclusive scan
//   moments   leaves from their particles (mass, centre of mass c, traceless
//             quadrupole Q_ij = sum m (3 d_i d_j - |d|^2 delta_ij), d = x - c,
//             two passes); parents from their children by the parallel-axis
//             rule Q = sum (Q_k + M_k (3 e e^T - |e|^2 I)), e = c_k - c
//   walk      per particle, depth first from the root with the children in
//             Morton order: a node whose box does not contain the particle and
//             whose longest side s satisfies s < theta |x - c| adds the
//             softened monopole and the quadrupole term; an opened leaf adds
//             its particles by the direct softened formula; other nodes are
//             opened.  A warp walks its 32 particles together on one stack of
//             (node, lane mask) entries (k_walk).
// Everything is FP64, and the walk visits nodes in the same order as the
// oracle's recursion.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_scan.cuh"

namespace sph {
namespace grav {

struct Node {
  double box_lo[3], box_hi[3];
  double size, M;
  double c[3];
  double Q[6];      // xx xy xz yy yz zz
  int32_t first;    // first child (node index), -1 for a leaf
  int32_t nchild;
  int32_t p0, np;   // particles [p0, p0 + np) of the sorted order
};

constexpr int kStack = 80;  // >= 7 * 8 + 8 pending nodes for up to 8 Morton bits

__device__ __forceinline__ uint32_t compact3(uint32_t v) {
  uint32_t r = 0;
  for (int i = 0; i < 10; ++i) r |= ((v >> (3 * i)) & 1u) << i;
  return r;
}

// Box and longest side of the node with Morton prefix `code` at level `l`.
__device__ __forceinline__ void node_box(const Grid& g, uint32_t code, int l, Node& nd) {
  const int span = 1 << (g.bits - l);
  const uint32_t c3[3] = {compact3(code), compact3(code >> 1), compact3(code >> 2)};
  double size = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    const int c0 = (int)c3[ax] * span;
    int c1 = c0 + span - 1;
    if (c1 > g.nc[ax] - 1) c1 = g.nc[ax] - 1;
    nd.box_lo[ax] = g.lo[ax] + c0 * g.cs[ax];
    nd.box_hi[ax] = g.lo[ax] + (c1 + 1) * g.cs[ax];
    const double ext = nd.box_hi[ax] - nd.box_lo[ax];
    size = ext > size ? ext : size;
  }
  nd.size = size;
}

__global__ void k_leaves(const Grid* gp, const uint32_t* occ, const uint32_t* tbl_start,
                         const uint32_t* tbl_count, int64_t n_occ, uint32_t* code, Node* nodes,
                         StateView s) {
  const Grid g = *gp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_occ;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cc = occ[i];
    code[i] = cc;
    Node nd;
    nd.first = -1;
    nd.nchild = 0;
    nd.p0 = (int32_t)tbl_start[cc];
    nd.np = (int32_t)tbl_count[cc];
    node_box(g, cc, g.bits, nd);
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int32_t b = nd.p0; b < nd.p0 + nd.np; ++b) {
      M += s.m[b];
      sx += s.m[b] * s.x[b];
      sy += s.m[b] * s.y[b];
      sz += s.m[b] * s.z[b];
    }
    nd.M = M;
    nd.c[0] = sx / M;
    nd.c[1] = sy / M;
    nd.c[2] = sz / M;
    double Q[6] = {0, 0, 0, 0, 0, 0};
    for (int32_t b = nd.p0; b < nd.p0 + nd.np; ++b) {
      const double dx = s.x[b] - nd.c[0], dy = s.y[b] - nd.c[1], dz = s.z[b] - nd.c[2];
      const double d2 = (dx * dx + dy * dy) + dz * dz;
      const double mb = s.m[b];
      Q[0] += mb * (3 * dx * dx - d2);
      Q[1] += mb * (3 * dx * dy);
      Q[2] += mb * (3 * dx * dz);
      Q[3] += mb * (3 * dy * dy - d2);
      Q[4] += mb * (3 * dy * dz);
      Q[5] += mb * (3 * dz * dz - d2);
    }
    for (int q = 0; q < 6; ++q) nd.Q[q] = Q[q];
    nodes[i] = nd;
  }
}

__global__ void k_run_flags(const uint32_t* code, int64_t m, int32_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || (code[i] >> 3) != (code[i - 1] >> 3)) ? 1 : 0;
}

// Parents of the m children at nodes[coff ..): code, first child, first particle.
__global__ void k_parents(const uint32_t* code, const int32_t* flag, const int64_t* idx, int64_t m,
                          int64_t coff, int64_t poff, uint32_t* pcode, Node* nodes) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    const int64_t j = idx[i];
    pcode[j] = code[i] >> 3;
    nodes[poff + j].first = (int32_t)(coff + i);
    nodes[poff + j].p0 = nodes[coff + i].p0;
  }
}

// Child counts, particle counts, boxes and moments (parallel-axis rule).
__global__ void k_parent_moments(const Grid* gp, const uint32_t* pcode, int64_t npar, int64_t m,
                                 int64_t coff, int64_t poff, int level, Node* nodes) {
  const Grid g = *gp;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < npar;
       j += (int64_t)gridDim.x * blockDim.x) {
    Node nd = nodes[poff + j];
    const int64_t f = nd.first - coff;
    const int64_t next = j + 1 < npar ? nodes[poff + j + 1].first - coff : m;
    nd.nchild = (int32_t)(next - f);
    const Node& last = nodes[coff + next - 1];
    nd.np = last.p0 + last.np - nd.p0;
    node_box(g, pcode[j], level, nd);
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t k = coff + f; k < coff + next; ++k) {
      const Node& ch = nodes[k];
      M += ch.M;
      sx += ch.M * ch.c[0];
      sy += ch.M * ch.c[1];
      sz += ch.M * ch.c[2];
    }
    nd.M = M;
    nd.c[0] = sx / M;
    nd.c[1] = sy / M;
    nd.c[2] = sz / M;
    double Q[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = coff + f; k < coff + next; ++k) {
      const Node& ch = nodes[k];
      const double ex = ch.c[0] - nd.c[0], ey = ch.c[1] - nd.c[1], ez = ch.c[2] - nd.c[2];
      const double e2 = (ex * ex + ey * ey) + ez * ez;
      Q[0] += ch.Q[0] + ch.M * (3 * ex * ex - e2);
      Q[1] += ch.Q[1] + ch.M * (3 * ex * ey);
      Q[2] += ch.Q[2] + ch.M * (3 * ex * ez);
      Q[3] += ch.Q[3] + ch.M * (3 * ey * ey - e2);
      Q[4] += ch.Q[4] + ch.M * (3 * ey * ez);
      Q[5] += ch.Q[5] + ch.M * (3 * ez * ez - e2);
    }
    for (int q = 0; q < 6; ++q) nd.Q[q] = Q[q];
    nodes[poff + j] = nd;
  }
}

// The opening decision: accept a node whose box does not contain p and whose
// longest side is below theta |p - c| (r = p - c, R2, R returned).
__device__ __forceinline__ bool accept64(const Node& nd, const double p[3], double theta,
                                         double r[3], double& R2, double& R) {
  bool inside = true;
  for (int ax = 0; ax < 3; ++ax)
    if (p[ax] < nd.box_lo[ax] || p[ax] > nd.box_hi[ax]) inside = false;
  for (int ax = 0; ax < 3; ++ax) r[ax] = p[ax] - nd.c[ax];
  R2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
  R = sqrt(R2);
  return !inside && nd.size < theta * R;
}

// The walk of a warp: 32 consecutive sorted particles (one lane each) share
// one depth-first stack whose entries carry the mask of lanes that reached
// the node through nodes they opened.  Every lane still takes its own
// decisions and sees its nodes in its own depth-first order (so the result
// equals a walk per particle), but node and particle loads are common to the
// warp and an opened leaf is summed by all its lanes in lockstep.
constexpr int kWalkWarps = 4;

__global__ void __launch_bounds__(32 * kWalkWarps) k_walk(const Node* nodes, int32_t root,
                                                          StateView s, int64_t n, double G,
                                                          double eps, double theta, double* gx,
                                                          double* gy, double* gz,
                                                          unsigned long long* stats,
                                                          uint32_t* err) {
  __shared__ int32_t st_node[kWalkWarps][kStack];
  __shared__ uint32_t st_mask[kWalkWarps][kStack];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long nodes_used = 0, pairs = 0;
  const double eps2 = eps * eps;
  const int64_t tiles = (n + 31) / 32;
  for (int64_t tile = blockIdx.x * (int64_t)kWalkWarps + w; tile < tiles;
       tile += (int64_t)gridDim.x * kWalkWarps) {
    const int64_t a = tile * 32 + lane;
    const bool valid = a < n;
    const double p[3] = {valid ? s.x[a] : 0.0, valid ? s.y[a] : 0.0, valid ? s.z[a] : 0.0};
    double acc[3] = {0.0, 0.0, 0.0};
    int sp = 0;
    const uint32_t all = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) {
      st_node[w][0] = root;
      st_mask[w][0] = all;
    }
    sp = 1;
    __syncwarp();
    bool overflow = false;
    while (sp > 0) {
      --sp;
      const int32_t k = st_node[w][sp];
      const uint32_t mask = st_mask[w][sp];
      __syncwarp();
      const Node& nd = nodes[k];
      const bool live = (mask >> lane) & 1u;
      bool open = false;
      if (live) {
        double r[3], R2, R;
        if (accept64(nd, p, theta, r, R2, R)) {
          // one reciprocal and one reciprocal square root per node: the FP64
          // pipe runs divisions and square roots as multi-instruction sequences
          const double inv_s = rsqrt(R2 + eps2);
          const double mono = G * nd.M * (inv_s * inv_s * inv_s);
          const double inv_R = 1.0 / R;
          const double inv_R2 = inv_R * inv_R;
          const double g5 = G * (inv_R2 * inv_R2 * inv_R);
          const double* Q = nd.Q;
          const double Qr[3] = {Q[0] * r[0] + Q[1] * r[1] + Q[2] * r[2],
                                Q[1] * r[0] + Q[3] * r[1] + Q[4] * r[2],
                                Q[2] * r[0] + Q[4] * r[1] + Q[5] * r[2]};
          const double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
          const double g7 = 2.5 * g5 * rQr * inv_R2;
          for (int i = 0; i < 3; ++i) acc[i] += -mono * r[i] + g5 * Qr[i] - g7 * r[i];
          ++nodes_used;
        } else {
          open = true;
        }
      }
      const uint32_t omask = __ballot_sync(0xffffffffu, open);
      if (omask == 0) continue;
      if (nd.first < 0) {
        // an opened leaf: its particles, in order, for the lanes that opened it
        for (int32_t b = nd.p0; b < nd.p0 + nd.np; ++b) {
          const double xb = s.x[b], yb = s.y[b], zb = s.z[b], mb = s.m[b];
          if (open && b != a) {
            const double d[3] = {p[0] - xb, p[1] - yb, p[2] - zb};
            const double inv = rsqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] + eps2);
            const double f = G * mb * (inv * inv * inv);
            for (int q = 0; q < 3; ++q) acc[q] -= f * d[q];
            ++pairs;
          }
        }
      } else {
        if (sp + nd.nchild > kStack) {  // cannot happen for <= 8 Morton bits; kept as a guard
          overflow = true;
          break;
        }
        if (lane == 0)
          for (int j = nd.nchild - 1, q = sp; j >= 0; --j, ++q) {
            st_node[w][q] = nd.first + j;
            st_mask[w][q] = omask;
          }
        sp += nd.nchild;
        __syncwarp();
      }
    }
    if (overflow && lane == 0) raise_flag(err, SPH_FLAG_CELL_OVERFLOW);
    if (valid) {
      gx[a] = acc[0];
      gy[a] = acc[1];
      gz[a] = acc[2];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nodes_used += __shfl_xor_sync(0xffffffffu, nodes_used, o);
    pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
  }
  if (lane == 0) {
    atomicAdd(stats, nodes_used);
    atomicAdd(stats + 1, pairs);
  }
}

// ---- FP32-mixed walk ------------------------------------------------------
// The node and particle terms in FP32, the opening decisions exact, and no
// FP64 operation inside the walk (the FP64 pipe runs at 1/64 of the FP32
// rate).  Coordinates are taken relative to the grid origin lo and split into
// an FP32 head and tail (v = hi + lo to about 2^-48 |v|), so r = x_a - c is
// (hi_a - hi_c) + (lo_a - lo_c) with FP32 rounding relative to |r| instead of
// to the box.  Each particle is stored relative to its leaf's centre of mass,
// so a lane that opens a leaf forms x_a - x_b as r - (x_b - c).

struct NodeF {     // 96 B, read with uniform (broadcast) loads
  float4 cm;       // hi(c - lo), M
  float4 q1;       // Q yz zz, size, lo(c - lo).x
  float4 lo;       // box_lo - lo, lo(c - lo).y
  float4 hi;       // box_hi - lo, lo(c - lo).z
  float4 q0;       // Q xx xy xz yy
  int4 t;          // first, nchild, p0, np
};

__device__ __forceinline__ void split2(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

__global__ void k_nodes32(const Node* nodes, int64_t nn, double lx, double ly, double lz,
                          NodeF* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn;
       k += (int64_t)gridDim.x * blockDim.x) {
    const Node& nd = nodes[k];
    float ch[3], cl[3];
    split2(nd.c[0] - lx, ch[0], cl[0]);
    split2(nd.c[1] - ly, ch[1], cl[1]);
    split2(nd.c[2] - lz, ch[2], cl[2]);
    NodeF f;
    f.cm = make_float4(ch[0], ch[1], ch[2], (float)nd.M);
    f.q1 = make_float4((float)nd.Q[4], (float)nd.Q[5], (float)nd.size, cl[0]);
    f.lo = make_float4((float)(nd.box_lo[0] - lx), (float)(nd.box_lo[1] - ly),
                       (float)(nd.box_lo[2] - lz), cl[1]);
    f.hi = make_float4((float)(nd.box_hi[0] - lx), (float)(nd.box_hi[1] - ly),
                       (float)(nd.box_hi[2] - lz), cl[2]);
    f.q0 = make_float4((float)nd.Q[0], (float)nd.Q[1], (float)nd.Q[2], (float)nd.Q[3]);
    f.t = make_int4(nd.first, nd.nchild, nd.p0, nd.np);
    out[k] = f;
  }
}

// Particle b of leaf k: (x_b - c_k, m_b) in FP32.
__global__ void k_leaf_offsets(const Node* nodes, int64_t n_leaves, StateView s, float4* po) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_leaves;
       k += (int64_t)gridDim.x * blockDim.x) {
    const Node& nd = nodes[k];
    for (int32_t b = nd.p0; b < nd.p0 + nd.np; ++b)
      po[b] = make_float4((float)(s.x[b] - nd.c[0]), (float)(s.y[b] - nd.c[1]),
                          (float)(s.z[b] - nd.c[2]), (float)s.m[b]);
  }
}

// Constants of the FP32 walk, converted on the host.
struct Walk32Consts {
  double lx, ly, lz;   // grid origin
  double theta;        // for the FP64 decision
  float G, eps2, th;
  float mb;            // box-face margin: covers the FP32 rounding of box and head
  float aL;            // absolute distance margin
};

// Same warp walk as k_walk.  The FP32 decision uses margins that cover the
// rounding of the stored box faces and of the particle's head (each <= L
// 2^-24, L the grid's largest extent) and of the FP32 distance (relative
// 2^-22 with rsqrtf): mb on a box face, aL + 2e-6 R on the distance.  A lane
// inside a margin takes the FP64 decision of k_walk (accept64 on the FP64
// node), so every lane accepts and opens exactly the nodes that the FP64 walk
// does.
__global__ void __launch_bounds__(32 * kWalkWarps) k_walk32(const Node* nodes,
                                                            const NodeF* nf, const float4* po,
                                                            int32_t root, StateView s,
                                                            int64_t n, Walk32Consts k32,
                                                            double* gx, double* gy, double* gz,
                                                            unsigned long long* stats,
                                                            uint32_t* err) {
  __shared__ int32_t st_node[kWalkWarps][kStack];
  __shared__ uint32_t st_mask[kWalkWarps][kStack];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long nodes_used = 0, pairs = 0;
  const int64_t tiles = (n + 31) / 32;
  for (int64_t tile = blockIdx.x * (int64_t)kWalkWarps + w; tile < tiles;
       tile += (int64_t)gridDim.x * kWalkWarps) {
    const int64_t a = tile * 32 + lane;
    const bool valid = a < n;
    const int32_t a32 = valid ? (int32_t)a : -1;
    float ph[3], pl[3];
    split2((valid ? s.x[a] : 0.0) - k32.lx, ph[0], pl[0]);
    split2((valid ? s.y[a] : 0.0) - k32.ly, ph[1], pl[1]);
    split2((valid ? s.z[a] : 0.0) - k32.lz, ph[2], pl[2]);
    float acc[3] = {0.f, 0.f, 0.f};
    const uint32_t all = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) {
      st_node[w][0] = root;
      st_mask[w][0] = all;
    }
    int sp = 1;
    __syncwarp();
    bool overflow = false;
    while (sp > 0) {
      --sp;
      const int32_t k = st_node[w][sp];
      const uint32_t mask = st_mask[w][sp];
      __syncwarp();
      const NodeF* f = nf + k;
      const float4 cm = __ldg(&f->cm);
      const float4 q1 = __ldg(&f->q1);
      const float4 blo = __ldg(&f->lo), bhi = __ldg(&f->hi);
      const int4 t = __ldg(&f->t);
      const bool live = (mask >> lane) & 1u;
      bool open = false;
      float r[3];
      r[0] = (ph[0] - cm.x) + (pl[0] - q1.w);
      r[1] = (ph[1] - cm.y) + (pl[1] - blo.w);
      r[2] = (ph[2] - cm.z) + (pl[2] - bhi.w);
      if (live) {
        const float R2 = fmaf(r[2], r[2], fmaf(r[1], r[1], r[0] * r[0]));
        const float inv_R = rsqrtf(R2);
        const float Rf = R2 * inv_R;
        const float size = q1.z, mb = k32.mb;
        // the box: certainly outside, certainly inside, or within mb of a face.
        // dmin is the smallest signed distance of the particle to a face
        // (negative outside); its own rounding (<= L 2^-24) adds to the
        // stored faces' and the head's, all within mb = 4 L 2^-24.
        const float dmin =
            fminf(fminf(fminf(ph[0] - blo.x, bhi.x - ph[0]), fminf(ph[1] - blo.y, bhi.y - ph[1])),
                  fminf(ph[2] - blo.z, bhi.z - ph[2]));
        const bool out_c = dmin < -mb;
        const bool in_c = dmin >= mb;
        const bool acc_c = size * (1.f + 1e-6f) < k32.th * (Rf * (1.f - 2e-6f) - k32.aL);
        const bool rej_c = size * (1.f - 1e-6f) > k32.th * (Rf * (1.f + 2e-6f) + k32.aL);
        bool accept;
        if (in_c || rej_c) {
          accept = false;
        } else if (out_c && acc_c) {
          accept = true;
        } else {
          // FP64 positions are reloaded here rather than kept live across the walk
          const double p[3] = {s.x[a], s.y[a], s.z[a]};
          double r64[3], R2_64, R64;
          accept = accept64(nodes[k], p, k32.theta, r64, R2_64, R64);
        }
        if (accept) {
          const float4 q0 = __ldg(&f->q0);
          const float inv_s = rsqrtf(R2 + k32.eps2);
          const float mono = k32.G * cm.w * (inv_s * inv_s * inv_s);
          const float inv_R2 = inv_R * inv_R;
          const float g5 = k32.G * (inv_R2 * inv_R2 * inv_R);
          const float Qr[3] = {q0.x * r[0] + q0.y * r[1] + q0.z * r[2],
                               q0.y * r[0] + q0.w * r[1] + q1.x * r[2],
                               q0.z * r[0] + q1.x * r[1] + q1.y * r[2]};
          const float rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
          const float g7 = 2.5f * g5 * rQr * inv_R2;
          for (int i = 0; i < 3; ++i) acc[i] += -mono * r[i] + g5 * Qr[i] - g7 * r[i];
          ++nodes_used;
        } else {
          open = true;
        }
      }
      const uint32_t omask = __ballot_sync(0xffffffffu, open);
      if (omask == 0) continue;
      if (t.x < 0) {
        // an opened leaf: x_a - x_b = r - (x_b - c), its particles in order
        for (int32_t b = t.z; b < t.z + t.w; ++b) {
          const float4 o = __ldg(po + b);
          if (open && b != a32) {
            const float d[3] = {r[0] - o.x, r[1] - o.y, r[2] - o.z};
            const float inv =
                rsqrtf(fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0])) + k32.eps2);
            const float fb = k32.G * o.w * (inv * inv * inv);
            for (int c = 0; c < 3; ++c) acc[c] -= fb * d[c];
            ++pairs;
          }
        }
      } else {
        if (sp + t.y > kStack) {  // cannot happen for <= 8 Morton bits; kept as a guard
          overflow = true;
          break;
        }
        if (lane == 0)
          for (int j = t.y - 1, q = sp; j >= 0; --j, ++q) {
            st_node[w][q] = t.x + j;
            st_mask[w][q] = omask;
          }
        sp += t.y;
        __syncwarp();
      }
    }
    if (overflow && lane == 0) raise_flag(err, SPH_FLAG_CELL_OVERFLOW);
    if (valid) {
      gx[a] = acc[0];
      gy[a] = acc[1];
      gz[a] = acc[2];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nodes_used += __shfl_xor_sync(0xffffffffu, nodes_used, o);
    pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
  }
  if (lane == 0) {
    atomicAdd(stats, nodes_used);
    atomicAdd(stats + 1, pairs);
  }
}

inline int blocks_for(int64_t n, int sm, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sm * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace grav
}  // namespace sph

namespace {

int gfail(sph_ctx* ctx, cudaError_t e, const char* what) { return sph::cuda_fail(ctx, e, what); }

// Grow-only scratch of the gravity call.
int grav_scratch(sph_ctx* ctx, size_t bytes) {
  if (ctx->grav_bytes >= bytes) return SPH_OK;
  if (ctx->grav_buf) cudaFree(ctx->grav_buf);
  ctx->grav_buf = nullptr;
  ctx->grav_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->grav_buf, bytes);
  if (e != cudaSuccess) return gfail(ctx, e, "sph_gravity scratch");
  ctx->grav_bytes = bytes;
  return SPH_OK;
}

}  // namespace

extern "C" int sph_gravity(sph_ctx* ctx, sph_state* state, double G, double eps, double theta,
                           double* gx, double* gy, double* gz, int64_t* interactions,
                           sph_stream_t stream) {
  using sph::grav::Node;
  if (!ctx) return SPH_ERR_INVALID_ARG;
  if (!state) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "NULL state");
  const int64_t n = state->n;
  if (n < 0 || n > ctx->n_max)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "n = %lld outside [0, n_max]", (long long)n);
  if (!(theta >= 0.0) || !(eps >= 0.0) || !(G == G))
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "theta and eps must be >= 0");
  for (int k = 0; k < 3; ++k)
    if (ctx->prm.periodic[k])
      return sph::set_error(ctx, SPH_ERR_INVALID_ARG,
                            "self-gravity needs open boundaries on every axis");
  if (n == 0) {  // nothing to read or write: the arrays may be NULL
    if (interactions) interactions[0] = interactions[1] = 0;
    return SPH_OK;
  }
  if (!gx || !gy || !gz) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "NULL output");
  const double* req[] = {state->x, state->y, state->z, state->vx, state->vy, state->vz,
                         state->vxh, state->vyh, state->vzh, state->h, state->m, state->u,
                         state->du_prev};
  for (const double* q : req)
    if (!q) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "a state array is NULL");
  if (!state->id) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "id is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  sph::StateView in;
  in.x = state->x;
  in.y = state->y;
  in.z = state->z;
  in.vx = state->vx;
  in.vy = state->vy;
  in.vz = state->vz;
  in.vxh = state->vxh;
  in.vyh = state->vyh;
  in.vzh = state->vzh;
  in.h = state->h;
  in.m = state->m;
  in.u = state->u;
  in.du_prev = state->du_prev;
  in.id = state->id;
  // the library's grid and Morton sort (the state is reordered in place)
  sph::launch_grid(ctx, in, n, st);
  sph::launch_sort_gather(ctx, in, n, st);
  sph::launch_copy_state(in, ctx->s, n, st, ctx);
  ctx->have_lists = 0;
  ctx->have_density = ctx->have_iad = 0;
  sph::Grid g;
  cudaError_t e = cudaMemcpyAsync(&g, ctx->grid, sizeof(g), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gfail(ctx, e, "sph_gravity grid");
  const int64_t n_occ = g.n_occ;
  const int bits = g.bits;
  // scratch: nodes (worst case n_occ per level), two code arrays, flags, scan
  const int64_t cap = n_occ * (bits + 1) + 1;
  const int64_t nparts = (n_occ + sph::scan::kScanItems - 1) / sph::scan::kScanItems + 1;
  const size_t off_code0 = sizeof(Node) * (size_t)cap;
  const size_t off_code1 = off_code0 + sizeof(uint32_t) * (size_t)n_occ;
  const size_t off_flag = off_code1 + sizeof(uint32_t) * (size_t)n_occ;
  const size_t off_idx = (off_flag + sizeof(int32_t) * (size_t)n_occ + 15) & ~(size_t)15;
  const size_t off_part = off_idx + sizeof(int64_t) * (size_t)(n_occ + 1);
  const size_t off_stats = off_part + sizeof(int64_t) * (size_t)nparts;
  const bool fp32 = ctx->prm.precision == SPH_FP32_MIXED;
  const size_t off_nf = (off_stats + 2 * sizeof(unsigned long long) + 127) & ~(size_t)127;
  const size_t off_po = off_nf + (fp32 ? sizeof(sph::grav::NodeF) * (size_t)cap : 0);
  const size_t bytes = off_po + (fp32 ? sizeof(float4) * (size_t)n : 0);
  int rc = grav_scratch(ctx, bytes);
  if (rc != SPH_OK) return rc;
  char* base = (char*)ctx->grav_buf;
  Node* nodes = (Node*)base;
  uint32_t* code_a = (uint32_t*)(base + off_code0);
  uint32_t* code_b = (uint32_t*)(base + off_code1);
  int32_t* flag = (int32_t*)(base + off_flag);
  int64_t* idx = (int64_t*)(base + off_idx);
  int64_t* part = (int64_t*)(base + off_part);
  unsigned long long* stats = (unsigned long long*)(base + off_stats);
  e = cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return gfail(ctx, e, "sph_gravity");
  const int sm = ctx->sm_count;
  sph::grav::k_leaves<<<sph::grav::blocks_for(n_occ, sm, 128), 128, 0, st>>>(
      ctx->grid, ctx->occ, ctx->tbl_start, ctx->tbl_count, n_occ, code_a, nodes, in);
  ctx->launches += 1;
  int64_t coff = 0, m = n_occ, noff = n_occ;
  for (int l = bits - 1; l >= 0; --l) {
    sph::grav::k_run_flags<<<sph::grav::blocks_for(m, sm, 256), 256, 0, st>>>(code_a, m, flag);
    sph::scan::exclusive_scan(flag, m, part, idx, st);
    int64_t npar = 0;
    e = cudaMemcpyAsync(&npar, idx + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return gfail(ctx, e, "sph_gravity tree level");
    sph::grav::k_parents<<<sph::grav::blocks_for(m, sm, 256), 256, 0, st>>>(
        code_a, flag, idx, m, coff, noff, code_b, nodes);
    sph::grav::k_parent_moments<<<sph::grav::blocks_for(npar, sm, 128), 128, 0, st>>>(
        ctx->grid, code_b, npar, m, coff, noff, l, nodes);
    ctx->launches += 6;
    uint32_t* t = code_a;
    code_a = code_b;
    code_b = t;
    coff = noff;
    noff += npar;
    m = npar;
  }
  const int32_t root = (int32_t)(noff - 1);
  const int64_t tiles = (n + 31) / 32;
  int wb = (int)((tiles + sph::grav::kWalkWarps - 1) / sph::grav::kWalkWarps);
  if (wb > sm * 256) wb = sm * 256;
  if (fp32) {
    sph::grav::NodeF* nf = (sph::grav::NodeF*)(base + off_nf);
    float4* po = (float4*)(base + off_po);
    double L = 0.0;
    for (int ax = 0; ax < 3; ++ax) L = fmax(L, 1.001 * g.nc[ax] * g.cs[ax]);
    sph::grav::k_nodes32<<<sph::grav::blocks_for(noff, sm, 128), 128, 0, st>>>(
        nodes, noff, g.lo[0], g.lo[1], g.lo[2], nf);
    sph::grav::k_leaf_offsets<<<sph::grav::blocks_for(n_occ, sm, 128), 128, 0, st>>>(
        nodes, n_occ, in, po);
    sph::grav::Walk32Consts k32;
    k32.lx = g.lo[0];
    k32.ly = g.lo[1];
    k32.lz = g.lo[2];
    k32.theta = theta;
    k32.G = (float)G;
    k32.eps2 = (float)(eps * eps);
    k32.th = (float)theta;
    k32.mb = (float)(4.0 * L * 5.9604644775390625e-8);  // 4 L 2^-24
    k32.aL = (float)(8.0 * L * 5.9604644775390625e-8);  // 8 L 2^-24
    sph::grav::k_walk32<<<wb, 32 * sph::grav::kWalkWarps, 0, st>>>(
        nodes, nf, po, root, in, n, k32, gx, gy, gz, stats, ctx->err);
    ctx->launches += 3;
  } else {
    sph::grav::k_walk<<<wb, 32 * sph::grav::kWalkWarps, 0, st>>>(nodes, root, in, n, G, eps,
                                                                 theta, gx, gy, gz, stats,
                                                                 ctx->err);
    ctx->launches += 1;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return gfail(ctx, e, "sph_gravity launch");
  if (interactions) {
    unsigned long long h[2];
    e = cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return gfail(ctx, e, "sph_gravity stats");
    interactions[0] = (int64_t)h[0];
    interactions[1] = (int64_t)h[1];
  }
  return SPH_OK;
}
