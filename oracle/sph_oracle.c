/*
 * sph_oracle.c -- plain, slow, FP64 CPU oracle of the SPH per-step pipeline.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference against
 * which the CUDA library is checked.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no source, header, table or constant with the CUDA library.
 *
 * Paper: Cavelan, Cabezon, Grabarczyk, Ciorba, "A Smoothed Particle
 * Hydrodynamics Mini-App for Exascale" (arXiv 2005.02656).  Section numbers
 * below are the paper's:
 *   section 4.1 "SPH": Eq. 1 (density), Eq. 2 (momentum), Eq. 3 (energy),
 *                      Eq. 4 (viscous acceleration), Eq. 5 (Pi'_ab),
 *                      Eq. 6 (sinc kernel family), integrator named in words;
 *   section 4.2: the global minimum time-step and the conservation sums;
 *   section 4.3: neighbour search over the tree / cells.
 * Where the paper is silent or garbled the reading applied is stated at the
 * function that applies it.
 *
 * Style: every loop follows the equations literally.  No blocking, fusion or
 * reordering; per-particle loops carry an OpenMP pragma only so large cases
 * finish in reasonable time (each iteration is independent, so the result
 * does not depend on the thread count).  Build with -ffp-contract=off so that
 * no multiply-add is fused: the neighbour criterion is then bit-reproducible.
 *
 * Conventions: arrays are structure-of-arrays in FP64, indexed by particle
 * index 0..n-1.  Functions that take (nt, targets) compute only for the listed
 * particle indices (targets == NULL means all n); their per-target outputs
 * are indexed by target slot t = 0..nt-1.  Neighbour lists are int64 particle
 * indices, nbr[t*max_nb + k], sorted ascending, self excluded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_INVALID_ARG (-1)
#define ORACLE_NB_OVERFLOW (-3)
#define ORACLE_SINGULAR_IAD (-4)
#define ORACLE_NONFINITE (-5)

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  double lo[3], hi[3]; /* box corners; used on periodic axes (and for cells) */
  int periodic[3];     /* 1 = periodic axis, 0 = open axis                   */
} oracle_box;

/* ------------------------------------------------------------------------- */
/* Sinc kernel family, section 4.1 Eq. 6.                                    */
/*   W(v,h) = B_n / h^3 * [ sin(pi v/2) / (pi v/2) ]^n   for 0 <= v <= 2,     */
/*   0 for v > 2, with v = |x_a - x_b| / h_a and d = 3.                       */
/* ------------------------------------------------------------------------- */

/* sinc(pi v / 2) with sinc(0) = 1; libm sin. */
static double sinc_half_pi(double v) {
  if (v == 0.0) return 1.0;
  double x = 0.5 * M_PI * v;
  return sin(x) / x;
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_m
 * (textbook construction: three-term recurrence for P_m, derivative from
 * P'_m = m (x P_m - P_{m-1}) / (x^2 - 1), weight 2 / ((1-x^2) P'_m^2)). */
static void gauss_legendre(int m, double* node, double* weight) {
  for (int i = 0; i < m; ++i) {
    double x = cos(M_PI * (i + 0.75) / (m + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < m; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = m * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    node[i] = x;
    weight[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

/* B_n from the normalisation 4 pi B_n int_0^2 S_n(pi v/2) v^2 dv = 1 (the
 * kernel integrates to one over 3-D space; the paper names B_n but prints no
 * value).  Composite Gauss-Legendre, 16 panels x 24 nodes on [0,2]. */
double oracle_kernel_norm(double sinc_n) {
  enum { PANELS = 16, NODES = 24 };
  double node[NODES], weight[NODES];
  gauss_legendre(NODES, node, weight);
  double integral = 0.0;
  for (int p = 0; p < PANELS; ++p) {
    double a = 2.0 * p / PANELS, b = 2.0 * (p + 1) / PANELS;
    double half = 0.5 * (b - a), mid = 0.5 * (a + b);
    for (int i = 0; i < NODES; ++i) {
      double v = mid + half * node[i];
      integral += half * weight[i] * pow(sinc_half_pi(v), sinc_n) * v * v;
    }
  }
  return 1.0 / (4.0 * M_PI * integral);
}

/* W(v, h) of Eq. 6, d = 3. */
double oracle_kernel_W(double v, double h, double sinc_n, double Bn) {
  if (v < 0.0 || v > 2.0) return 0.0;
  return Bn / (h * h * h) * pow(sinc_half_pi(v), sinc_n);
}

/* ------------------------------------------------------------------------- */
/* Lookup-table kernel (section 4.5: 20,000 precomputed kernel values and a   */
/* linear interpolation in the relative distance v instead of sin and pow).   */
/* Reading: nodes v_i = 2 i / (N - 1), i = 0..N-1, values T_i = S(v_i)^n;     */
/* for 0 <= v <= 2, with q = v (N - 1) / 2, i = min(floor(q), N - 2) and      */
/* f = q - i:  W = B_n / h^3 (T_i + (T_{i+1} - T_i) f).                       */
/* The mode is process-wide: oracle_set_kernel_mode(1) builds the table for  */
/* the given n and makes every kernel evaluation below use it; mode 0 (the   */
/* default) is the exact kernel.  The Python wrapper sets it before each     */
/* call from its parameters.                                                 */
/* ------------------------------------------------------------------------- */
#define ORACLE_TABLE_N 20000
static int g_kernel_mode = 0;
static double g_table_n = -1.0;
static double g_table[ORACLE_TABLE_N];

void oracle_set_kernel_mode(int mode, double sinc_n) {
  g_kernel_mode = mode;
  if (mode == 1 && g_table_n != sinc_n) {
    for (int i = 0; i < ORACLE_TABLE_N; ++i)
      g_table[i] = pow(sinc_half_pi(2.0 * i / (ORACLE_TABLE_N - 1)), sinc_n);
    g_table_n = sinc_n;
  }
}

int oracle_kernel_mode(void) { return g_kernel_mode; }

/* The kernel used by the sums: W of Eq. 6, or its tabulated form. */
static double kernel_value(double v, double h, double sinc_n, double Bn) {
  if (g_kernel_mode != 1) return oracle_kernel_W(v, h, sinc_n, Bn);
  if (v < 0.0 || v > 2.0) return 0.0;
  double q = v * (0.5 * (ORACLE_TABLE_N - 1));
  int i = (int)floor(q);
  if (i > ORACLE_TABLE_N - 2) i = ORACLE_TABLE_N - 2;
  double f = q - i;
  return Bn / (h * h * h) * (g_table[i] + (g_table[i + 1] - g_table[i]) * f);
}

double oracle_kernel_W_table(double v, double h, double sinc_n, double Bn) {
  int saved = g_kernel_mode;
  oracle_set_kernel_mode(1, sinc_n);
  double w = kernel_value(v, h, sinc_n, Bn);
  g_kernel_mode = saved;
  return w;
}

/* dW/dv of Eq. 6 at fixed h: B_n/h^3 n S^(n-1) dS/dv with S = sin(x)/x,
 * x = pi v / 2, dS/dv = (pi/2) (x cos x - sin x) / x^2 (0 at v = 0). */
double oracle_kernel_dWdv(double v, double h, double sinc_n, double Bn) {
  if (v <= 0.0 || v > 2.0) return 0.0;
  double x = 0.5 * M_PI * v;
  double S = sin(x) / x;
  double dS = 0.5 * M_PI * (x * cos(x) - sin(x)) / (x * x);
  return Bn / (h * h * h) * sinc_n * pow(S, sinc_n - 1.0) * dS;
}

/* dW/dh at fixed separation r, v = r / h: W = B_n h^-3 f(v) gives
 * dW/dh = -(3 W + v dW/dv) / h. */
double oracle_kernel_dWdh(double v, double h, double sinc_n, double Bn) {
  if (v < 0.0 || v > 2.0) return 0.0;
  return -(3.0 * oracle_kernel_W(v, h, sinc_n, Bn) + v * oracle_kernel_dWdv(v, h, sinc_n, Bn)) / h;
}

/* ------------------------------------------------------------------------- */
/* Pair separation and the neighbour criterion (section 4.1: b runs over the  */
/* neighbours of a; the kernel's support is v <= 2 with v = r / h_a).         */
/* Reading: b is a neighbour of a iff b != a and r_ab^2 < (2 h_a)^2 (strict), */
/* with the minimum image on periodic axes computed as below, and r^2 summed  */
/* in the order (dx*dx + dy*dy) + dz*dz with no fused multiply-add.           */
/* ------------------------------------------------------------------------- */

/* Component b - a along one axis, minimum image on periodic axes. */
static double sep(const oracle_box* box, int axis, double xa, double xb) {
  double d = xb - xa;
  if (box->periodic[axis]) {
    double L = box->hi[axis] - box->lo[axis];
    if (d > 0.5 * L)
      d -= L;
    else if (d < -0.5 * L)
      d += L;
  }
  return d;
}

static int is_neighbor(const oracle_box* box, const double* x, const double* y, const double* z,
                       const double* h, int64_t a, int64_t b) {
  if (a == b) return 0;
  double dx = sep(box, 0, x[a], x[b]);
  double dy = sep(box, 1, y[a], y[b]);
  double dz = sep(box, 2, z[a], z[b]);
  double r2 = (dx * dx + dy * dy) + dz * dz;
  double two_h = 2.0 * h[a];
  return r2 < two_h * two_h;
}

static int cmp_i64(const void* p, const void* q) {
  int64_t a = *(const int64_t*)p, b = *(const int64_t*)q;
  return (a > b) - (a < b);
}

/* Neighbour lists.  brute != 0: every pair is tested (O(n^2)).  brute == 0:
 * a uniform cell grid of side >= 2 h_max per axis; each distinct cell of the
 * 3x3x3 stencil is visited once (periodic wrap on periodic axes, clipped on
 * open ones); candidates are tested with the same criterion and each list is
 * sorted ascending.  nn[t] always receives the true count; entries beyond
 * max_nb are dropped and ORACLE_NB_OVERFLOW is returned. */
int oracle_find_neighbors(const oracle_box* box, int64_t n, const double* x, const double* y,
                          const double* z, const double* h, int64_t nt, const int64_t* targets,
                          int brute, int max_nb, int32_t* nn, int64_t* nbr) {
  if (n < 0 || nt < 0 || max_nb < 0) return ORACLE_INVALID_ARG;
  if (nt == 0) return ORACLE_OK;
  double hmax = 0.0;
  for (int64_t i = 0; i < n; ++i) hmax = h[i] > hmax ? h[i] : hmax;
  for (int ax = 0; ax < 3; ++ax)
    if (box->periodic[ax] && !(2.0 * hmax < 0.5 * (box->hi[ax] - box->lo[ax]))) return ORACLE_INVALID_ARG;

  int overflow = 0;
  if (brute) {
#pragma omp parallel for schedule(dynamic, 64) reduction(| : overflow)
    for (int64_t t = 0; t < nt; ++t) {
      int64_t a = targets ? targets[t] : t;
      int cnt = 0;
      for (int64_t b = 0; b < n; ++b) {
        if (is_neighbor(box, x, y, z, h, a, b)) {
          if (cnt < max_nb) nbr[t * max_nb + cnt] = b;
          ++cnt;
        }
      }
      nn[t] = cnt;
      if (cnt > max_nb) overflow = 1;
    }
    return overflow ? ORACLE_NB_OVERFLOW : ORACLE_OK;
  }

  /* cell grid */
  double lo[3], cs[3];
  int nc[3];
  double* pos[3] = {(double*)x, (double*)y, (double*)z};
  for (int ax = 0; ax < 3; ++ax) {
    double a = box->lo[ax], b = box->hi[ax];
    if (!box->periodic[ax]) {
      a = pos[ax][0];
      b = pos[ax][0];
      for (int64_t i = 1; i < n; ++i) {
        a = pos[ax][i] < a ? pos[ax][i] : a;
        b = pos[ax][i] > b ? pos[ax][i] : b;
      }
    }
    double L = b - a;
    int c = (hmax > 0.0) ? (int)floor(L / (2.0 * hmax)) : 1;
    if (c < 1) c = 1;
    if (c > 512) c = 512;
    lo[ax] = a;
    nc[ax] = c;
    cs[ax] = L / c;
  }
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t* cell_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!cell_of || !head || !order) {
    free(cell_of);
    free(head);
    free(order);
    return ORACLE_INVALID_ARG;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t c3[3];
    for (int ax = 0; ax < 3; ++ax) {
      int64_t c = cs[ax] > 0.0 ? (int64_t)floor((pos[ax][i] - lo[ax]) / cs[ax]) : 0;
      if (c < 0) c = 0;
      if (c >= nc[ax]) c = nc[ax] - 1;
      c3[ax] = c;
    }
    cell_of[i] = c3[0] + (int64_t)nc[0] * (c3[1] + (int64_t)nc[1] * c3[2]);
  }
  /* counting sort of particle indices by cell (stable) */
  memset(head, 0, sizeof(int64_t) * (size_t)(ncell + 1));
  for (int64_t i = 0; i < n; ++i) head[cell_of[i] + 1]++;
  for (int64_t c = 0; c < ncell; ++c) head[c + 1] += head[c];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, head, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) order[fill[cell_of[i]]++] = i;
    free(fill);
  }

#pragma omp parallel for schedule(dynamic, 64) reduction(| : overflow)
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = targets ? targets[t] : t;
    int64_t ca = cell_of[a];
    int64_t c3[3] = {ca % nc[0], (ca / nc[0]) % nc[1], ca / ((int64_t)nc[0] * nc[1])};
    int64_t visited[27];
    int nvis = 0;
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int64_t q[3] = {c3[0] + dx, c3[1] + dy, c3[2] + dz};
          int ok = 1;
          for (int ax = 0; ax < 3; ++ax) {
            if (q[ax] < 0 || q[ax] >= nc[ax]) {
              if (box->periodic[ax])
                q[ax] = (q[ax] + nc[ax]) % nc[ax];
              else
                ok = 0;
            }
          }
          if (!ok) continue;
          int64_t cb = q[0] + (int64_t)nc[0] * (q[1] + (int64_t)nc[1] * q[2]);
          int seen = 0;
          for (int v = 0; v < nvis; ++v) seen |= (visited[v] == cb);
          if (seen) continue;
          visited[nvis++] = cb;
          for (int64_t s = head[cb]; s < head[cb + 1]; ++s) {
            int64_t b = order[s];
            if (is_neighbor(box, x, y, z, h, a, b)) {
              if (cnt < max_nb) nbr[t * max_nb + cnt] = b;
              ++cnt;
            }
          }
        }
    nn[t] = cnt;
    if (cnt > max_nb) overflow = 1;
    qsort(nbr + t * max_nb, (size_t)(cnt < max_nb ? cnt : max_nb), sizeof(int64_t), cmp_i64);
  }
  free(cell_of);
  free(head);
  free(order);
  return overflow ? ORACLE_NB_OVERFLOW : ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Density, section 4.1 Eq. 1:  rho_a = sum_b m_b W_ab(h_a).                  */
/* Reading: the sum includes b = a (the self term m_a W(0, h_a)); without it  */
/* a uniform lattice would come out about a quarter of its true density.      */
/* Equation of state (not printed in the paper): ideal gas,                   */
/*   P = (gamma - 1) rho u,   c = sqrt(gamma P / rho).                        */
/* Grad-h terms (section 4.1 names Omega_a, "the grad-h terms that take into  */
/* account the changes in the local smoothing length", without a formula).   */
/* Reading, the standard definition for h tied to the density (h ~ rho^-1/3, */
/* so dh/drho = -h / (3 rho)) and the same sum as Eq. 1, self term included: */
/*   Omega_a = 1 - (dh_a/drho_a) sum_b m_b dW_ab(h_a)/dh_a                    */
/*           = 1 + h_a / (3 rho_a) sum_b m_b dW_ab(h_a)/dh_a.                 */
/* omega == NULL skips it (Omega = 1 everywhere).                            */
/* ------------------------------------------------------------------------- */
void oracle_density_eos(const oracle_box* box, const double* x, const double* y, const double* z,
                        const double* h, const double* m, const double* u, int64_t nt,
                        const int64_t* targets, const int32_t* nn, const int64_t* nbr, int max_nb,
                        double sinc_n, double Bn, double gamma, double* rho, double* p, double* c,
                        double* omega) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = targets ? targets[t] : t;
    double sum = m[a] * kernel_value(0.0, h[a], sinc_n, Bn);
    double dsum = omega ? m[a] * oracle_kernel_dWdh(0.0, h[a], sinc_n, Bn) : 0.0;
    for (int k = 0; k < nn[t]; ++k) {
      int64_t b = nbr[t * max_nb + k];
      double dx = sep(box, 0, x[a], x[b]), dy = sep(box, 1, y[a], y[b]), dz = sep(box, 2, z[a], z[b]);
      double r = sqrt((dx * dx + dy * dy) + dz * dz);
      sum += m[b] * kernel_value(r / h[a], h[a], sinc_n, Bn);
      if (omega) dsum += m[b] * oracle_kernel_dWdh(r / h[a], h[a], sinc_n, Bn);
    }
    rho[t] = sum;
    p[t] = (gamma - 1.0) * sum * u[a];
    c[t] = sqrt(gamma * p[t] / sum);
    if (omega) omega[t] = 1.0 + h[a] / (3.0 * sum) * dsum;
  }
}

/* ------------------------------------------------------------------------- */
/* Integral approach to derivatives (section 4.1 cites IAD for the terms      */
/* A_{i,ab}(h); the formula is not printed).  Reading, the method's standard  */
/* definition:                                                                */
/*   tau_a   = sum_b (m_b / rho_b) (x_b - x_a)(x_b - x_a)^T W_ab(h_a)         */
/*   C_a     = tau_a^{-1}                                                     */
/*   A_ab(h) = C (x_b - x_a) W_ab(h)  with C the matrix of the particle whose */
/*             h is used.                                                     */
/* C is returned as its 6 unique entries (xx, xy, xz, yy, yz, zz).  The       */
/* inverse is by cofactors over the determinant; |det| <= 1e-12 * max|tau|^3  */
/* (or a non-finite det) marks tau singular: C is set to zero and the return  */
/* code is ORACLE_SINGULAR_IAD.                                               */
/* ------------------------------------------------------------------------- */
int oracle_iad(const oracle_box* box, const double* x, const double* y, const double* z,
               const double* h, const double* m, const double* rho, int64_t nt,
               const int64_t* targets, const int32_t* nn, const int64_t* nbr, int max_nb,
               double sinc_n, double Bn, double* iad, double* tau_out) {
  int singular = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : singular)
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = targets ? targets[t] : t;
    double T[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < nn[t]; ++k) {
      int64_t b = nbr[t * max_nb + k];
      double d[3] = {sep(box, 0, x[a], x[b]), sep(box, 1, y[a], y[b]), sep(box, 2, z[a], z[b])};
      double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      double w = m[b] / rho[b] * kernel_value(r / h[a], h[a], sinc_n, Bn);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] += w * d[i] * d[j];
    }
    double cof[3][3];
    cof[0][0] = T[1][1] * T[2][2] - T[1][2] * T[2][1];
    cof[0][1] = -(T[1][0] * T[2][2] - T[1][2] * T[2][0]);
    cof[0][2] = T[1][0] * T[2][1] - T[1][1] * T[2][0];
    cof[1][0] = -(T[0][1] * T[2][2] - T[0][2] * T[2][1]);
    cof[1][1] = T[0][0] * T[2][2] - T[0][2] * T[2][0];
    cof[1][2] = -(T[0][0] * T[2][1] - T[0][1] * T[2][0]);
    cof[2][0] = T[0][1] * T[1][2] - T[0][2] * T[1][1];
    cof[2][1] = -(T[0][0] * T[1][2] - T[0][2] * T[1][0]);
    cof[2][2] = T[0][0] * T[1][1] - T[0][1] * T[1][0];
    double det = T[0][0] * cof[0][0] + T[0][1] * cof[0][1] + T[0][2] * cof[0][2];
    double tmax = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) tmax = fabs(T[i][j]) > tmax ? fabs(T[i][j]) : tmax;
    double Cm[3][3];
    if (!isfinite(det) || fabs(det) <= 1e-12 * tmax * tmax * tmax) {
      singular = 1;
      memset(Cm, 0, sizeof(Cm));
    } else {
      /* inverse = adjugate / det; adjugate = transpose of the cofactor matrix */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Cm[i][j] = cof[j][i] / det;
    }
    double* o = iad + 6 * t;
    o[0] = Cm[0][0];
    o[1] = Cm[0][1];
    o[2] = Cm[0][2];
    o[3] = Cm[1][1];
    o[4] = Cm[1][2];
    o[5] = Cm[2][2];
    if (tau_out) {
      double* q = tau_out + 6 * t;
      q[0] = T[0][0];
      q[1] = T[0][1];
      q[2] = T[0][2];
      q[3] = T[1][1];
      q[4] = T[1][2];
      q[5] = T[2][2];
    }
  }
  return singular ? ORACLE_SINGULAR_IAD : ORACLE_OK;
}

/* 3x3 symmetric C (6 unique entries) times vector d. */
static void sym_mul(const double* C6, const double* d, double* out) {
  out[0] = C6[0] * d[0] + C6[1] * d[1] + C6[2] * d[2];
  out[1] = C6[1] * d[0] + C6[3] * d[1] + C6[4] * d[2];
  out[2] = C6[2] * d[0] + C6[4] * d[1] + C6[5] * d[2];
}

/* ------------------------------------------------------------------------- */
/* Momentum and energy with IAD and artificial viscosity, section 4.1         */
/* Eqs. 2-5, with Omega_a = 1 (the grad-h terms are named but not defined).   */
/* With x_ab = x_a - x_b, v_ab = v_a - v_b, r = |x_ab|, d = x_b - x_a:        */
/*   A_a = A_ab(h_a) = C_a d W(r/h_a, h_a),  A_b = A_ab(h_b) = C_b d W(r/h_b,h_b) */
/*   X_a = P_a / rho_a^2                                                      */
/*   w_ab = v_ab . x_ab / r (0 when r = 0),  v_sig = c_a + c_b - 3 w_ab       */
/*   Pi_ab = -(alpha/2) v_sig w_ab if x_ab . v_ab < 0, else 0       (Eq. 5)   */
/*   Abar = A_a / rho_a + A_b / rho_b                                          */
/*   dv_a/dt = -sum_b m_b (X_a A_a + X_b A_b) - 1/2 sum_b m_b Pi_ab Abar       */
/*   du_a/dt =  X_a sum_b m_b v_ab . A_a + 1/4 sum_b m_b Pi_ab v_ab . Abar     */
/* With the grad-h terms (omega != NULL) X_a = P_a / (Omega_a rho_a^2), as    */
/* printed in Eqs. 2-3; the viscous terms carry no Omega (Eq. 4).             */
/* Readings of two garbled points: the energy prefactor of Eq. 3 is taken as  */
/* P_a/(Omega_a rho_a^2) (the dimensionally consistent form, and the one that */
/* makes the pair exchange conserve energy), and the viscous acceleration of  */
/* Eq. 4 enters with a minus sign (with A pointing from a to b, the printed   */
/* plus sign would accelerate approaching particles toward each other).  The  */
/* viscous energy term is Eq. 3's 1/2 sum_b v_ab . a^AV with a^AV the pair    */
/* term of the corrected Eq. 4.                                               */
/* Outputs per target: a (3), du, and the normalisation scales sa and sdu:   */
/* the pair terms with every factor in magnitude (|X| |A|, |Pi| |Abar|,       */
/* |v_ab| |A|), the scale of the rounding error of the sums.                  */
/* The viscosity switch of Eq. 5 (x_ab . v_ab < 0) can be recorded per list   */
/* entry (av_out[t*max_nb+k] = 1 where it is on) and imposed instead of       */
/* decided (av_force, same layout): a rollout with its lists frozen is then a */
/* smooth function of its inputs, which central differences need.  Both NULL */
/* means the switch is decided from the sign, as printed.                     */
/* ------------------------------------------------------------------------- */
void oracle_momentum_energy(const oracle_box* box, const double* x, const double* y,
                            const double* z, const double* vx, const double* vy, const double* vz,
                            const double* h, const double* m, const double* rho, const double* p,
                            const double* c, const double* iad, const double* omega, int64_t nt,
                            const int64_t* targets,
                            const int32_t* nn, const int64_t* nbr, int max_nb, double sinc_n,
                            double Bn, double alpha, const int8_t* av_force, int8_t* av_out,
                            double* ax, double* ay, double* az, double* du, double* sa,
                            double* sdu) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = targets ? targets[t] : t;
    double acc[3] = {0, 0, 0}, energy = 0.0, sacc = 0.0, sen = 0.0;
    double Xa = p[a] / ((omega ? omega[a] : 1.0) * rho[a] * rho[a]);
    for (int k = 0; k < nn[t]; ++k) {
      int64_t b = nbr[t * max_nb + k];
      double d[3] = {sep(box, 0, x[a], x[b]), sep(box, 1, y[a], y[b]), sep(box, 2, z[a], z[b])};
      double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      double Wa = kernel_value(r / h[a], h[a], sinc_n, Bn);
      double Wb = kernel_value(r / h[b], h[b], sinc_n, Bn);
      double Ca_d[3], Cb_d[3], Aa[3], Ab[3];
      sym_mul(iad + 6 * a, d, Ca_d);
      sym_mul(iad + 6 * b, d, Cb_d);
      for (int i = 0; i < 3; ++i) {
        Aa[i] = Ca_d[i] * Wa;
        Ab[i] = Cb_d[i] * Wb;
      }
      double xab[3] = {-d[0], -d[1], -d[2]};
      double vab[3] = {vx[a] - vx[b], vy[a] - vy[b], vz[a] - vz[b]};
      double xv = xab[0] * vab[0] + xab[1] * vab[1] + xab[2] * vab[2];
      double w = r > 0.0 ? xv / r : 0.0;
      double vsig = c[a] + c[b] - 3.0 * w;
      int on = av_force ? av_force[t * max_nb + k] != 0 : xv < 0.0;
      if (av_out) av_out[t * max_nb + k] = (int8_t)on;
      double Pi = on ? -0.5 * alpha * vsig * w : 0.0;
      double Xb = p[b] / ((omega ? omega[b] : 1.0) * rho[b] * rho[b]);
      double Abar[3];
      for (int i = 0; i < 3; ++i) Abar[i] = Aa[i] / rho[a] + Ab[i] / rho[b];
      double term[3];
      for (int i = 0; i < 3; ++i) term[i] = -m[b] * (Xa * Aa[i] + Xb * Ab[i]) - 0.5 * m[b] * Pi * Abar[i];
      double vA = vab[0] * Aa[0] + vab[1] * Aa[1] + vab[2] * Aa[2];
      double vAbar = vab[0] * Abar[0] + vab[1] * Abar[1] + vab[2] * Abar[2];
      double eterm = Xa * m[b] * vA + 0.25 * m[b] * Pi * vAbar;
      for (int i = 0; i < 3; ++i) acc[i] += term[i];
      energy += eterm;
      /* error-analysis scales: each product's factors taken in magnitude, so
       * that cancellation inside a dot product does not shrink the scale */
      double nAa = sqrt(Aa[0] * Aa[0] + Aa[1] * Aa[1] + Aa[2] * Aa[2]);
      double nAb = sqrt(Ab[0] * Ab[0] + Ab[1] * Ab[1] + Ab[2] * Ab[2]);
      double nv = sqrt(vab[0] * vab[0] + vab[1] * vab[1] + vab[2] * vab[2]);
      double nAbar = nAa / rho[a] + nAb / rho[b];
      sacc += m[b] * (fabs(Xa) * nAa + fabs(Xb) * nAb) + 0.5 * m[b] * fabs(Pi) * nAbar;
      sen += m[b] * fabs(Xa) * nv * nAa + 0.25 * m[b] * fabs(Pi) * nv * nAbar;
    }
    ax[t] = acc[0];
    ay[t] = acc[1];
    az[t] = acc[2];
    du[t] = energy;
    if (sa) sa[t] = sacc;
    if (sdu) sdu[t] = sen;
  }
}

/* ------------------------------------------------------------------------- */
/* Time step (section 4.2: a global minimum time step, formula not printed).  */
/* Reading: Courant condition  dt_c = courant * min_a h_a / c_a, capped by    */
/* growth:  dt = min(dt_c, dt_growth * dt_prev) when dt_prev > 0.             */
/* ------------------------------------------------------------------------- */
double oracle_timestep(int64_t n, const double* h, const double* c, double courant,
                       double dt_growth, double dt_prev) {
  double mn = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double q = h[i] / c[i];
    mn = q < mn ? q : mn;
  }
  double dt = courant * mn;
  if (dt_prev > 0.0) {
    double cap = dt_growth * dt_prev;
    dt = cap < dt ? cap : dt;
  }
  return dt;
}

/* Reading (opt-in, energy_dt > 0): the step is also limited by the rate of    */
/* change of the internal energy, dt <= energy_dt * min_a u_a / |du_a| over   */
/* the particles with du_a != 0, so that one forward-Euler step changes no u   */
/* by more than the fraction energy_dt of itself.  Applied before the growth  */
/* cap; energy_dt = 0 gives oracle_timestep.                                 */
double oracle_timestep_u(int64_t n, const double* h, const double* c, const double* u,
                         const double* du, double courant, double energy_dt, double dt_growth,
                         double dt_prev) {
  double mn = INFINITY, mu = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double q = h[i] / c[i];
    mn = q < mn ? q : mn;
    if (energy_dt > 0.0 && du[i] != 0.0) {
      double r = u[i] / fabs(du[i]);
      mu = r < mu ? r : mu;
    }
  }
  double dt = courant * mn;
  if (energy_dt > 0.0) {
    double du_lim = energy_dt * mu;
    dt = du_lim < dt ? du_lim : dt;
  }
  if (dt_prev > 0.0) {
    double cap = dt_growth * dt_prev;
    dt = cap < dt ? cap : dt;
  }
  return dt;
}

/* ------------------------------------------------------------------------- */
/* Update (section 4.1: positions and velocities by a second-order Press     */
/* method, energy by second-order Adams-Bashforth; no formulas printed).      */
/* Reading: velocity-Verlet style leapfrog with variable step, one force      */
/* evaluation per step:                                                       */
/*   Delta = (dt + dt_prev) / 2                                               */
/*   vh   <- vh + a Delta                    (v^{n+1/2})                      */
/*   x    <- x + dt vh, wrapped into [lo, hi) on periodic axes                */
/*   v    <- vh + (dt / 2) a                 (predicted v^{n+1})              */
/*   u    <- u + dt [(1 + dt/(2 dt_prev)) du - dt/(2 dt_prev) du_prev]        */
/*           (forward Euler when dt_prev = 0)                                 */
/*   du_prev <- du                                                            */
/* Smoothing length (toward a target neighbour count n_t, rule not printed):  */
/*   h <- h * (1 + (n_t / max(nn, 1))^(1/3)) / 2   when n_t > 0.              */
/* ------------------------------------------------------------------------- */
void oracle_update(const oracle_box* box, int64_t n, double* x, double* y, double* z, double* vx,
                   double* vy, double* vz, double* vxh, double* vyh, double* vzh, double* u,
                   double* du_prev, double* h, const double* ax, const double* ay,
                   const double* az, const double* du, const int32_t* nn, double dt,
                   double dt_prev, int ng_target) {
  double delta = 0.5 * (dt + dt_prev);
  double* pos[3] = {x, y, z};
  double* vel[3] = {vx, vy, vz};
  double* velh[3] = {vxh, vyh, vzh};
  const double* acc[3] = {ax, ay, az};
  for (int64_t i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) {
      velh[d][i] = velh[d][i] + acc[d][i] * delta;
      double xn = pos[d][i] + dt * velh[d][i];
      if (box->periodic[d]) {
        double L = box->hi[d] - box->lo[d];
        if (xn >= box->hi[d])
          xn -= L;
        else if (xn < box->lo[d])
          xn += L;
      }
      pos[d][i] = xn;
      vel[d][i] = velh[d][i] + 0.5 * dt * acc[d][i];
    }
    if (dt_prev > 0.0) {
      double q = dt / (2.0 * dt_prev);
      u[i] = u[i] + dt * ((1.0 + q) * du[i] - q * du_prev[i]);
    } else {
      u[i] = u[i] + dt * du[i];
    }
    du_prev[i] = du[i];
    if (ng_target > 0) {
      int k = nn[i] > 1 ? nn[i] : 1;
      h[i] = h[i] * 0.5 * (1.0 + cbrt((double)ng_target / (double)k));
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Conservation sums (section 4.2: total momentum and energy are reduced to   */
/* check that they are conserved).  Compensated (Kahan) FP64 sums.            */
/*   out = {Px, Py, Pz, E_kin, E_int, Lx, Ly, Lz}                             */
/*   P = sum m v,  E_kin = sum m |v|^2 / 2,  E_int = sum m u,  L = sum m x x v */
/* ------------------------------------------------------------------------- */
void oracle_diagnostics(int64_t n, const double* x, const double* y, const double* z,
                        const double* vx, const double* vy, const double* vz, const double* m,
                        const double* u, double* out) {
  double s[8] = {0}, comp[8] = {0};
  for (int64_t i = 0; i < n; ++i) {
    double term[8];
    term[0] = m[i] * vx[i];
    term[1] = m[i] * vy[i];
    term[2] = m[i] * vz[i];
    term[3] = 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
    term[4] = m[i] * u[i];
    term[5] = m[i] * (y[i] * vz[i] - z[i] * vy[i]);
    term[6] = m[i] * (z[i] * vx[i] - x[i] * vz[i]);
    term[7] = m[i] * (x[i] * vy[i] - y[i] * vx[i]);
    for (int k = 0; k < 8; ++k) {
      double yk = term[k] - comp[k];
      double tk = s[k] + yk;
      comp[k] = (tk - s[k]) - yk;
      s[k] = tk;
    }
  }
  for (int k = 0; k < 8; ++k) out[k] = s[k];
}

/* Threads the per-particle loops use (the OpenMP default of this process). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the thread count of the per-particle loops (results do not depend on
 * it); returns the count now in effect. */
int oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
  return oracle_num_threads();
}

/* Non-finite scan helper: returns 1 if any of the n values is NaN or inf. */
int oracle_any_nonfinite(int64_t n, const double* v) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 1;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Self-gravity (section 4.1: a multipolar expansion evaluated on the tree    */
/* used to find neighbours; no formula is printed).  Reading:                 */
/*   g_a = -G sum_{b != a} m_b (x_a - x_b) / (|x_a - x_b|^2 + eps^2)^(3/2)    */
/* (Newtonian gravity with Plummer softening eps, open boundaries), which    */
/* oracle_gravity_direct evaluates exactly, and its tree approximation       */
/* oracle_gravity_tree:                                                      */
/*  - leaves: the cells of the neighbour grid on open axes (per axis lo =    */
/*    min x, L = extent, nc = min(floor(L / (2 h_max (1 + 1e-9))), 256) and  */
/*    at least 1, cs = L / nc, cell = floor((x - lo) * (1 / cs)) clamped),   */
/*    keyed by the Morton code of the cell (bit i of the x cell at 3i, y at  */
/*    3i+1, z at 3i+2; bits = ceil(log2(max nc)) per axis);                  */
/*  - node at level l (0 = root, bits = leaves): the cells sharing the top   */
/*    3 l bits of the code; its box is those cells' union, its size s the   */
/*    box's longest side; its moments (about its centre of mass c) are the   */
/*    mass M and the traceless quadrupole Q_ij = sum m (3 d_i d_j - |d|^2   */
/*    delta_ij), d = x - c;                                                  */
/*  - for target a, depth-first from the root with children in Morton order: */
/*    a node whose box does not contain x_a and with s / |x_a - c| < theta   */
/*    adds, with r = x_a - c, R = |r|:                                       */
/*      -G M r / (R^2 + eps^2)^(3/2) + G Q r / R^5 - (5/2) G (r.Q.r) r / R^7  */
/*    (the gradient of -G (M/R + r.Q.r / (2 R^5)), the monopole softened);    */
/*    an opened leaf adds its particles by the direct formula; other nodes   */
/*    open their children.                                                   */
/* ------------------------------------------------------------------------- */
void oracle_gravity_direct(int64_t n, const double* x, const double* y, const double* z,
                           const double* m, double G, double eps, int64_t nt,
                           const int64_t* targets, double* gx, double* gy, double* gz) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = targets ? targets[t] : t;
    double s[3] = {0, 0, 0};
    for (int64_t b = 0; b < n; ++b) {
      if (b == a) continue;
      double d[3] = {x[a] - x[b], y[a] - y[b], z[a] - z[b]};
      double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] + eps * eps;
      double f = m[b] / (r2 * sqrt(r2));
      for (int k = 0; k < 3; ++k) s[k] -= G * f * d[k];
    }
    gx[t] = s[0];
    gy[t] = s[1];
    gz[t] = s[2];
  }
}

typedef struct {
  uint32_t code;     /* Morton prefix */
  int level;
  int64_t first;     /* first child (index into the node array), or -1 for a leaf */
  int nchild;
  int64_t p0, np;    /* particles of the node: order[p0 .. p0 + np) */
  double box_lo[3], box_hi[3], size;
  double M, c[3], Q[6];   /* xx xy xz yy yz zz */
} oracle_node;

static uint32_t spread_bits(uint32_t v) {
  uint32_t r = 0;
  for (int i = 0; i < 10; ++i) r |= ((v >> i) & 1u) << (3 * i);
  return r;
}

typedef struct {
  uint32_t code;
  int64_t index;
} code_index;

static int cmp_code_index(const void* p, const void* q) {
  const code_index* a = (const code_index*)p;
  const code_index* b = (const code_index*)q;
  if (a->code != b->code) return a->code < b->code ? -1 : 1;
  return (a->index > b->index) - (a->index < b->index);
}

static void node_moments(oracle_node* nd, const int64_t* order, const double* x, const double* y,
                         const double* z, const double* m) {
  double M = 0, s[3] = {0, 0, 0};
  for (int64_t i = nd->p0; i < nd->p0 + nd->np; ++i) {
    int64_t b = order[i];
    M += m[b];
    s[0] += m[b] * x[b];
    s[1] += m[b] * y[b];
    s[2] += m[b] * z[b];
  }
  nd->M = M;
  for (int k = 0; k < 3; ++k) nd->c[k] = s[k] / M;
  double Q[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = nd->p0; i < nd->p0 + nd->np; ++i) {
    int64_t b = order[i];
    double d[3] = {x[b] - nd->c[0], y[b] - nd->c[1], z[b] - nd->c[2]};
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    Q[0] += m[b] * (3 * d[0] * d[0] - d2);
    Q[1] += m[b] * (3 * d[0] * d[1]);
    Q[2] += m[b] * (3 * d[0] * d[2]);
    Q[3] += m[b] * (3 * d[1] * d[1] - d2);
    Q[4] += m[b] * (3 * d[1] * d[2]);
    Q[5] += m[b] * (3 * d[2] * d[2] - d2);
  }
  memcpy(nd->Q, Q, sizeof(Q));
}

static void tree_walk(const oracle_node* nodes, int64_t k, const int64_t* order, const double* x,
                      const double* y, const double* z, const double* m, int64_t a, double G,
                      double eps, double theta, double* acc, int64_t* counts) {
  const oracle_node* nd = &nodes[k];
  double p[3] = {x[a], y[a], z[a]};
  int inside = 1;
  for (int ax = 0; ax < 3; ++ax)
    if (p[ax] < nd->box_lo[ax] || p[ax] > nd->box_hi[ax]) inside = 0;
  double r[3] = {p[0] - nd->c[0], p[1] - nd->c[1], p[2] - nd->c[2]};
  double R2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
  double R = sqrt(R2);
  if (!inside && nd->size < theta * R) {
    double s2 = R2 + eps * eps;
    double mono = G * nd->M / (s2 * sqrt(s2));
    const double* Q = nd->Q;
    double Qr[3] = {Q[0] * r[0] + Q[1] * r[1] + Q[2] * r[2],
                    Q[1] * r[0] + Q[3] * r[1] + Q[4] * r[2],
                    Q[2] * r[0] + Q[4] * r[1] + Q[5] * r[2]};
    double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
    double R5 = R2 * R2 * R;
    double R7 = R5 * R2;
    for (int i = 0; i < 3; ++i)
      acc[i] += -mono * r[i] + G * Qr[i] / R5 - 2.5 * G * rQr * r[i] / R7;
    counts[0] += 1;
    return;
  }
  if (nd->first < 0) {
    for (int64_t i = nd->p0; i < nd->p0 + nd->np; ++i) {
      int64_t b = order[i];
      if (b == a) continue;
      double d[3] = {p[0] - x[b], p[1] - y[b], p[2] - z[b]};
      double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] + eps * eps;
      double f = m[b] / (r2 * sqrt(r2));
      for (int q = 0; q < 3; ++q) acc[q] -= G * f * d[q];
      counts[1] += 1;
    }
    return;
  }
  for (int j = 0; j < nd->nchild; ++j)
    tree_walk(nodes, nd->first + j, order, x, y, z, m, a, G, eps, theta, acc, counts);
}

/* Returns ORACLE_OK, or ORACLE_INVALID_ARG (n < 1, or no positive h).
 * stats (optional, 2 values): node and particle interactions summed over the
 * targets. */
int oracle_gravity_tree(int64_t n, const double* x, const double* y, const double* z,
                        const double* h, const double* m, double G, double eps, double theta,
                        int64_t nt, const int64_t* targets, double* gx, double* gy, double* gz,
                        int64_t* stats) {
  if (n < 1) return ORACLE_INVALID_ARG;
  const double* pos[3] = {x, y, z};
  double lo[3], L[3], cs[3], inv[3], hmax = 0.0;
  int nc[3], maxnc = 1;
  for (int64_t i = 0; i < n; ++i) hmax = h[i] > hmax ? h[i] : hmax;
  if (!(hmax > 0.0)) return ORACLE_INVALID_ARG;
  for (int ax = 0; ax < 3; ++ax) {
    double mn = pos[ax][0], mx = pos[ax][0];
    for (int64_t i = 1; i < n; ++i) {
      mn = pos[ax][i] < mn ? pos[ax][i] : mn;
      mx = pos[ax][i] > mx ? pos[ax][i] : mx;
    }
    lo[ax] = mn;
    L[ax] = mx - mn;
    int c = 1;
    if (L[ax] > 0.0) {
      double q = floor(L[ax] / (2.0 * hmax * (1.0 + 1e-9)));
      c = q < 1.0 ? 1 : (q > 256.0 ? 256 : (int)q);
    }
    nc[ax] = c;
    cs[ax] = L[ax] > 0.0 ? L[ax] / c : 0.0;
    inv[ax] = cs[ax] > 0.0 ? 1.0 / cs[ax] : 0.0;
    maxnc = c > maxnc ? c : maxnc;
  }
  int bits = 0;
  while ((1 << bits) < maxnc) ++bits;
  code_index* ci = (code_index*)malloc(sizeof(code_index) * (size_t)n);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    uint32_t cell[3];
    for (int ax = 0; ax < 3; ++ax) {
      double q = floor((pos[ax][i] - lo[ax]) * inv[ax]);
      int v = q < 0.0 ? 0 : (q >= (double)nc[ax] ? nc[ax] - 1 : (int)q);
      cell[ax] = (uint32_t)v;
    }
    ci[i].code = spread_bits(cell[0]) | (spread_bits(cell[1]) << 1) | (spread_bits(cell[2]) << 2);
    ci[i].index = i;
  }
  qsort(ci, (size_t)n, sizeof(code_index), cmp_code_index);
  for (int64_t i = 0; i < n; ++i) order[i] = ci[i].index;
  /* nodes level by level from the leaves up: a node = a run of equal prefixes */
  int64_t cap = (int64_t)(bits + 1) * n + 1, nn = 0;
  oracle_node* nodes = (oracle_node*)calloc((size_t)cap, sizeof(oracle_node));
  int64_t* level_start = (int64_t*)malloc(sizeof(int64_t) * (bits + 2));
  /* leaves */
  level_start[bits] = 0;
  for (int64_t i = 0; i < n;) {
    int64_t j = i;
    while (j < n && ci[j].code == ci[i].code) ++j;
    oracle_node* nd = &nodes[nn++];
    nd->code = ci[i].code;
    nd->level = bits;
    nd->first = -1;
    nd->p0 = i;
    nd->np = j - i;
    i = j;
  }
  int64_t prev0 = 0, prev1 = nn;
  for (int l = bits - 1; l >= 0; --l) {
    level_start[l] = nn;
    for (int64_t i = prev0; i < prev1;) {
      uint32_t pc = nodes[i].code >> 3;
      int64_t j = i;
      while (j < prev1 && (nodes[j].code >> 3) == pc) ++j;
      oracle_node* nd = &nodes[nn++];
      nd->code = pc;
      nd->level = l;
      nd->first = i;
      nd->nchild = (int)(j - i);
      nd->p0 = nodes[i].p0;
      nd->np = nodes[j - 1].p0 + nodes[j - 1].np - nodes[i].p0;
      i = j;
    }
    prev0 = level_start[l];
    prev1 = nn;
  }
  /* boxes and moments (each node from its own particles) */
  for (int64_t k = 0; k < nn; ++k) {
    oracle_node* nd = &nodes[k];
    int span = 1 << (bits - nd->level);
    uint32_t c3[3] = {0, 0, 0};
    for (int i = 0; i < 10; ++i)
      for (int ax = 0; ax < 3; ++ax) c3[ax] |= ((nd->code >> (3 * i + ax)) & 1u) << i;
    double size = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
      int c0 = (int)c3[ax] * span, c1 = c0 + span - 1;
      if (c1 > nc[ax] - 1) c1 = nc[ax] - 1;
      nd->box_lo[ax] = lo[ax] + c0 * cs[ax];
      nd->box_hi[ax] = lo[ax] + (c1 + 1) * cs[ax];
      double ext = nd->box_hi[ax] - nd->box_lo[ax];
      size = ext > size ? ext : size;
    }
    nd->size = size;
    node_moments(nd, order, x, y, z, m);
  }
  int64_t root = nn - 1;
  int64_t tot[2] = {0, 0};
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : tot[:2])
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = targets ? targets[t] : t;
    double acc[3] = {0, 0, 0};
    int64_t counts[2] = {0, 0};
    tree_walk(nodes, root, order, x, y, z, m, a, G, eps, theta, acc, counts);
    gx[t] = acc[0];
    gy[t] = acc[1];
    gz[t] = acc[2];
    tot[0] += counts[0];
    tot[1] += counts[1];
  }
  if (stats) {
    stats[0] = tot[0];
    stats[1] = tot[1];
  }
  free(level_start);
  free(nodes);
  free(order);
  free(ci);
  return ORACLE_OK;
}
