// C ABI of libsph (declared in include/sph.h): context management, argument
// checks, scratch allocation and the order of kernel launches of each stage.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sph_device.cuh"
#include "sph_internal.cuh"
#include "sph_tile.cuh"

using sph::OutView;
using sph::StateView;

namespace sph {

int set_error(sph_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->last_error, sizeof(ctx->last_error), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(sph_ctx* ctx, cudaError_t e, const char* what) {
  return set_error(ctx, e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA, "%s: %s",
                   what, cudaGetErrorString(e));
}

}  // namespace sph

namespace {

// B_n of Eq. 6 from 4 pi B_n int_0^2 S(v)^n v^2 dv = 1: composite Simpson rule
// with 2^16 panels and a compensated sum (host, once per context).
double kernel_norm_host(double n) {
  const int N = 1 << 16;
  const double hstep = 2.0 / N;
  auto f = [n](double v) {
    if (v == 0.0) return 0.0;
    const double x = 1.5707963267948966192 * v;
    return pow(sin(x) / x, n) * v * v;
  };
  double s = 0.0, comp = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double w = (i == 0 || i == N) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    const double y = w * f(i * hstep) - comp;
    const double t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  const double integral = s * hstep / 3.0;
  return 1.0 / (4.0 * 3.14159265358979323846 * integral);
}

int check_params(sph_ctx* ctx, const sph_params* p) {
  if (!p) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "params is NULL");
  for (int k = 0; k < 3; ++k) {
    if (p->periodic[k] && !(p->box_hi[k] > p->box_lo[k]))
      return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "periodic axis %d needs box_hi > box_lo", k);
  }
  if (!(p->gamma > 1.0)) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "gamma must be > 1");
  if (!(p->alpha >= 0.0)) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "alpha must be >= 0");
  if (!(p->courant > 0.0)) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "courant must be > 0");
  if (!(p->dt_growth >= 1.0))
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "dt_growth must be >= 1");
  if (p->ng_target < 0) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "ng_target < 0");
  if (p->max_nb < 4 || p->max_nb > 4096 || p->max_nb % 4 != 0)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "max_nb must be a multiple of 4 in [4, 4096]");
  if (!(p->sinc_n >= 1.0 && p->sinc_n <= 12.0) || p->sinc_n != floor(p->sinc_n))
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "sinc_n must be an integer in [1, 12]");
  if (p->precision != SPH_FP64 && p->precision != SPH_FP32_MIXED)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "unknown precision %d", p->precision);
  if (p->kernel_mode != SPH_KERNEL_EXACT && p->kernel_mode != SPH_KERNEL_TABLE)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "unknown kernel_mode %d", p->kernel_mode);
  if (p->gradh != 0 && p->gradh != 1)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "gradh must be 0 or 1");
  if (p->gradh && p->kernel_mode != SPH_KERNEL_EXACT)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "gradh needs SPH_KERNEL_EXACT");
  if (p->pair_mode != SPH_PAIRS_STAGED && p->pair_mode != SPH_PAIRS_LISTS)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "unknown pair_mode %d", p->pair_mode);
  if (!(p->energy_dt >= 0.0) || !isfinite(p->energy_dt))
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "energy_dt must be finite and >= 0");
  if (p->angular_sums != 0 && p->angular_sums != 1)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "angular_sums must be 0 or 1");
  return SPH_OK;
}

// SPH_KERNEL_TABLE: T_i = S(v_i)^n at v_i = 2 i / (N - 1) with libm sin and
// pow on the host (section 4.5), stored as (T_i, T_{i+1} - T_i) in FP64 and
// FP32; rebuilt when sinc_n changes.
int build_kernel_table(sph_ctx* ctx) {
  if (ctx->prm.kernel_mode != SPH_KERNEL_TABLE || ctx->ktab_n == ctx->prm.sinc_n) return SPH_OK;
  const int N = sph::kKernelTableN;
  cudaError_t e = cudaSuccess;
  if (!ctx->ktab64) e = cudaMalloc((void**)&ctx->ktab64, sizeof(double2) * N);
  if (e == cudaSuccess && !ctx->ktab32) e = cudaMalloc((void**)&ctx->ktab32, sizeof(float2) * N);
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "kernel table");
  double* T = (double*)malloc(sizeof(double) * N);
  double2* t64 = (double2*)malloc(sizeof(double2) * N);
  float2* t32 = (float2*)malloc(sizeof(float2) * N);
  if (!T || !t64 || !t32) {
    free(T);
    free(t64);
    free(t32);
    return sph::set_error(ctx, SPH_ERR_OOM, "kernel table");
  }
  for (int i = 0; i < N; ++i) {
    const double v = 2.0 * i / (N - 1);
    double S = 1.0;
    if (v != 0.0) {
      const double x = 0.5 * 3.14159265358979323846 * v;
      S = sin(x) / x;
    }
    T[i] = pow(S, ctx->prm.sinc_n);
  }
  for (int i = 0; i < N; ++i) {
    const double d = i + 1 < N ? T[i + 1] - T[i] : 0.0;
    t64[i] = make_double2(T[i], d);
    t32[i] = make_float2((float)T[i], (float)d);
  }
  e = cudaMemcpy(ctx->ktab64, t64, sizeof(double2) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->ktab32, t32, sizeof(float2) * N, cudaMemcpyHostToDevice);
  free(T);
  free(t64);
  free(t32);
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "kernel table");
  ctx->ktab_n = ctx->prm.sinc_n;
  return SPH_OK;
}

int check_state(sph_ctx* ctx, const sph_state* s, bool need_outputs) {
  if (!ctx) return SPH_ERR_INVALID_ARG;
  if (!s) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "state is NULL");
  if (s->n < 0 || s->n > ctx->n_max)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "n = %lld outside [0, n_max = %lld]",
                          (long long)s->n, (long long)ctx->n_max);
  if (s->n == 0) return SPH_OK;  // empty arrays may be NULL
  const void* req[] = {s->x, s->y, s->z, s->vx, s->vy, s->vz, s->h, s->m, s->u,
                       s->vxh, s->vyh, s->vzh, s->du_prev, s->id};
  for (const void* q : req)
    if (!q) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "a state array is NULL");
  if (need_outputs) {
    const void* outs[] = {s->rho, s->p, s->c, s->iad, s->ax, s->ay, s->az, s->du};
    for (const void* q : outs)
      if (!q) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "an output array is NULL");
  }
  return SPH_OK;
}

StateView view_of(const sph_state* s) {
  StateView v;
  v.x = s->x;
  v.y = s->y;
  v.z = s->z;
  v.vx = s->vx;
  v.vy = s->vy;
  v.vz = s->vz;
  v.vxh = s->vxh;
  v.vyh = s->vyh;
  v.vzh = s->vzh;
  v.h = s->h;
  v.m = s->m;
  v.u = s->u;
  v.du_prev = s->du_prev;
  v.id = s->id;
  return v;
}

OutView outs_of(const sph_state* s) {
  OutView o;
  o.rho = s->rho;
  o.p = s->p;
  o.c = s->c;
  o.iad = s->iad;
  o.ax = s->ax;
  o.ay = s->ay;
  o.az = s->az;
  o.du = s->du;
  o.omega = s->omega;
  return o;
}

int finish(sph_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, what);
  return SPH_OK;
}

template <typename T>
int dalloc(sph_ctx* ctx, T** p, size_t count, size_t* total) {
  size_t b = count * sizeof(T);
  if (b == 0) b = sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, b);
  if (e != cudaSuccess) {
    *p = nullptr;
    return sph::cuda_fail(ctx, e, "cudaMalloc");
  }
  *total += b;
  return SPH_OK;
}

void free_all(sph_ctx* ctx) {
  void* ptrs[] = {ctx->grid, ctx->err, ctx->dt_dev, ctx->diag, ctx->hfac, ctx->cell_org,
                  ctx->ktab64,
                  ctx->ktab32, ctx->code, ctx->slot,
                  ctx->perm_tmp, ctx->perm, ctx->tbl_count, ctx->tbl_start, ctx->occ,
                  ctx->scan_part, ctx->cell_of, ctx->s.x, ctx->s_id_buf, ctx->pos32,
                  ctx->cell3, ctx->nn, ctx->nbr, ctx->wcache, ctx->vol, ctx->rec_d, ctx->rec_i,
                  ctx->rec_m, ctx->cmeta, ctx->sent, ctx->masks, ctx->salloc, ctx->cells, ctx->recA, ctx->recV,
                  ctx->recQ, ctx->recC, ctx->recC2, ctx->red.part, ctx->red.counter, ctx->stats,
                  ctx->hm_buf, ctx->hm_id, ctx->grav_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

void run_search(sph_ctx* ctx, const StateView& s, int64_t n, cudaStream_t st) {
  if (sph::staged_pairs(ctx))
    sph::launch_find_masks(ctx, s, n, st);
  else
    sph::launch_find_neighbors(ctx, s, n, st);
}

void run_density(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n, cudaStream_t st) {
  if (sph::staged_pairs(ctx))
    sph::launch_density_staged(ctx, s, o, n, st);
  else if (ctx->prm.precision == SPH_FP32_MIXED)
    sph::launch_density_f32(ctx, s, o, n, st);
  else
    sph::launch_density_f64(ctx, s, o, n, st);
}

void run_iad(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n, cudaStream_t st) {
  if (sph::staged_pairs(ctx))
    sph::launch_iad_staged(ctx, s, o, n, st);
  else if (ctx->prm.precision == SPH_FP32_MIXED)
    sph::launch_iad_f32(ctx, s, o, n, st);
  else
    sph::launch_iad_f64(ctx, s, o, n, st);
}

void run_momentum(sph_ctx* ctx, const StateView& s, const OutView& o, int64_t n,
                  cudaStream_t st) {
  if (sph::staged_pairs(ctx))
    sph::launch_momentum_staged(ctx, s, o, n, st);
  else if (ctx->prm.precision == SPH_FP32_MIXED)
    sph::launch_momentum_f32(ctx, s, o, n, st);
  else
    sph::launch_momentum_f64(ctx, s, o, n, st);
}

// Step events per ring slot: marks 0..SPH_NSTAGE at the stage boundaries and
// mark SPH_NSTAGE + 1 after the second gather part, which runs between the
// search and density and is counted with the sort.
constexpr int kProfMarks = SPH_NSTAGE + 2;
constexpr int kMarkGatherB = SPH_NSTAGE + 1;

inline void prof_mark(sph_ctx* ctx, int k, cudaStream_t st) {
  if (ctx->prof) cudaEventRecord(ctx->prof_ev[ctx->prof_slot * kProfMarks + k], st);
}

// Folds the recorded event sets into prof_ms (synchronises on them).
int prof_fold(sph_ctx* ctx) {
  for (int slot = 0; slot < ctx->prof_slot; ++slot) {
    cudaEvent_t* e = ctx->prof_ev + slot * kProfMarks;
    cudaError_t err = cudaEventSynchronize(e[SPH_NSTAGE]);
    if (err != cudaSuccess) return sph::cuda_fail(ctx, err, "profile events");
    for (int k = 0; k < SPH_NSTAGE; ++k) {
      // density (stage 2) starts after the second gather part
      const cudaEvent_t from = k == 2 ? e[kMarkGatherB] : e[k];
      float ms = 0.0f;
      err = cudaEventElapsedTime(&ms, from, e[k + 1]);
      if (err != cudaSuccess) return sph::cuda_fail(ctx, err, "profile events");
      ctx->prof_ms[k] += ms;
    }
    float gb = 0.0f;  // the second gather part belongs to the sort
    err = cudaEventElapsedTime(&gb, e[2], e[kMarkGatherB]);
    if (err != cudaSuccess) return sph::cuda_fail(ctx, err, "profile events");
    ctx->prof_ms[0] += gb;
    ctx->prof_steps += 1;
  }
  ctx->prof_slot = 0;
  return SPH_OK;
}

}  // namespace

extern "C" {

void sph_default_params(sph_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  for (int k = 0; k < 3; ++k) {
    p->box_lo[k] = 0.0;
    p->box_hi[k] = 1.0;
    p->periodic[k] = 1;
  }
  p->gamma = 5.0 / 3.0;
  p->alpha = 1.0;
  p->courant = 0.2;
  p->dt_growth = 1.1;
  p->ng_target = 100;
  p->max_nb = 160;
  p->sinc_n = 6.0;
  p->precision = SPH_FP64;
  p->kernel_mode = SPH_KERNEL_EXACT;
  p->gradh = 0;
  p->pair_mode = SPH_PAIRS_STAGED;
  p->energy_dt = 0.0;
  p->angular_sums = 0;
}

int sph_init(const sph_params* params, int64_t n_max, sph_ctx** out) {
  if (!out) return SPH_ERR_INVALID_ARG;
  *out = nullptr;
  sph_ctx* ctx = (sph_ctx*)calloc(1, sizeof(sph_ctx));
  if (!ctx) return SPH_ERR_OOM;
  int rc = check_params(ctx, params);
  if (rc != SPH_OK || n_max < 1 || n_max > sph::kMaxParticles) {
    free(ctx);
    return rc != SPH_OK ? rc : SPH_ERR_INVALID_ARG;
  }
  ctx->prm = *params;
  ctx->n_max = n_max;
  ctx->hfac_ng = -1;
  ctx->ktab_n = -1.0;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e != cudaSuccess) {
    free(ctx);
    return SPH_ERR_CUDA;
  }
  ctx->Bn = kernel_norm_host(params->sinc_n);
  size_t total = 0;
  const int64_t n = n_max;
  const int mb = params->max_nb;
  rc = SPH_OK;
#define ALLOC(ptr, cnt) \
  if (rc == SPH_OK) rc = dalloc(ctx, &(ptr), (size_t)(cnt), &total)
  ALLOC(ctx->grid, 1);
  ALLOC(ctx->err, 1);
  ALLOC(ctx->dt_dev, 1);
  ALLOC(ctx->diag, 32);
  ALLOC(ctx->hfac, sph::kHTab);
  ALLOC(ctx->cell_org, 3 << sph::kMaxCellBits);
  ALLOC(ctx->code, n);
  ALLOC(ctx->slot, n);
  ALLOC(ctx->perm_tmp, n);
  ALLOC(ctx->perm, n);
  ALLOC(ctx->tbl_count, sph::kMaxTable);
  ALLOC(ctx->tbl_start, sph::kMaxTable);
  ALLOC(ctx->occ, n);
  ALLOC(ctx->scan_part, 2 * (sph::kMaxTable / sph::kScanItems));
  ALLOC(ctx->cell_of, n);
  double* sbuf = nullptr;
  ALLOC(sbuf, 13 * n);
  ALLOC(ctx->s_id_buf, n);
  ALLOC(ctx->pos32, n);
  ALLOC(ctx->cell3, n);
  ALLOC(ctx->nn, n);
  ALLOC(ctx->nbr, (size_t)mb * n);
  if (params->precision == SPH_FP64) ALLOC(ctx->wcache, (size_t)mb * n);
  ALLOC(ctx->vol, 5 * n);
  ALLOC(ctx->rec_d, n);
  ALLOC(ctx->rec_i, n);
  ALLOC(ctx->rec_m, 5 * n);
  // cell-staged pair passes: at most 27 n staged entries (a cell appears in
  // at most 27 stencils) and kMaskWords hit-mask words per particle
  ctx->sent_cap = 27 * n;
  ctx->mask_cap = (int64_t)sph::kMaskWords * n;
  ALLOC(ctx->cmeta, n);
  ALLOC(ctx->sent, (size_t)ctx->sent_cap);
  ALLOC(ctx->masks, (size_t)ctx->mask_cap);
  ALLOC(ctx->salloc, 5);
  ALLOC(ctx->cells, 3 * n);
  ALLOC(ctx->recA, n);
  ALLOC(ctx->recV, n);
  ALLOC(ctx->recQ, n);
  ALLOC(ctx->recC, n);
  ALLOC(ctx->recC2, n);
  ALLOC(ctx->red.part, sph::kReduceBlocks * 16);
  ALLOC(ctx->red.counter, 8);
  ALLOC(ctx->stats, sph::kStats);
#undef ALLOC
  if (sbuf) {
    double** f[13] = {&ctx->s.x, &ctx->s.y, &ctx->s.z, &ctx->s.vx, &ctx->s.vy, &ctx->s.vz,
                      &ctx->s.vxh, &ctx->s.vyh, &ctx->s.vzh, &ctx->s.h, &ctx->s.m, &ctx->s.u,
                      &ctx->s.du_prev};
    for (int k = 0; k < 13; ++k) *f[k] = sbuf + (size_t)k * n;
    ctx->s.id = ctx->s_id_buf;
  }
  if (ctx->vol) {
    ctx->X = ctx->vol + n;
    ctx->inv_rho = ctx->vol + 2 * n;
  }
  if (rc == SPH_OK) {
    e = cudaMemset(ctx->err, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->red.counter, 0, 8 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(ctx->diag, 0, 32 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(ctx->stats, 0, sph::kStats * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->tbl_count, 0, sph::kMaxTable * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = sph::cuda_fail(ctx, e, "init");
  }
  if (rc == SPH_OK) rc = build_kernel_table(ctx);
  if (rc != SPH_OK) {
    free_all(ctx);
    free(ctx);
    return rc;
  }
  *out = ctx;
  return SPH_OK;
}

void sph_destroy(sph_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  if (ctx->prof_ev) {
    for (int k = 0; k < sph::kProfRing * kProfMarks; ++k)
      if (ctx->prof_ev[k]) cudaEventDestroy(ctx->prof_ev[k]);
    free(ctx->prof_ev);
  }
  if (ctx->hs_stream) cudaStreamDestroy(ctx->hs_stream);
  for (cudaEvent_t ev : ctx->hs_ev)
    if (ev) cudaEventDestroy(ev);
  free_all(ctx);
  free(ctx);
}

int sph_set_params(sph_ctx* ctx, const sph_params* params) {
  if (!ctx) return SPH_ERR_INVALID_ARG;
  int rc = check_params(ctx, params);
  if (rc != SPH_OK) return rc;
  if (params->max_nb != ctx->prm.max_nb || params->sinc_n != ctx->prm.sinc_n)
    return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "max_nb and sinc_n are fixed at sph_init");
  if (params->precision == SPH_FP64 && !ctx->wcache) {
    // a context created for FP32-mixed gets the FP64 kernel-value cache now
    cudaError_t e = cudaMalloc((void**)&ctx->wcache,
                               sizeof(double) * (size_t)ctx->prm.max_nb * (size_t)ctx->n_max);
    if (e != cudaSuccess) {
      ctx->wcache = nullptr;
      return sph::cuda_fail(ctx, e, "sph_set_params: FP64 kernel-value cache");
    }
  }
  const bool staged_before = sph::staged_pairs(ctx);
  ctx->prm = *params;
  // the masks of the staged form are not lists (and the other way round)
  if (sph::staged_pairs(ctx) != staged_before) ctx->have_lists = 0;
  ctx->have_density = ctx->have_iad = 0;
  return build_kernel_table(ctx);
}

double sph_kernel_norm(const sph_ctx* ctx) { return ctx ? ctx->Bn : 0.0; }

int sph_find_neighbors(sph_ctx* ctx, sph_state* state, sph_stream_t stream) {
  int rc = check_state(ctx, state, false);
  if (rc != SPH_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const StateView in = view_of(state);
  if (state->n == 0) {
    ctx->have_lists = 1;
    ctx->have_density = ctx->have_iad = 0;
    return SPH_OK;
  }
  sph::launch_grid(ctx, in, state->n, st);
  sph::launch_sort_gather(ctx, in, state->n, st);
  sph::launch_copy_state(in, ctx->s, state->n, st, ctx);
  run_search(ctx, in, state->n, st);
  rc = finish(ctx, "sph_find_neighbors");
  ctx->have_lists = rc == SPH_OK;
  ctx->have_density = ctx->have_iad = 0;
  return rc;
}

int sph_get_neighbors(sph_ctx* ctx, const sph_state* state, int32_t* counts, int64_t* ids,
                      sph_stream_t stream) {
  int rc = check_state(ctx, state, false);
  if (rc != SPH_OK) return rc;
  if (!counts || !ids) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "NULL output");
  if (!ctx->have_lists)
    return sph::set_error(ctx, SPH_ERR_ORDER, "no neighbour lists: call sph_find_neighbors");
  if (sph::staged_pairs(ctx))
    sph::launch_export_masks(ctx, view_of(state), state->n, counts, ids, (cudaStream_t)stream);
  else
    sph::launch_export_neighbors(ctx, view_of(state), state->n, counts, ids,
                                 (cudaStream_t)stream);
  return finish(ctx, "sph_get_neighbors");
}

int sph_density(sph_ctx* ctx, sph_state* state, sph_stream_t stream) {
  int rc = check_state(ctx, state, true);
  if (rc != SPH_OK) return rc;
  if (!ctx->have_lists)
    return sph::set_error(ctx, SPH_ERR_ORDER, "no neighbour lists: call sph_find_neighbors");
  run_density(ctx, view_of(state), outs_of(state), state->n, (cudaStream_t)stream);
  rc = finish(ctx, "sph_density");
  ctx->have_density = rc == SPH_OK;
  ctx->have_iad = 0;
  return rc;
}

int sph_iad(sph_ctx* ctx, sph_state* state, sph_stream_t stream) {
  int rc = check_state(ctx, state, true);
  if (rc != SPH_OK) return rc;
  if (!ctx->have_density) return sph::set_error(ctx, SPH_ERR_ORDER, "call sph_density first");
  run_iad(ctx, view_of(state), outs_of(state), state->n, (cudaStream_t)stream);
  rc = finish(ctx, "sph_iad");
  ctx->have_iad = rc == SPH_OK;
  return rc;
}

int sph_momentum_energy(sph_ctx* ctx, sph_state* state, sph_stream_t stream) {
  int rc = check_state(ctx, state, true);
  if (rc != SPH_OK) return rc;
  if (!ctx->have_iad) return sph::set_error(ctx, SPH_ERR_ORDER, "call sph_iad first");
  run_momentum(ctx, view_of(state), outs_of(state), state->n, (cudaStream_t)stream);
  return finish(ctx, "sph_momentum_energy");
}

int sph_step(sph_ctx* ctx, sph_state* state, double* dt_inout, sph_stream_t stream) {
  int rc = check_state(ctx, state, true);
  if (rc != SPH_OK) return rc;
  if (!dt_inout) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "dt_inout is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = state->n;
  if (n == 0) return SPH_OK;  // nothing to advance; dt is left unchanged
  const StateView in = view_of(state);
  const OutView o = outs_of(state);
  if (ctx->prof && ctx->prof_slot == sph::kProfRing) {
    rc = prof_fold(ctx);
    if (rc != SPH_OK) return rc;
  }
  prof_mark(ctx, 0, st);
  sph::launch_grid(ctx, in, n, st);
  sph::launch_sort(ctx, in, n, st, ctx->hook_wait_a);
  if (ctx->hook_sorted) cudaEventRecord(ctx->hook_sorted, st);
  prof_mark(ctx, 1, st);
  run_search(ctx, ctx->s, n, st);
  prof_mark(ctx, 2, st);
  // velocities and integrator history: a host caller may still be copying
  // them in while the search runs
  if (ctx->hook_wait) cudaStreamWaitEvent(st, ctx->hook_wait, 0);
  sph::launch_gather_b(ctx, in, n, st);
  prof_mark(ctx, kMarkGatherB, st);
  run_density(ctx, ctx->s, o, n, st);
  prof_mark(ctx, 3, st);
  run_iad(ctx, ctx->s, o, n, st);
  prof_mark(ctx, 4, st);
  run_momentum(ctx, ctx->s, o, n, st);
  if (ctx->hook_mom) cudaEventRecord(ctx->hook_mom, st);
  prof_mark(ctx, 5, st);
  sph::launch_timestep(ctx, ctx->s, o, n, dt_inout, st);
  prof_mark(ctx, 6, st);
  sph::launch_update(ctx, ctx->s, o, ctx->hook_update_dst ? *ctx->hook_update_dst : in, n,
                     dt_inout, st);
  prof_mark(ctx, 7, st);
  if (ctx->prof) ctx->prof_slot += 1;
  rc = finish(ctx, "sph_step");
  // the lists index the pre-update positions, which are now overwritten
  ctx->have_lists = 0;
  ctx->have_density = ctx->have_iad = 0;
  return rc;
}

int sph_step_host(sph_ctx* ctx, sph_state* hs, double* dt_inout, sph_stream_t stream) {
  int rc = check_state(ctx, hs, false);
  if (rc != SPH_OK) return rc;
  if (!dt_inout) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "dt_inout is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = hs->n;
  if (n == 0) return SPH_OK;  // nothing to advance; dt is left unchanged
  const int64_t nm = ctx->n_max;
  cudaError_t e = cudaSuccess;
  if (!ctx->hm_buf) {
    e = cudaMalloc((void**)&ctx->hm_buf, sizeof(double) * (size_t)nm * 26);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->hm_id, sizeof(int64_t) * (size_t)nm);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->hs_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&ctx->hs_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "sph_step_host mirrors");
  }
  cudaStream_t cs = ctx->hs_stream;
  cudaEvent_t ev_start = ctx->hs_ev[0], ev_in_a = ctx->hs_ev[1], ev_in = ctx->hs_ev[2],
              ev_sorted = ctx->hs_ev[3], ev_mom = ctx->hs_ev[4], ev_done = ctx->hs_ev[5];
  sph_state ds;
  memset(&ds, 0, sizeof(ds));  // omega stays NULL: not mirrored
  double* base = ctx->hm_buf;
  double** dfields[21] = {&ds.x, &ds.y, &ds.z, &ds.vx, &ds.vy, &ds.vz, &ds.h, &ds.m, &ds.u,
                          &ds.vxh, &ds.vyh, &ds.vzh, &ds.du_prev, &ds.rho, &ds.p, &ds.c,
                          &ds.ax, &ds.ay, &ds.az, &ds.du, &ds.iad};
  for (int k = 0; k < 20; ++k) *dfields[k] = base + (size_t)k * nm;
  ds.iad = base + (size_t)20 * nm;  // 6 * nm
  ds.id = ctx->hm_id;
  ds.n = n;
  const size_t b = sizeof(double) * (size_t)n;
  // Copies in: x, y, z, h (read by the cell keys) on the caller's stream;
  // m, u and id on the second stream, overlapping the cell keys and order
  // (the step waits for them before its first gather part); velocities and
  // the integrator history after them, overlapping the search (waited for
  // before the second gather part).  The second stream starts after all
  // earlier work of the caller's stream, so the device mirrors are free.
  double* hin_a[4] = {hs->x, hs->y, hs->z, hs->h};
  double* din_a[4] = {ds.x, ds.y, ds.z, ds.h};
  double* hin_b[7] = {hs->vx, hs->vy, hs->vz, hs->vxh, hs->vyh, hs->vzh, hs->du_prev};
  double* din_b[7] = {ds.vx, ds.vy, ds.vz, ds.vxh, ds.vyh, ds.vzh, ds.du_prev};
  e = cudaEventRecord(ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(din_a[k], hin_a[k], b, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->dt_dev, dt_inout, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds.m, hs->m, b, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds.u, hs->u, b, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ds.id, hs->id, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ev_in_a, cs);
  for (int k = 0; k < 7 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(din_b[k], hin_b[k], b, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ev_in, cs);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(cs);
    return sph::cuda_fail(ctx, e, "sph_step_host copy in");
  }
  // Pinned caller arrays can be written by the update kernel itself, so the
  // new state crosses the host link while the update runs instead of after
  // it.  Pageable arrays take the copy path.
  double* hout_s[11] = {hs->x, hs->y, hs->z, hs->vx, hs->vy, hs->vz, hs->vxh, hs->vyh, hs->vzh,
                        hs->u, hs->h};
  double* zc[11];
  bool direct = true;
  for (int k = 0; k < 11 && direct; ++k) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, hout_s[k]) != cudaSuccess || at.type != cudaMemoryTypeHost ||
        !at.devicePointer)
      direct = false;
    else
      zc[k] = (double*)at.devicePointer;
  }
  cudaGetLastError();  // a failed attribute query is not an error of this call
  sph::StateView zdst;
  memset(&zdst, 0, sizeof(zdst));
  if (direct) {
    zdst.x = zc[0];
    zdst.y = zc[1];
    zdst.z = zc[2];
    zdst.vx = zc[3];
    zdst.vy = zc[4];
    zdst.vz = zc[5];
    zdst.vxh = zc[6];
    zdst.vyh = zc[7];
    zdst.vzh = zc[8];
    zdst.u = zc[9];
    zdst.h = zc[10];
  }
  ctx->hook_wait_a = ev_in_a;
  ctx->hook_wait = ev_in;
  ctx->hook_sorted = ev_sorted;
  ctx->hook_mom = ev_mom;
  ctx->hook_update_dst = direct ? &zdst : nullptr;
  rc = sph_step(ctx, &ds, ctx->dt_dev, stream);
  ctx->hook_wait_a = ctx->hook_wait = ctx->hook_sorted = ctx->hook_mom = nullptr;
  ctx->hook_update_dst = nullptr;
  if (rc != SPH_OK) {
    cudaStreamSynchronize(cs);
    return rc;
  }
  // Copies out on the second stream as soon as their values are final: m and
  // id after the sort (the sorted scratch holds what the update writes back),
  // du_prev = du after the momentum pass.  Their copies in (earlier on the
  // same stream) have completed by then.
  e = cudaStreamWaitEvent(cs, ev_sorted, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs->m, ctx->s.m, b, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hs->id, ctx->s.id, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost,
                        cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_mom, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs->du_prev, ds.du, b, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaEventRecord(ev_done, cs);
  // the rest after the update, on the caller's stream (already written by
  // the update kernel when the arrays are pinned)
  double* dout_s[11] = {ds.x, ds.y, ds.z, ds.vx, ds.vy, ds.vz, ds.vxh, ds.vyh, ds.vzh, ds.u, ds.h};
  for (int k = 0; k < 11 && e == cudaSuccess && !direct; ++k)
    e = cudaMemcpyAsync(hout_s[k], dout_s[k], b, cudaMemcpyDeviceToHost, st);
  double* hout[7] = {hs->rho, hs->p, hs->c, hs->ax, hs->ay, hs->az, hs->du};
  double* dout[7] = {ds.rho, ds.p, ds.c, ds.ax, ds.ay, ds.az, ds.du};
  for (int k = 0; k < 7 && e == cudaSuccess; ++k)
    if (hout[k]) e = cudaMemcpyAsync(hout[k], dout[k], b, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hs->iad)
    e = cudaMemcpyAsync(hs->iad, ds.iad, 6 * b, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dt_inout, ctx->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_done, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(cs);
    return sph::cuda_fail(ctx, e, "sph_step_host copy out");
  }
  return SPH_OK;
}

int sph_diagnostics(sph_ctx* ctx, const sph_state* state, double* out, sph_stream_t stream) {
  int rc = check_state(ctx, state, false);
  if (rc != SPH_OK) return rc;
  if (!out) return sph::set_error(ctx, SPH_ERR_INVALID_ARG, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  sph::launch_diagnostics(ctx, view_of(state), state->n, st);
  cudaError_t e = cudaMemcpyAsync(out, ctx->diag + 16, 8 * sizeof(double),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "sph_diagnostics");
  return SPH_OK;
}

int sph_last_diagnostics(sph_ctx* ctx, double* out, sph_stream_t stream) {
  if (!ctx || !out) return SPH_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(out, ctx->diag, 12 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "sph_last_diagnostics");
  return SPH_OK;
}

int sph_error_word(sph_ctx* ctx, uint32_t* flags) {
  if (!ctx || !flags) return SPH_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(flags, ctx->err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->err, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "sph_error_word");
  return SPH_OK;
}

const char* sph_last_error(const sph_ctx* ctx) { return ctx ? ctx->last_error : "no context"; }

int64_t sph_launch_count(const sph_ctx* ctx) { return ctx ? ctx->launches : 0; }

int sph_stats(sph_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return SPH_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(out, ctx->stats, sph::kStats * sizeof(unsigned long long),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "sph_stats");
  return SPH_OK;
}

int sph_profile(sph_ctx* ctx, int enable) {
  if (!ctx) return SPH_ERR_INVALID_ARG;
  if (enable && !ctx->prof_ev) {
    const int total = sph::kProfRing * kProfMarks;
    ctx->prof_ev = (cudaEvent_t*)calloc(total, sizeof(cudaEvent_t));
    if (!ctx->prof_ev) return sph::set_error(ctx, SPH_ERR_OOM, "profile events");
    for (int k = 0; k < total; ++k) {
      cudaError_t e = cudaEventCreate(&ctx->prof_ev[k]);
      if (e != cudaSuccess) return sph::cuda_fail(ctx, e, "cudaEventCreate");
    }
  }
  if (!enable && ctx->prof) {
    int rc = prof_fold(ctx);
    if (rc != SPH_OK) return rc;
  }
  ctx->prof = enable ? 1 : 0;
  return SPH_OK;
}

int sph_stage_times(sph_ctx* ctx, double* ms, int64_t* steps) {
  if (!ctx || !ms || !steps) return SPH_ERR_INVALID_ARG;
  int rc = prof_fold(ctx);
  if (rc != SPH_OK) return rc;
  for (int k = 0; k < SPH_NSTAGE; ++k) {
    ms[k] = ctx->prof_ms[k];
    ctx->prof_ms[k] = 0.0;
  }
  *steps = ctx->prof_steps;
  ctx->prof_steps = 0;
  return SPH_OK;
}

}  // extern "C"
