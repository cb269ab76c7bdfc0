/*
 * sph.h -- C ABI of the GB300 SPH neighbour-pipeline library (libsph.so).
 *
 * The library advances a particle state by the per-step pipeline of
 * Cavelan et al., "A Smoothed Particle Hydrodynamics Mini-App for Exascale"
 * (arXiv 2005.02656): neighbour search, density (section 4.1, Eq. 1) with an
 * ideal-gas equation of state, the IAD matrix (section 4.1, A_ab terms),
 * momentum and energy with artificial viscosity (Eqs. 2-5), the global
 * minimum time step (section 4.2) and the position/velocity/energy update
 * (section 4.1, second-order Press and Adams-Bashforth integrators).  Every
 * step runs in the library's own CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point:
 *  - Return value: SPH_OK (0) or a negative SPH_ERR_* code.  A non-zero code
 *    leaves a message readable with sph_last_error().
 *  - All work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *    void*; NULL means the legacy default stream) unless stated otherwise.
 *    Faults found on the device (overflowing neighbour lists, a singular IAD
 *    matrix, a non-finite value, an invalid box) do not fail the call: they
 *    set bits of the context's error word, read with sph_error_word().
 *  - Pointers inside sph_state are caller-owned DEVICE memory (except for
 *    sph_step_host).  The library never frees caller memory.  Every array
 *    has state.n elements (iad has 6*n) and is contiguous.
 *  - A context is bound to the CUDA device that was current at sph_init();
 *    calls must be made with that device current.  A context may be used
 *    from one host thread at a time; calls on one context must be ordered
 *    (same stream, or synchronised).
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SPH_API __attribute__((visibility("default")))
#else
#define SPH_API
#endif

typedef struct sph_ctx sph_ctx;
typedef void* sph_stream_t; /* cudaStream_t */

/* Return codes. */
enum {
  SPH_OK = 0,
  SPH_ERR_INVALID_ARG = -1, /* bad pointer, size or parameter               */
  SPH_ERR_CUDA = -2,        /* a CUDA runtime call failed                   */
  SPH_ERR_NB_OVERFLOW = -3, /* (error-word bit) a list exceeded max_nb      */
  SPH_ERR_SINGULAR_IAD = -4,/* (error-word bit) tau_a not invertible        */
  SPH_ERR_NONFINITE = -5,   /* (error-word bit) NaN/inf in a result         */
  SPH_ERR_TIMEOUT = -6,     /* a bounded device wait gave up                */
  SPH_ERR_OOM = -7,         /* device allocation failed                     */
  SPH_ERR_ORDER = -8        /* a stage was called before its inputs exist   */
};

/* Bits of the device error word (sph_error_word). */
#define SPH_FLAG_NB_OVERFLOW 0x1u   /* some particle had more than max_nb neighbours; its
                                       list was truncated (nn keeps the true count)       */
#define SPH_FLAG_SINGULAR_IAD 0x2u  /* |det tau_a| <= 1e-12 max|tau_a|^3; C_a set to 0   */
#define SPH_FLAG_NONFINITE 0x4u     /* a density, acceleration, du or dt was NaN/inf      */
#define SPH_FLAG_BAD_BOX 0x8u       /* 2 h_max >= L/2 on a periodic axis (minimum image
                                       undefined); the step's results are not valid       */
#define SPH_FLAG_CELL_OVERFLOW 0x10u/* more than 65535 particles in one cell stencil      */
#define SPH_FLAG_TIMEOUT 0x20u      /* a bounded device-side wait expired                 */

/* Arithmetic of the pair sums. */
enum {
  SPH_FP64 = 0,       /* every step in FP64                                          */
  SPH_FP32_MIXED = 1  /* pair separations, kernel values and the density, IAD and
                         force sums in FP32; positions, integration, dt and the
                         conservation sums in FP64                                    */
};

/* Kernel evaluation (section 4.5 of the paper mentions a 20,000-entry lookup
 * table; SPH_KERNEL_EXACT evaluates sinc by a polynomial).                     */
enum { SPH_KERNEL_EXACT = 0, SPH_KERNEL_TABLE = 1 };
/* SPH_KERNEL_TABLE (section 4.5): the paper's lookup table of 20,000 kernel
 * values S(v_i)^n at v_i = 2 i / 19999, built on the host with libm sin and
 * pow, interpolated linearly in v = r / h (q = v * 19999 / 2, i = floor(q)
 * capped at 19998, W = B_n / h^3 (T_i + (T_{i+1} - T_i) (q - i))).  It
 * differs from the exact kernel by the interpolation error, relative
 * ~1e-8; gradh, the ensemble and the differentiable rollout require
 * SPH_KERNEL_EXACT. */

/* How the FP32-mixed pair sums reach the neighbours (SPH_FP64 always uses
 * SPH_PAIRS_LISTS).
 *  SPH_PAIRS_STAGED: the neighbour search records, per occupied cell, the
 *    candidates it staged (the particles of the cell's 3x3x3 stencil within
 *    reach of the cell's targets, in stencil order) and, per target, one
 *    64-bit hit mask per 64 staged candidates (bit set: r^2 < (2 h_a)^2
 *    decided exactly as by sph_find_neighbors).  Density, IAD and momentum
 *    then work cell by cell: the cell's staged candidate records are copied
 *    into shared memory once and each target's sum runs over the staged slots
 *    of its hit bits (slot lists the search writes from the masks).
 *    The masks and staged entries live in the list buffer and a 108-byte-per-
 *    particle entry buffer; a state whose masks do not fit (more than
 *    max_nb / 2 mask words per particle on average) raises
 *    SPH_FLAG_NB_OVERFLOW.
 *  SPH_PAIRS_LISTS: the search writes int32 neighbour lists (max_nb per
 *    particle) and every pair kernel gathers its neighbours' records from
 *    global memory; the batched ensemble uses this form, and a single box
 *    run with it equals the ensemble's result for that box bit for bit.
 * Both give the same neighbour sets and the same sums up to FP32 rounding
 * (summation order, and the order in which per-particle factors such as
 * 1/h^2 and P/rho^2 are formed). */
enum { SPH_PAIRS_STAGED = 0, SPH_PAIRS_LISTS = 1 };

/* Particle state: structure of arrays of caller-owned device memory.
 *  inputs (persistent state): x y z (positions), vx vy vz (velocity at integer
 *    time, v^n), vxh vyh vzh (half-step velocity v^{n-1/2}; set equal to v
 *    before the first step), h (smoothing length), m (mass), u (specific
 *    internal energy), du_prev (du/dt of the previous step; 0 before the first
 *    step), id (caller's particle ids, permuted with the state).
 *  outputs of a step (valid for the state as it was before the update):
 *    rho, p, c (density, pressure, sound speed), iad (6 per particle: the
 *    symmetric IAD matrix C = tau^{-1} as xx xy xz yy yz zz, particle-major),
 *    ax ay az (acceleration), du (du/dt); omega (the grad-h terms Omega of
 *    Eqs. 2-3, written when params.gradh = 1; may be NULL).
 * The library reorders every array of the state in place (particles are kept
 * sorted by cell in Morton order), so callers identify particles by id. */
typedef struct {
  double *x, *y, *z, *vx, *vy, *vz, *h, *m, *u;
  double *vxh, *vyh, *vzh, *du_prev;
  double *rho, *p, *c, *iad, *ax, *ay, *az, *du, *omega;
  int64_t* id;
  int64_t n;
} sph_state;

/* Parameters.  Defaults in brackets (sph_default_params). */
typedef struct {
  double box_lo[3], box_hi[3]; /* box corners; used on periodic axes            */
  int periodic[3];             /* 1 periodic, 0 open (open axes take their extent
                                  from the particles every step)                */
  double gamma;                /* adiabatic index of the ideal gas [5/3]        */
  double alpha;                /* viscosity coefficient of Eq. 5 [1]            */
  double courant;              /* Courant factor of the time step [0.2]         */
  double dt_growth;            /* max dt_n / dt_{n-1} [1.1]                     */
  int ng_target;               /* target neighbour count for h adaptation [100];
                                  0 keeps h fixed                               */
  int max_nb;                  /* neighbour-list capacity per particle, a
                                  multiple of 4 in [4, 4096] [160]              */
  double sinc_n;               /* exponent n of the sinc kernel, integer 1..12 [6] */
  int precision;               /* SPH_FP64 or SPH_FP32_MIXED [SPH_FP64]         */
  int kernel_mode;             /* SPH_KERNEL_EXACT or SPH_KERNEL_TABLE [EXACT]  */
  int gradh;                   /* grad-h terms of Eqs. 2-3 (section 4.1): 0 sets
                                  Omega = 1; 1 computes Omega_a = 1 + h_a/(3 rho_a)
                                  sum_b m_b dW_ab(h_a)/dh_a in the density pass
                                  (self term included) and uses P/(Omega rho^2)
                                  in momentum and energy [0]                    */
  int pair_mode;               /* SPH_PAIRS_STAGED or SPH_PAIRS_LISTS, read by
                                  SPH_FP32_MIXED contexts [SPH_PAIRS_STAGED]     */
  double energy_dt;            /* energy-rate limit of the time step (a reading;
                                  section 4.2 names only a global minimum):
                                  dt_n <= energy_dt * min_a u_a / |du_a| over
                                  the particles with du_a != 0; 0 turns it off
                                  [0].  Must be >= 0; not used by the ensemble
                                  (sph_ensemble_init rejects a nonzero value)   */
  int angular_sums;            /* 1: sph_step also sums the angular momentum
                                  of the new state (sph_last_diagnostics
                                  out[5..7]); 0: out[5..7] are NaN and the
                                  update saves 12 FP64 operations per particle
                                  (section 4.2 makes the conservation reduction
                                  optional; momentum and energy are always
                                  summed) [0].  Must be 0 or 1                   */
} sph_params;

/* Fills *p with the defaults above and a periodic unit box. */
SPH_API void sph_default_params(sph_params* p);

/* Creates a context for states of up to n_max particles (1 <= n_max <= 2^27)
 * on the current
 * device, allocating the library-owned scratch (sort buffers, cell tables,
 * neighbour lists of n_max * max_nb int32, per-particle work arrays and
 * reduction buffers).  Computes B_n (the kernel normalisation of Eq. 6) on
 * the host.  Returns SPH_ERR_INVALID_ARG for a bad parameter, SPH_ERR_OOM if
 * an allocation fails.  Synchronous. */
SPH_API int sph_init(const sph_params* params, int64_t n_max, sph_ctx** out);

/* Frees the context and its scratch (synchronises the device first). */
SPH_API void sph_destroy(sph_ctx* ctx);

/* Replaces the physical parameters (gamma, alpha, courant, dt_growth,
 * ng_target, precision, box).  max_nb and sinc_n must not change. */
SPH_API int sph_set_params(sph_ctx* ctx, const sph_params* params);

/* The normalisation constant B_n in use (section 4.1, Eq. 6). */
SPH_API double sph_kernel_norm(const sph_ctx* ctx);

/* Neighbour search (section 4.1: b runs over the neighbours of a, the
 * kernel's support being |x_a - x_b| <= 2 h_a; section 4.3: particles kept in
 * space-filling-curve order).  Computes the cell grid (cell side >= 2 h_max;
 * open axes from the particles' extent), sorts the state in place by cell
 * Morton code (ties by previous position), and builds for every particle a
 * the list of b != a with r_ab^2 < (2 h_a)^2, where r_ab is the minimum-image
 * separation on periodic axes and r^2 = (dx*dx + dy*dy) + dz*dz is evaluated
 * in FP64 without fused multiply-adds (bit-identical to that definition).
 * Must precede sph_density/sph_iad/sph_momentum_energy on the same state. */
SPH_API int sph_find_neighbors(sph_ctx* ctx, sph_state* state, sph_stream_t stream);

/* Exports the lists of the last sph_find_neighbors/sph_step in id space:
 * counts[p] = number of neighbours of the particle at (current) position p,
 * ids[p*max_nb + k], k < min(counts[p], max_nb) = ids of its neighbours in
 * ascending order.  Both are caller device arrays of n and n*max_nb entries. */
SPH_API int sph_get_neighbors(sph_ctx* ctx, const sph_state* state, int32_t* counts, int64_t* ids,
                      sph_stream_t stream);

/* Density (Eq. 1, self term included) and the ideal-gas equation of state
 * P = (gamma-1) rho u, c = sqrt(gamma P / rho).  Writes rho, p, c. */
SPH_API int sph_density(sph_ctx* ctx, sph_state* state, sph_stream_t stream);

/* IAD matrix: tau_a = sum_b (m_b/rho_b) (x_b-x_a)(x_b-x_a)^T W_ab(h_a),
 * C_a = tau_a^{-1}.  Writes iad (6 per particle). */
SPH_API int sph_iad(sph_ctx* ctx, sph_state* state, sph_stream_t stream);

/* Momentum and energy equations with IAD and artificial viscosity (Eqs. 2-5,
 * Omega = 1; the energy prefactor read as P_a/rho_a^2 and the viscous
 * acceleration entering with a minus sign).  Writes ax, ay, az, du. */
SPH_API int sph_momentum_energy(sph_ctx* ctx, sph_state* state, sph_stream_t stream);

/* One full step: neighbour search, density + EOS, IAD, momentum/energy, the
 * global time step dt_n = min(courant * min_a h_a/c_a, dt_growth * dt_{n-1})
 * (and energy_dt * min_a u_a/|du_a| when energy_dt > 0)
 * (no cap when dt_{n-1} = 0), and the update (half-step velocity kick by
 * (dt_n + dt_{n-1})/2, drift, predicted velocity, Adams-Bashforth energy,
 * periodic wrap, h <- h (1 + (ng_target/max(nn,1))^(1/3)) / 2).
 * dt_inout: DEVICE pointer to one double holding dt_{n-1} on entry (0 before
 * the first step) and dt_n on return.  Also accumulates the conservation
 * sums of the new state (sph_last_diagnostics). */
SPH_API int sph_step(sph_ctx* ctx, sph_state* state, double* dt_inout, sph_stream_t stream);

/* sph_step for callers whose state lives in HOST memory (pinned or pageable):
 * copies the state in, steps, copies the new state and the outputs back and
 * synchronises the stream.  dt_inout is a HOST pointer.  Uses device mirrors,
 * a second stream and events owned by the context (created on first use):
 * velocities and the integrator history are copied in on the second stream
 * while the sort and the neighbour search run, and m, id and du_prev are
 * copied out as soon as the step has produced them, so pinned buffers let
 * copies and kernels overlap.  When x, y, z, vx, vy, vz, vxh, vyh, vzh, u and h
 * are pinned (page-locked, device-accessible) host memory, the update kernel
 * writes the new state straight into them; otherwise they are copied back.
 * The call returns after every copy and write has completed. */
SPH_API int sph_step_host(sph_ctx* ctx, sph_state* host_state, double* dt_inout, sph_stream_t stream);

/* Conservation sums of a state {Px, Py, Pz, E_kin, E_int, Lx, Ly, Lz}
 * (section 4.2: total momentum and energy) in FP64: per-thread partial sums,
 * then fixed-shape warp, block and grid trees, so the result is the same on
 * every run (within 1e-13 relative of an exactly rounded sum on the tested
 * states).  out: HOST array of 8.  Synchronises the stream. */
SPH_API int sph_diagnostics(sph_ctx* ctx, const sph_state* state, double* out, sph_stream_t stream);

/* Conservation sums accumulated by the last sph_step (of its new state) and
 * its dt, without a separate pass: out[0..7] as sph_diagnostics (out[5..7]
 * NaN unless params.angular_sums = 1), out[8] = dt,
 * out[9] = min nn, out[10] = max nn, out[11] = sum nn.  HOST array of 12;
 * synchronises the stream. */
SPH_API int sph_last_diagnostics(sph_ctx* ctx, double* out, sph_stream_t stream);

/* Reads and clears the device error word (SPH_FLAG_* bits).  Synchronous. */
SPH_API int sph_error_word(sph_ctx* ctx, uint32_t* flags);

/* Message of the last failing call on this context ("" if none). */
SPH_API const char* sph_last_error(const sph_ctx* ctx);

/* The conservation sums of sph_diagnostics for callers that cannot allocate
 * device memory: a host program that owns the whole device memory through its
 * own pool and forbids any other allocation, or a component that holds no
 * sph_ctx and must not create one.  No context is needed and nothing is
 * allocated: the per-block partial sums live in a file-scope static device
 * array of about 512 KB that every device loading the library holds until the
 * process exits.  The paper has no counterpart; it is an interface
 * convenience.
 *   state: as for sph_diagnostics; only x y z vx vy vz m u and n are read
 *          (device arrays); n must be <= 16,777,216, larger states are
 *          rejected with SPH_ERR_INVALID_ARG.
 *   out:   HOST array of 8, filled as by sph_diagnostics.
 * The call copies the sums to the host and synchronises the stream, so it
 * cannot run on a stream that is being captured into a CUDA graph: such a
 * stream is refused with SPH_ERR_INVALID_ARG before any other CUDA call, and
 * the capture is left intact.  The first call on a device, with that device
 * current, looks up the static array's device address.  All calls share the
 * static array: calls that overlap on the GPU (other streams or host threads)
 * race.  Returns SPH_OK, SPH_ERR_INVALID_ARG or SPH_ERR_CUDA. */
SPH_API int sph_diagnostics_noalloc(const sph_state* state, double* out, sph_stream_t stream);

/* Self-gravity (section 4.1: a multipolar expansion evaluated on the tree
 * used for the neighbour search), as an acceleration added by the caller:
 *   g_a = -G sum_{b != a} m_b (x_a - x_b) / (|x_a - x_b|^2 + eps^2)^(3/2),
 * approximated on a tree whose leaves are the occupied cells of the
 * neighbour grid (side >= 2 h_max) and whose level-l nodes are the cells
 * sharing the top 3 l Morton bits.  Each node carries its mass, centre of
 * mass c and traceless quadrupole Q; a node whose box does not contain x_a
 * and whose longest side s satisfies s < theta |x_a - c| contributes
 * -G M r / (|r|^2 + eps^2)^(3/2) + G Q r / |r|^5 - (5/2) G (r.Q.r) r / |r|^7
 * (r = x_a - c); leaves that are opened contribute their particles directly.
 * theta = 0 gives the direct sum.  All axes must be open (params.periodic all
 * 0).  Sorts the state in place like sph_find_neighbors (and invalidates the
 * lists); gx gy gz (DEVICE, n each) receive g in the new order.
 * interactions (HOST, optional, 2 values): node and particle interactions.
 * Precision follows params.precision.  SPH_FP64: everything in FP64.
 * SPH_FP32_MIXED: the node and particle terms are evaluated and summed in
 * FP32 (node coordinates relative to the grid origin, particles relative to
 * their leaf's centre of mass, the target's offset from a leaf formed in
 * FP64); the opening decisions are exact (an FP32 test with a margin that
 * covers its rounding, the FP64 test inside the margin), so both precisions
 * make the same interactions.  Scratch: about 150 B per occupied cell and
 * level, plus 16 B per particle in SPH_FP32_MIXED (grow-only, kept by ctx).
 * Synchronises the stream. */
SPH_API int sph_gravity(sph_ctx* ctx, sph_state* state, double G, double eps, double theta,
                        double* gx, double* gy, double* gz, int64_t* interactions,
                        sph_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched ensemble: independent boxes of uneven sizes, each with its own    */
/* box, periodicity, viscosity alpha and time step, advanced together by one */
/* persistent cooperative kernel per call (the single-box pipeline, phase by */
/* phase over all boxes, FP32-mixed).  The launch can be captured in a CUDA  */
/* graph and replayed.  Phases are separated by a device-side grid barrier   */
/* whose wait is bounded (about 2 s): on expiry the kernel sets              */
/* SPH_FLAG_TIMEOUT and returns; sph_ensemble_error_word reads and clears it */
/* and re-arms the barrier.                                                  */
/* ------------------------------------------------------------------------ */
typedef struct sph_ens sph_ens;

/* Tuning knobs of the ensemble kernel (picked by the Python autotuner). */
typedef struct {
  double cell_factor;  /* cells of side >= cell_factor * 2 h_max, in [1, 4] [1]   */
  int blocks_per_sm;   /* persistent CTAs per SM, 0 = the occupancy maximum [0]   */
  int test_skip_block; /* test hook: this CTA leaves before the first barrier so
                          the others' bounded wait expires; -1 disables [-1]     */
  int find_window;     /* tile shape of the neighbour search: candidate slots
                          staged per warp, 128, 256 or 512 [512]; smaller
                          windows leave more of the SM's L1 to the pair phases */
  int threads_per_particle; /* lanes sharing one particle's neighbour list in
                          the density and IAD phases: 1, 2 or 4 [1] */
  int momentum_threads;  /* lanes sharing one particle's neighbour list in the
                          momentum phase: 1, 2 or 4 [4].  With the defaults
                          (1 and 4, the single-box kernels' split) a box's
                          results equal a single-box sph_step */
} sph_ens_config;

/* Fills c with the defaults in brackets above (host only, no device work). */
SPH_API void sph_ens_default_config(sph_ens_config* c);

/* Creates an ensemble of n_boxes boxes.  Box b owns particles
 * [sum_{c<b} box_n[c], ... + box_n[b]) of the concatenated state; box_lo,
 * box_hi (3 per box) and box_periodic (3 per box) describe it, box_alpha[b] is
 * its viscosity coefficient (Eq. 5).  common: gamma, courant, dt_growth,
 * ng_target, max_nb, sinc_n and precision (must be SPH_FP32_MIXED) shared by
 * all boxes.  All pointers are HOST arrays.  Every box_n[b] must be >= 1 and
 * n_boxes >= 1 (SPH_ERR_INVALID_ARG otherwise).  Allocates the device scratch
 * (about 1 KB per particle at max_nb = 160). */
SPH_API int sph_ensemble_init(const sph_params* common, int n_boxes, const int64_t* box_n,
                              const double* box_lo, const double* box_hi,
                              const int* box_periodic, const double* box_alpha, sph_ens** out);
/* Synchronises the device and frees the ensemble's device scratch and graph. */
SPH_API void sph_ensemble_destroy(sph_ens* e);
/* Sets the tuning knobs for the next step or capture; SPH_ERR_INVALID_ARG for
 * a value outside the ranges above (the configuration is then unchanged). */
SPH_API int sph_ensemble_set_config(sph_ens* e, const sph_ens_config* c);

/* Advances every box by `steps` steps in one persistent launch.  state: the
 * concatenated state (device arrays, n = total particles; each box's range is
 * reordered in place as by sph_step); dt: DEVICE array of n_boxes doubles,
 * dt_{n-1} per box on entry (0 before the first step), dt_n on return. */
SPH_API int sph_ensemble_step(sph_ens* e, sph_state* state, double* dt, int steps,
                              sph_stream_t stream);

/* Captures the launch of sph_ensemble_step(state, dt, steps) into a CUDA graph
 * (stream must not be the legacy default stream); sph_ensemble_replay then
 * launches the graph, advancing the same arrays by `steps` more steps. */
SPH_API int sph_ensemble_capture(sph_ens* e, sph_state* state, double* dt, int steps,
                                 sph_stream_t stream);
SPH_API int sph_ensemble_replay(sph_ens* e, sph_stream_t stream);

/* Synchronises, returns the device error bits of all boxes (SPH_FLAG_*) in
 * *flags, clears them and re-arms the grid barrier. */
SPH_API int sph_ensemble_error_word(sph_ens* e, uint32_t* flags);
/* Message of the last failed call on e. */
SPH_API const char* sph_ensemble_last_error(const sph_ens* e);
/* out[0] particles, out[1] boxes, out[2] persistent CTAs, out[3] launches. */
SPH_API int sph_ensemble_info(const sph_ens* e, int64_t* out);
/* Phases of one ensemble step, in launch order (SPH_ENS_NPHASE of them). */
#define SPH_ENS_NPHASE 15
/* Milliseconds per phase (ms[SPH_ENS_NPHASE], HOST) accumulated over *steps
 * steps since the last call, measured on the device by block 0 between grid
 * barriers (the slowest block's time for each phase; with SPH_FLAG_TIMEOUT the
 * sums are partial).  Phases: reset, extent, grid, count, scan, cell items,
 * scatter, in-cell order, gather, find, density, IAD, momentum, dt, update.
 * Synchronises the device and clears the sums. */
SPH_API int sph_ensemble_phase_times(sph_ens* e, double* ms, int64_t* steps);

/* ------------------------------------------------------------------------ */
/* Differentiable rollout: the gradient of a scalar of the state after K     */
/* FP64 steps (plus one density pass on the final state) with respect to    */
/* the initial state and the viscosity alpha of Eq. 5, by hand-written       */
/* adjoint kernels of the update, momentum/energy (Eqs. 2-5), IAD and        */
/* density + EOS (Eq. 1).  The neighbour lists, smoothing lengths, time      */
/* steps and the viscosity switch of Eq. 5 are held at their values on the   */
/* forward trajectory: the result is the derivative of the rollout with      */
/* those frozen, which is the rollout's own derivative wherever none of them */
/* changes under a small perturbation.  The forward pass keeps a state       */
/* checkpoint every `checkpoint_every` steps; the backward pass re-runs each */
/* segment from its checkpoint, recording what the reverse kernels need,     */
/* then runs the segment's reverse steps.  Every reduction is in a fixed     */
/* order: two backward passes give bit-identical gradients.                  */
/* All pointers are DEVICE memory of the current device; calls are           */
/* asynchronous on `stream` except where stated.                             */
/* ------------------------------------------------------------------------ */
typedef struct sph_adj sph_adj;

/* Creates a rollout of `steps` >= 1 steps for states of up to n_max
 * particles; 1 <= checkpoint_every <= steps.  params->precision must be
 * SPH_FP64 and max_nb <= 4096.  Device memory is allocated here only:
 * per particle of n_max, (checkpoint_every + 1) * (192 + 4 max_nb) bytes of
 * tape, 112 bytes per checkpoint (ceil(steps / checkpoint_every) of them),
 * 120 * max_nb bytes of pair and reverse-list scratch and about 620 bytes
 * of working arrays, plus one FP64 sph_ctx. */
SPH_API int sph_adjoint_init(const sph_params* params, int64_t n_max, int steps,
                             int checkpoint_every, sph_adj** out);
/* Synchronises the device and frees the rollout's tape, checkpoints and context. */
SPH_API void sph_adjoint_destroy(sph_adj* a);

/* Runs the forward rollout from s0 (its 13 state arrays are read; id and the
 * output arrays are ignored and may be NULL; s0 is not modified) with the
 * previous time step dt_prev0 (0 = first step) and viscosity alpha.
 * final_out (8 n doubles) receives x, y, z, vx, vy, vz, u after the last
 * step and rho of the final density pass, each n long, particle i at index
 * i as in s0.  Synchronises the stream and reads the error word: returns
 * SPH_ERR_NB_OVERFLOW, SPH_ERR_SINGULAR_IAD or SPH_ERR_NONFINITE if a step
 * raised that flag (and SPH_ERR_INVALID_ARG for SPH_FLAG_BAD_BOX or
 * SPH_FLAG_CELL_OVERFLOW); the gradient is then not available. */
SPH_API int sph_adjoint_forward(sph_adj* a, const sph_state* s0, double dt_prev0, double alpha,
                                double* final_out, sph_stream_t stream);

/* Reverse pass of the last sph_adjoint_forward.  g_final (8 n doubles, the
 * layout of final_out) holds dL/d(final_out).  g_init (11 n doubles)
 * receives dL/d of the initial x, y, z, vx, vy, vz, vxh, vyh, vzh, u,
 * du_prev (in that order, particle order of s0); *g_alpha (one device
 * double) receives dL/dalpha.  Returns SPH_ERR_ORDER before a forward. */
SPH_API int sph_adjoint_backward(sph_adj* a, const double* g_final, double* g_init,
                                 double* g_alpha, sph_stream_t stream);

/* out[0] device bytes held, out[1] kernel launches so far, out[2] steps
 * re-run from checkpoints so far, out[3] backward passes so far (HOST). */
SPH_API int sph_adjoint_info(const sph_adj* a, int64_t* out);
/* The `steps` time steps of the last forward into dt (HOST).  Synchronous. */
SPH_API int sph_adjoint_time_steps(sph_adj* a, double* dt);
SPH_API const char* sph_adjoint_last_error(const sph_adj* a);

/* Stages of sph_step timed by sph_profile. */
enum {
  SPH_STAGE_SORT = 0,     /* grid, Morton counting sort, both gather
                             parts (the second runs after the search)   */
  SPH_STAGE_FIND = 1,     /* neighbour lists                             */
  SPH_STAGE_DENSITY = 2,  /* density + EOS                               */
  SPH_STAGE_IAD = 3,      /* IAD matrix                                  */
  SPH_STAGE_MOMENTUM = 4, /* momentum and energy                         */
  SPH_STAGE_DT = 5,       /* global time step                            */
  SPH_STAGE_UPDATE = 6,   /* integrator, h, conservation sums            */
  SPH_NSTAGE = 7
};

/* Enables (1) or disables (0) per-stage timing of sph_step with CUDA events
 * recorded on the step's stream (the events add no synchronisation). */
SPH_API int sph_profile(sph_ctx* ctx, int enable);

/* Accumulated milliseconds per stage (ms[SPH_NSTAGE], HOST) over the steps
 * timed since the last call, and their number in *steps; then resets.
 * Synchronises on the last recorded event. */
SPH_API int sph_stage_times(sph_ctx* ctx, double* ms, int64_t* steps);

/* Cumulative device counters since sph_init (synchronous read), HOST array
 * of 6:
 * out[0] (target, candidate) pairs tested by the neighbour search,
 * out[1] of which decided by the exact FP64 criterion (inside the FP32
 *        prefilter's error margin),
 * out[2] neighbour pairs found by sph_step (sum over steps of sum_a nn_a),
 * out[3] particle updates done by sph_step (sum over steps of n),
 * out[4] staged candidate slots recorded by the SPH_PAIRS_STAGED search
 *        (sum over cells of S, one 4-byte entry each),
 * out[5] hit-mask words it wrote (sum over cells of na ceil(S / 64), 8 bytes
 *        each). */
SPH_API int sph_stats(sph_ctx* ctx, uint64_t* out);

/* The FP32 fused-multiply-add rate of the current device in TFLOP/s,
 * measured by the library's own kernel: every thread of SMs x 8 blocks of 256
 * runs 8 independent chains of 65,536 dependent FFMAs, timed with CUDA events
 * on `stream` after one untimed launch (2 flops per FFMA).  It is the
 * measured denominator of the FP32-pipe roofline of the pair sums.  The paper
 * has no counterpart; it is a measurement utility.  Synchronous; allocates
 * nothing but two events.  Returns SPH_OK, SPH_ERR_INVALID_ARG (NULL
 * tflops) or SPH_ERR_CUDA. */
SPH_API int sph_measure_fp32_peak(double* tflops, sph_stream_t stream);

/* Number of kernels the library launched on this context so far. */
SPH_API int64_t sph_launch_count(const sph_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
