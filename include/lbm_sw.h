/*
 * lbm_sw.h — C ABI of the GB300 (sm_103a) library for the vectorial lattice
 * Boltzmann schemes of F. Dubois, "Simulation of strong nonlinear waves with
 * vectorial lattice Boltzmann schemes" (DSFD 2013), applied to the shallow-water
 * equations:
 *
 *   1D: the D1Q3Q2 scheme of section 2 — populations f on D1Q3 (velocities
 *       0, +lambda, -lambda) carry the depth h, populations g on D1Q2
 *       (+lambda, -lambda) carry the discharge h u.
 *   2D: the D2Q5Q4Q4 scheme of section 3 — f on D2Q5 (Eq. 3-stencil-d2q5),
 *       gx and gy on D2Q4 (no rest population), carrying h, h u and h v.
 *
 * Equilibria are the derivatives of the potentials h_j^* of the kinetic
 * decomposition of the dual entropy (section 1; Eqs. 2-potentiels-st-venant-1d,
 * 2-potentiels-st-venant-1d-suite, 3-st-venant-contraintes-2, 3-st-venant-enplus),
 * with p = g h^2 / 2 (the gamma = 2 system), and the collision is the BGK form of
 * Eq. 2-relaxation (every rate equal to s).  Streaming moves each population one
 * cell per step (lambda = dx/dt).  The 2D BGK kernels evaluate f + s (f^eq - f) as
 * (1 - s) f + s f^eq with s folded into the equilibrium's constants: the same
 * operator, with 13 operations fewer per cell; a state at equilibrium settles within
 * about one unit in the last place of itself instead of mapping to itself bit for bit
 * (the MRT form, lbm_sw_set_relaxation, relaxes f^eq - f and keeps that fixed point).
 *
 * Every compute step runs in hand-written CUDA kernels on the caller's stream;
 * there is no CPU fallback.  No function throws; every function that can fail
 * returns a status code (LBM_SW_OK = 0 or a negative LBM_SW_E_*), and the handle
 * keeps a message for the last failure (lbm_sw_last_error).  Many handles may
 * coexist; the library keeps no global state.
 *
 * Layouts at this boundary
 *   - Moment fields (h, hu, hv) are FP64 arrays of nx*ny values, row-major
 *     [ny][nx], x fastest, in either precision mode (conversion happens on the
 *     device).  In 1D, ny = 1 and hv is ignored (may be NULL).
 *   - Raw populations are dense planes [q][ny][nx] of the handle's precision
 *     (float or double), q = 5 in 1D (f0, f+, f-, g+, g-) and 13 in 2D
 *     (f0 f1 f2 f3 f4 gx1 gx2 gx3 gx4 gy1 gy2 gy3 gy4, v1 = (lambda,0),
 *     v2 = (0,lambda), v3 = (-lambda,0), v4 = (0,-lambda)).
 *   - "on_device" = 1: the pointer is device memory of the current CUDA device
 *     (e.g. a torch tensor's data_ptr), 0: host memory (pageable or pinned).
 *     Caller-owned in both cases; the library never frees caller memory.
 *
 * State convention: the library stores post-collision populations, the values
 * that stream out of each cell at the next step.  A collision conserves h, h u
 * and h v, so the moments of the stored state are those of the current time
 * level.
 */
#ifndef LBM_SW_H
#define LBM_SW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_SW_ABI_VERSION 1

#if defined(__GNUC__)
#define LBM_SW_API __attribute__((visibility("default")))
#else
#define LBM_SW_API
#endif

/* Opaque handle: one simulation (parameters, two device population buffers, the
 * caller's stream, scratch for reductions).  Owned by the library; create with
 * lbm_sw_create, release with lbm_sw_destroy. */
typedef struct lbm_sw lbm_sw;

/* ---- status codes ---- */
#define LBM_SW_OK 0
#define LBM_SW_E_ARG (-1)      /* invalid argument (NULL, size, parameter out of range) */
#define LBM_SW_E_CUDA (-2)     /* a CUDA call failed; see lbm_sw_last_error */
#define LBM_SW_E_UNSTABLE (-3) /* a diagnostic found NaN/Inf or a depth h <= 0 */
/* (-4 is not used: no kernel of this library waits on a flag or on another grid) */
#define LBM_SW_E_STATE (-5)    /* call not valid in the handle's state (e.g. no state set) */
#define LBM_SW_E_NOMEM (-6)    /* device allocation failed */

/* ---- boundary kinds (section 3, last paragraph: bounce-back and anti-bounce-back) ----
 * The ghost cell beyond a side holds
 *   PERIODIC: the cell on the opposite side (the opposite side must be PERIODIC too);
 *   WALL:     the mirror image of the boundary cell: the incoming population takes
 *             the post-collision value of its reflected partner at the same cell,
 *             with the momentum family normal to the wall negated (slip wall, zero
 *             normal flux, exact mass conservation);
 *   OUTFLOW:  a copy of the boundary cell (zero-gradient open boundary);
 *   INFLOW:   the equilibrium of the prescribed state inflow[side] = (h, hu, hv). */
#define LBM_SW_BC_PERIODIC 0
#define LBM_SW_BC_WALL 1
#define LBM_SW_BC_OUTFLOW 2
#define LBM_SW_BC_INFLOW 3

/* sides, in the order of lbm_sw_params.bc */
#define LBM_SW_SIDE_XM 0
#define LBM_SW_SIDE_XP 1
#define LBM_SW_SIDE_YM 2
#define LBM_SW_SIDE_YP 3

/* storage and arithmetic precision of the populations */
#define LBM_SW_FP32 0
#define LBM_SW_FP64 1

/* form of populations handed to lbm_sw_set_populations */
#define LBM_SW_POST_COLLISION 0 /* stored as given */
#define LBM_SW_PRE_COLLISION 1  /* collided on the device first (moments, equilibria, relaxation) */

/* step kernel variants */
#define LBM_SW_KERNEL_AUTO 0    /* library choice: TEMPORAL for 2D FP32 grids of >= 3 * 2^17 cells
                                   (628^2 and up) with every side periodic or an even
                                   temporal_steps (with MRT relaxation: >= 2^19 cells), else VEC in
                                   2D; CLUSTER in 1D */
#define LBM_SW_KERNEL_SIMPLE 1  /* one launch per step, one thread per cell, scalar loads */
#define LBM_SW_KERNEL_VEC 2     /* 2D: 16-byte vectors along x (4 FP32 or 2 FP64 cells per thread),
                                   x-neighbours exchanged with warp shuffles */
#define LBM_SW_KERNEL_CLUSTER 3 /* 1D: all n steps of lbm_sw_step in one thread-block-cluster
                                   launch, the line held in shared memory (up to 16384 cells on a
                                   GB300; longer lines use SIMPLE) */
#define LBM_SW_KERNEL_TEMPORAL 4 /* 2D FP32: temporal_steps steps per launch (temporal
                                    blocking: a row wavefront through shared memory, 104/k bytes of
                                    HBM traffic per cell update plus halos), BGK, or MRT with an even
                                    temporal_steps; the tail of n runs as shorter fused launches
                                    (lbm_sw_step), obstacles use their own kernel; results equal
                                    VEC bit for bit */

typedef struct lbm_sw_params {
  int dim;             /* 1 (D1Q3Q2) or 2 (D2Q5Q4Q4) */
  int nx, ny;          /* cells; ny must be 1 when dim == 1; nx, ny >= 1 */
  int precision;       /* LBM_SW_FP32 or LBM_SW_FP64 */
  double g;            /* gravity, > 0 (p = g h^2 / 2) */
  double lambda;       /* lattice velocity dx/dt, > 0 */
  double s;            /* BGK relaxation rate, 0 <= s < 2 */
  double a;            /* weight of the rest potential h_0^* = (a/2) K theta^2, >= 0 */
  int bc[4];           /* LBM_SW_BC_* for sides x-, x+, y-, y+ (y sides unused in 1D) */
  double inflow[4][3]; /* (h, hu, hv) imposed on INFLOW sides */
  void* stream;        /* cudaStream_t borrowed from the caller (NULL = legacy default) */
  int kernel;          /* LBM_SW_KERNEL_*: AUTO, SIMPLE, VEC or TEMPORAL (2D), CLUSTER (1D) */
  int graph_chunk;     /* steps per captured CUDA graph in lbm_sw_step; 0 = default, < 0 = off */
  int temporal_steps;  /* steps fused per launch by the TEMPORAL kernel: 2 .. 8; 0 = default (4 below
                          2^20 cells, else 6) */
  int reserved[5];     /* must be zero */
} lbm_sw_params;

typedef struct lbm_sw_info {
  int q;                     /* populations per cell: 5 (1D) or 13 (2D) */
  int kernel;                /* step kernel variant in use */
  size_t pitch;              /* elements per stored row (multiple of 32) */
  size_t population_bytes;   /* bytes of one dense population set, q * nx * ny * sizeof(T) */
  double bytes_per_update;   /* algorithmic DRAM bytes per lattice-cell update: 2 q sizeof(T) */
  long long steps_done;      /* steps taken since the last set_state / set_populations */
  long long kernel_launches; /* kernels this handle has launched */
  int steps_per_launch;      /* steps one step-kernel launch advances: temporal_steps where
                                TEMPORAL fuses steps (see LBM_SW_KERNEL_TEMPORAL), 0 for CLUSTER
                                (all n steps of lbm_sw_step in one launch), else 1 */
} lbm_sw_info;

/* Fill *p with defaults: dim 2, FP32, g = 1, lambda = 8, s = 1.8, a = 0.05,
 * periodic sides, NULL stream, automatic kernel choice, nx = ny = 0 (must be set).
 * Returns LBM_SW_E_ARG if p is NULL. */
LBM_SW_API int lbm_sw_params_init(lbm_sw_params* p);

/* Validate *p, allocate two pitched population buffers (double buffering, 256-byte
 * aligned planes) on the current device, and return a handle in *out.  The
 * populations start undefined: call lbm_sw_set_state or lbm_sw_set_populations.
 * Errors: LBM_SW_E_ARG (NULL, sizes, parameter ranges, mismatched periodic sides,
 * nonzero reserved fields), LBM_SW_E_NOMEM, LBM_SW_E_CUDA; *out is then NULL. */
LBM_SW_API int lbm_sw_create(const lbm_sw_params* p, lbm_sw** out);

/* Release the handle and its device memory (synchronises its stream). NULL-safe.
 * A utility of the library: no passage of the paper corresponds to it. */
LBM_SW_API void lbm_sw_destroy(lbm_sw* h);

/* Set the populations to the equilibrium of W = (h, hu, hv) (paper: the state at
 * t = 0 is taken at equilibrium, f = f^eq(W)).  Arrays: FP64 [ny][nx]; hv ignored in
 * 1D.  Host arrays are copied before return; device arrays must stay valid until the
 * stream reaches this work.  Errors: LBM_SW_E_ARG, LBM_SW_E_CUDA. */
LBM_SW_API int lbm_sw_set_state(lbm_sw* h, const double* depth, const double* hu, const double* hv, int on_device);

/* Advance n >= 0 time steps (each: streaming with the boundary rules, moments,
 * equilibria, relaxation), asynchronously on the handle's stream.  How the steps map to
 * kernel launches depends on the kernel in use (lbm_sw_get_info):
 *   TEMPORAL: fused launches of up to temporal_steps = K steps each (temporal blocking):
 *             launches of K while more than K + 8 steps remain, then the cheapest split of
 *             the rest into launches of at most K steps (K and even counts always; other
 *             odd counts above one only on BGK grids with every side periodic; at most one
 *             single step), e.g. 20 = 6 + 6 + 4 + 4 at K = 6;
 *             lbm_sw_step_plan lists the launches;
 *   CLUSTER:  one launch for all n steps (1D lines up to 16384 cells);
 *   VEC, SIMPLE, obstacles: one launch per step; long runs replay a captured CUDA graph of
 *             graph_chunk steps.
 * Every mapping gives the same bits.  Errors: LBM_SW_E_ARG (n < 0), LBM_SW_E_STATE (no
 * state set), LBM_SW_E_CUDA (launch failure; kernel faults surface at the next
 * synchronising call). */
LBM_SW_API int lbm_sw_step(lbm_sw* h, int n);

/* The kernel launches lbm_sw_step(h, n) would make now: writes the steps each launch
 * advances, in order, to sizes[0 .. min(count, max_sizes) - 1] and returns count (the
 * number of launches; 0 for n = 0).  A utility of the library (no passage of the paper
 * corresponds to it); launches nothing.  Errors: LBM_SW_E_ARG (NULL handle, n < 0,
 * max_sizes < 0, or sizes NULL with max_sizes > 0). */
LBM_SW_API int lbm_sw_step_plan(const lbm_sw* h, int n, int* sizes, int max_sizes);

/* Relax each moment at its own rate: the MRT form of Eq. 2-relaxation,
 * m*_l = m_l + s_l (m_l^eq - m_l), on the moment bases the paper gives.  rates[count]:
 *   2D (count 13): rho, J_x, J_y, eps_rho, XX_rho, q_x, f_xx, f_xy, XX_u, q_y, f_yx, f_yy, XX_v
 *                  (section 3; J_x = lam (f1 - f3), eps_rho = f1 + f2 + f3 + f4 - 4 f0, ...);
 *   1D (count 5):  rho, J_rho, eps_rho, q, J_q (section 2; eps_rho = lam^2 (f+ + f- - 2 f0)).
 * The entries of the conserved moments (rho, q_x, q_y / rho, q) are ignored.  Every other
 * rate must lie in [0, 2); all equal to s reproduces the BGK step up to rounding.
 * rates == NULL returns to BGK with the rate s of the parameters.  Applies to the following
 * steps and to lbm_sw_set_populations(PRE_COLLISION).  The adjoint (lbm_sw_tape_create)
 * supports BGK only.  Errors: LBM_SW_E_ARG. */
LBM_SW_API int lbm_sw_set_relaxation(lbm_sw* h, const double* rates, int count);

/* Obstacles inside a 2D domain (section 4, second test case: a forward-facing step in the
 * channel).  solid[ny][nx] (x fastest, one byte per cell, nonzero = solid) is copied;
 * on_device says whether it is a device pointer; the caller keeps ownership and may reuse it
 * when the call returns.  A face between a fluid cell and a solid cell (inside the domain or
 * across a periodic side) is a wall with the rule of a WALL side: the population that
 * would arrive from the solid cell takes the value of the fluid cell's own reflected
 * population, the momentum family normal to the face negated.  Solid cells hold no fluid:
 * they are not collided or streamed and keep the populations they hold (also through
 * lbm_sw_set_populations(PRE_COLLISION)); their moments still count in the diagnostics.
 * With obstacles every step runs an obstacle kernel, one step per launch: the vectorised row
 * kernel (warps with no solid cell near them take the plain path), or one thread per cell
 * when the params' kernel is SIMPLE; both give the same bits.  solid == NULL removes the
 * obstacles.  The adjoint does not support them.
 * Errors: LBM_SW_E_ARG (1D handle), LBM_SW_E_NOMEM, LBM_SW_E_CUDA. */
LBM_SW_API int lbm_sw_set_obstacle(lbm_sw* h, const unsigned char* solid, int on_device);

/* Write the conserved moments (h = sum f, hu = sum gx, hv = sum gy; Eq.
 * 1-hyp-N-vconserv) of the current state as FP64 [ny][nx] arrays.  With host
 * arrays the call synchronises; with device arrays it is asynchronous on the stream.
 * hv may be NULL (and is ignored in 1D). */
LBM_SW_API int lbm_sw_get_moments(lbm_sw* h, double* depth, double* hu, double* hv, int on_device);

/* Reduce the current state on the device (FP64 accumulation, warp shuffles, then a
 * fixed-order second pass) and synchronise: out[0] = sum h, out[1] = sum hu,
 * out[2] = sum hv (0 in 1D), out[3] = min h.  Returns LBM_SW_E_UNSTABLE when any
 * cell holds NaN/Inf or h <= 0 (out is still written). */
LBM_SW_API int lbm_sw_diagnostics(lbm_sw* h, double out[4]);

/* Copy the stored (post-collision) populations out as dense planes [q][ny][nx] of
 * the handle's precision; lbm_sw_get_info gives the byte count.  Synchronises for
 * host memory.  A utility of the library (checkpoints, parity checks): no passage of the
 * paper corresponds to it. */
LBM_SW_API int lbm_sw_get_populations(lbm_sw* h, void* dst, int on_device);

/* Load dense planes [q][ny][nx] of the handle's precision.  form =
 * LBM_SW_POST_COLLISION stores them as they are (a checkpoint written by
 * lbm_sw_get_populations); LBM_SW_PRE_COLLISION collides them on the device first
 * (Eq. 2-relaxation with the equilibria of sections 2-3), so that the next step streams
 * their post-collision values.  The `form` argument extends the population exchange of
 * the plain set/get pair: it lets a caller start from arbitrary (non-equilibrium)
 * populations as the oracle does.  A utility of the library otherwise: no passage of the
 * paper corresponds to loading raw populations. */
LBM_SW_API int lbm_sw_set_populations(lbm_sw* h, const void* src, int on_device, int form);

/* ---- Rows of a 2D state: domain decomposition across GPUs ----
 * One grid split into bands of rows, one band per GPU: each band's handle holds its rows
 * plus H ghost rows on every side that borders another band.  Streaming moves every
 * population one cell per step (section 3, Eq. 3-stencil-d2q5), so k <= H steps change
 * the ghost rows' influence only k rows deep: after k steps the band's own rows are exact,
 * and copying the neighbours' outermost H rows into the ghost rows restores the state
 * (paper_1401_0427_gb300/decomposition.py drives this over torch.distributed).
 *
 * lbm_sw_get_rows / lbm_sw_set_rows copy rows [y0, y0 + nrows) of every population plane
 * of the stored state out to / in from dense planes [q][nrows][nx] of the handle's
 * precision (on_device as elsewhere; host copies synchronise).  lbm_sw_diagnostics_rows
 * is lbm_sw_diagnostics over rows [y0, y0 + nrows) only (the band without its ghost rows).
 * Errors: LBM_SW_E_ARG (1D handle for the copies, rows outside [0, ny), NULL pointers),
 * LBM_SW_E_STATE (no state set), LBM_SW_E_CUDA; LBM_SW_E_UNSTABLE as lbm_sw_diagnostics. */
LBM_SW_API int lbm_sw_get_rows(lbm_sw* h, int y0, int nrows, void* dst, int on_device);
LBM_SW_API int lbm_sw_set_rows(lbm_sw* h, int y0, int nrows, const void* src, int on_device);
LBM_SW_API int lbm_sw_diagnostics_rows(lbm_sw* h, int y0, int nrows, double out[4]);

/* ---- Batched instances ----
 * Many independent D2Q5Q4Q4 grids of uneven sizes (e.g. an ensemble of dam-breaks), all with
 * the same scheme parameters and boundary kinds, advanced together: one kernel launch per
 * time step walks a list of tiles (rows x 32 vectors) covering every instance, either one CTA
 * per tile or a persistent grid of a few CTAs per SM striding through the list,
 * and long runs replay a CUDA graph of graph_chunk steps; FP32 batches fuse temporal_steps
 * steps per launch instead (temporal blocking).  Each instance evolves exactly as
 * it would in its own lbm_sw handle (same device arithmetic, bit for bit).  Tile shape and
 * schedule come from lbm_sw_batch_autotune (or the params).  All instances share two device
 * buffers (double buffering); instance i stores its planes like a single handle does
 * (pitch = nx rounded up to 32 elements, 256-byte aligned planes). */
typedef struct lbm_sw_batch lbm_sw_batch;

typedef struct lbm_sw_batch_params {
  int count;              /* instances, 1 .. 65536 */
  const int* nx;          /* count widths (host array, copied by create), each >= 1 */
  const int* ny;          /* count heights (host array, copied by create), each >= 1 */
  int precision;          /* LBM_SW_FP32 or LBM_SW_FP64 */
  double g, lambda, s, a; /* as in lbm_sw_params */
  int bc[4];              /* boundary kinds shared by every instance */
  double inflow[4][3];    /* (h, hu, hv) of INFLOW sides */
  void* stream;           /* cudaStream_t borrowed from the caller */
  int tile_rows;          /* rows per CTA tile: 1, 2, 4 or 8; 0 = default (4) */
  int ctas_per_sm;        /* persistent CTAs per SM, 1 .. 32; 0 = one CTA per tile (default) */
  int graph_chunk;        /* steps per captured CUDA graph; 0 = default (50), < 0 = off */
  int temporal_steps;     /* steps fused per launch (temporal blocking, FP32; an even value
                             unless every side is periodic): 2 .. 8; 1 = one step per launch;
                             0 = default (6 in FP32, else 1; lbm_sw_batch_autotune may change it) */
  int reserved[4];        /* must be zero */
} lbm_sw_batch_params;

typedef struct lbm_sw_batch_tuning {
  int tile_rows;          /* chosen rows per tile */
  int ctas_per_sm;        /* chosen persistent CTAs per SM (0: one CTA per tile) */
  int candidates;         /* configurations timed by the last autotune (0 if none) */
  double ms_per_step;     /* time per step of the chosen configuration (0 if not timed) */
  long long tiles;        /* tiles in the work list */
  long long cells;        /* cells over all instances */
  int temporal_steps;     /* steps fused per launch (1: one step per launch) */
} lbm_sw_batch_tuning;

/* Defaults as for lbm_sw_params_init (count = 0, nx = ny = NULL must be set). */
LBM_SW_API int lbm_sw_batch_params_init(lbm_sw_batch_params* p);

/* Validate, allocate the two shared buffers and the tile list.  Errors as lbm_sw_create
 * (message from lbm_sw_create_error). */
LBM_SW_API int lbm_sw_batch_create(const lbm_sw_batch_params* p, lbm_sw_batch** out);

/* Release the batch (synchronises its stream).  NULL-safe. */
LBM_SW_API void lbm_sw_batch_destroy(lbm_sw_batch* b);

/* Equilibrium state f = f^eq(W) of one instance (arrays FP64 [ny_i][nx_i]; hv may be NULL
 * for host input: zero).  Every instance needs a state before lbm_sw_batch_step. */
LBM_SW_API int lbm_sw_batch_set_state(lbm_sw_batch* b, int instance, const double* depth, const double* hu,
                                      const double* hv, int on_device);

/* Advance every instance n >= 0 steps: with temporal_steps = K >= 2, one launch of a
 * work list of wavefronts (instance, column strip, row segment; the units balanced over one
 * wave of resident CTAs) per K steps, the rest of n one tile-list launch per step; else
 * one tile-list launch per step.  Results equal one step per launch bit for bit.  Errors:
 * LBM_SW_E_ARG, LBM_SW_E_STATE (an instance has no state), LBM_SW_E_CUDA. */
LBM_SW_API int lbm_sw_batch_step(lbm_sw_batch* b, int n);

/* Moments of one instance (as lbm_sw_get_moments). */
LBM_SW_API int lbm_sw_batch_get_moments(lbm_sw_batch* b, int instance, double* depth, double* hu, double* hv,
                                        int on_device);

/* Post-collision populations of one instance, dense [13][ny_i][nx_i] of the batch precision. */
LBM_SW_API int lbm_sw_batch_get_populations(lbm_sw_batch* b, int instance, void* dst, int on_device);

/* FP64 totals of one instance (as lbm_sw_diagnostics, including LBM_SW_E_UNSTABLE). */
LBM_SW_API int lbm_sw_batch_diagnostics(lbm_sw_batch* b, int instance, double out[4]);

/* Time trial_steps launches (>= 1) of every candidate tile shape (1, 2, 4, 8 rows) and
 * schedule (one CTA per tile, or 2, 4, 8 persistent CTAs per SM) of the one-step kernel and,
 * when the params left temporal_steps at 0 and the batch allows it, of the temporal kernel
 * at K = 4, 6 and 8 steps per launch (per step: launch time / K); keep the fastest per
 * step, and report it.  The trials read the current state and write the spare buffer, so
 * the state does not change.  Needs every instance's state.  Synchronises. */
LBM_SW_API int lbm_sw_batch_autotune(lbm_sw_batch* b, int trial_steps, lbm_sw_batch_tuning* out);

/* The tile shape and schedule in use. */
LBM_SW_API int lbm_sw_batch_get_tuning(const lbm_sw_batch* b, lbm_sw_batch_tuning* out);

/* Message of the last failure on this batch ("" if none). */
LBM_SW_API const char* lbm_sw_batch_last_error(const lbm_sw_batch* b);

/* ---- Discrete adjoint (gradients through time, 2D) ----
 * For a loss L(W^T) of the moments after T steps, the adjoint of the fused step gives
 * dL/dW^0 of the discrete scheme exactly (up to rounding):
 *   Phi^T = M^T dL/dW^T,  Phi^{n-1} = J_C(W^{n-1})^T S^T Phi^n,  dL/dW^0 = D(W^0)^T Phi^0,
 * where S is the streaming with the boundary rules (its transpose pulls in the reverse
 * direction), M sums each family, D = df^eq/dW (the equilibria of section 3) and
 * J_C = (1 - s) I + s D M is the Jacobian of the BGK collision (Eq. 2-relaxation).  A tape
 * stores the state every `interval` steps (about sqrt(T) by default) in FP64; the backward
 * pass replays each segment from its checkpoint (bit for bit: widening FP32 to FP64 is
 * exact), keeping only the moments W^n (3 planes per step), then runs the adjoint steps.
 * Phi and the replay use the handle's precision.  The tape owns all of its memory; the
 * handle's own state is not touched by lbm_sw_adjoint. */
typedef struct lbm_sw_tape lbm_sw_tape;

typedef struct lbm_sw_tape_info {
  int steps;               /* T */
  int interval;            /* steps between checkpoints */
  int checkpoints;         /* ceil(T / interval) */
  int recorded;            /* 1 after lbm_sw_forward_record */
  size_t checkpoint_bytes; /* FP64 checkpoint storage */
  size_t replay_bytes;     /* moments of one segment, two adjoint and two replay buffers */
} lbm_sw_tape_info;

/* Tape for `steps` >= 1 steps of 2D handle h, checkpoints every `interval` steps
 * (0 = ceil(sqrt(steps))).  Errors: LBM_SW_E_ARG (1D handle, bad counts), LBM_SW_E_NOMEM. */
LBM_SW_API int lbm_sw_tape_create(lbm_sw* h, int steps, int interval, lbm_sw_tape** out);

/* Release a tape (synchronises the owner's stream).  NULL-safe. */
LBM_SW_API void lbm_sw_tape_destroy(lbm_sw_tape* t);

/* Advance h by the tape's steps from its current state (its W^0 is the state at this
 * call), storing the checkpoints.  Errors: LBM_SW_E_ARG (tape of another handle),
 * LBM_SW_E_STATE (no state), LBM_SW_E_CUDA. */
LBM_SW_API int lbm_sw_forward_record(lbm_sw* h, lbm_sw_tape* t);

/* Given dL/dW^T (g_h required, g_hu and g_hv may be NULL = 0; FP64 [ny][nx]), write
 * dL/dW^0 (d_h required, d_hu and d_hv may be NULL).  on_device selects device or host
 * pointers for all six arrays; host calls synchronise.  Errors: LBM_SW_E_STATE (not
 * recorded), LBM_SW_E_ARG, LBM_SW_E_CUDA. */
LBM_SW_API int lbm_sw_adjoint(lbm_sw* h, lbm_sw_tape* t, const double* g_h, const double* g_hu, const double* g_hv,
                              double* d_h, double* d_hu, double* d_hv, int on_device);

/* Sizes of a tape. */
LBM_SW_API int lbm_sw_tape_get_info(const lbm_sw_tape* t, lbm_sw_tape_info* out);

/* Message of the last failure on this tape ("" if none). */
LBM_SW_API const char* lbm_sw_tape_last_error(const lbm_sw_tape* t);

/* Allocation-free diagnostics (the paper has no counterpart: this is a service of the
 * library, not a step of the scheme).  Some callers cannot allocate device memory at the
 * moment they need a health check of a state: a caller whose memory manager owns the whole
 * device and forbids allocations outside it, a caller with a fixed device-memory budget
 * fixed at start-up, or a caller that has just hit an out-of-memory error and wants to know
 * whether the state it still holds is sound.  This entry point computes the same numbers as
 * lbm_sw_diagnostics without any allocation: no cudaMalloc, no cudaFree, no allocating
 * library routine.
 *
 * Input: populations, a device pointer to q planes (q = 5 in 1D, 13 in 2D, the population
 * order above) of the given precision, each ny rows of row_pitch elements (row_pitch >= nx),
 * planes plane_pitch elements apart (plane_pitch >= row_pitch * ny); dense planes from
 * lbm_sw_get_populations have row_pitch = nx and plane_pitch = nx * ny.  Output: out, a
 * device pointer to 5 doubles, written asynchronously on `stream` (a cudaStream_t, NULL =
 * legacy default): sum h, sum hu, sum hv (0 in 1D), min h, and the number of cells with
 * NaN/Inf or h <= 0 (the call does not synchronise, so it reports that count in out[4]
 * instead of returning LBM_SW_E_UNSTABLE).  Totals are accumulated in FP64.
 *
 * Limit: ny <= LBM_SW_NOALLOC_MAX_ROWS (one partial per row lives in a static device array
 * of 8192 * 5 doubles = 327,680 bytes, which every GPU that loads this library holds until the
 * process exits).  Larger ny, NULL pointers, bad sizes or pitches return LBM_SW_E_ARG without
 * launching anything; a failed CUDA call returns LBM_SW_E_CUDA.
 *
 * Every call looks up the device address of the static array in the current context
 * (cudaGetSymbolAddress; not cached, so a device reset or a second context of the device
 * gets the address of its own copy).  The first call in a context loads the library's
 * device code there: make that first call before any stream capture.  All calls share the array
 * and each call fully rewrites the part it reads, so nothing needs clearing between calls;
 * calls whose work overlaps on the GPU (different streams, or different threads) race on the
 * array and must be serialised by the caller. */
#define LBM_SW_NOALLOC_MAX_ROWS 8192
LBM_SW_API int lbm_sw_diagnostics_noalloc(const void* populations, int dim, int precision, int nx, int ny,
                                          size_t row_pitch, size_t plane_pitch, double* out, void* stream);

/* Wait for all work queued by the handle; returns LBM_SW_E_CUDA on a kernel fault. */
LBM_SW_API int lbm_sw_synchronize(lbm_sw* h);

/* Sizes and counters of the handle. */
LBM_SW_API int lbm_sw_get_info(const lbm_sw* h, lbm_sw_info* out);

/* Message of the last failure on this handle ("" if none); valid until the next call.
 * Utilities from here on: no passage of the paper corresponds to them. */
LBM_SW_API const char* lbm_sw_last_error(const lbm_sw* h);

/* Message of the last failed lbm_sw_create on the calling thread ("" if it succeeded). */
LBM_SW_API const char* lbm_sw_create_error(void);

/* Static text for a status code. */
LBM_SW_API const char* lbm_sw_status_string(int status);

/* LBM_SW_ABI_VERSION of the loaded library. */
LBM_SW_API int lbm_sw_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_SW_H */
