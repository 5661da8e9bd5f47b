/*
 * sac.h -- C ABI of the B300 SAC-family 2D ideal-MHD step (arXiv 1710.06423),
 * with batched runs, a learned coarse-grid correction and a 3D form (sac3_*).
 *
 * The library advances the 2D ideal-MHD equations of section 2 of the paper
 * (mass, momentum, energy and induction in conservative form, total pressure
 * p_t = p_k + B^2/2, kinetic pressure p_k = (gamma-1)(e - rho v^2/2 - B^2/2),
 * units with mu0 = 1) in perturbation/background split form, with the
 * section 2 numerics: fourth-order central differences of the fluxes,
 * hyper-diffusion / hyper-resistivity scaled by the maximum wave speed plus a
 * compression-activated shock viscosity, and classical fourth-order
 * Runge-Kutta stepping whose CFL step comes from a grid-wide maximum of the
 * signal speed.  Every step runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *   - Return value: SAC_OK (0) or a negative SAC_ERR_* code; sac_last_error()
 *     gives a one-line description of the last failure of a context.
 *   - State arrays are conserved PERTURBATION variables, field-major,
 *     w[f][j][i] with f in (rho~, m_x, m_y, e~, B~_x, B~_y), j the row (y) and
 *     i the column (x, fastest), nx*ny cells per field, no ghost cells.
 *     Background arrays are bg[f][j][i] with f in (rho_b, e_b, B_bx, B_by).
 *     With no background the perturbations are the full variables.
 *   - Host buffers belong to the caller; the library copies in and out and
 *     keeps no host pointer after the call returns.  Device memory of a
 *     context belongs to the context and is released by sac_free().
 *   - A context is bound to one device and one CUDA stream (params.stream,
 *     NULL = the legacy default stream).  Calls on one context are not thread
 *     safe.  Calls marked ASYNC only enqueue work on that stream.
 *   - Errors found on the device (non-finite state or step) are recorded in
 *     the context and reported by the next synchronising call
 *     (sac_run_to, sac_step, sac_get_state*, sac_dt, sac_time, sac_cmax,
 *     sac_sums, sac_divb, sac_sync).
 *     After SAC_ERR_NONFINITE the state is left as computed, for inspection,
 *     and further steps are skipped until sac_set_state*.
 */
#ifndef SAC_H
#define SAC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sac_ctx sac_ctx;

enum {
    SAC_OK = 0,
    SAC_ERR_ARG = -1,        /* invalid argument or parameter */
    SAC_ERR_STATE = -2,      /* call out of order (e.g. step before set_state) */
    SAC_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    SAC_ERR_OOM = -4,        /* device allocation failed */
    SAC_ERR_NONFINITE = -5,  /* the state or the CFL step became NaN/Inf or dt <= 0 */
    SAC_ERR_TIMEOUT = -6     /* a bounded device wait gave up */
};

enum { SAC_BC_PERIODIC = 0, SAC_BC_FIXED = 1, SAC_BC_OUTFLOW = 2 };
enum { SAC_FP64 = 0, SAC_FP32 = 1 };

/*
 * Run parameters (section 2 numerics; section 5 test problems).
 *   nx, ny            interior cells (ny = 1 for a 1D run); 1 <= nx, ny <= 65536
 *   x0,x1,y0,y1       domain; cell-centred grid, dx = (x1-x0)/nx, dy = (y1-y0)/ny
 *   gamma             adiabatic index (> 1)
 *   courant           CFL number C of dt = C min(dx/cmax_x, dy/cmax_y)
 *   bc_x, bc_y        SAC_BC_*: periodic = wrapped interior; outflow = nearest
 *                     interior cell of the current stage; fixed = nearest
 *                     interior cell of the state given to sac_set_state, held
 *   precision         SAC_FP64: all arithmetic in FP64, same operation order as
 *                     the FP64 oracle.  SAC_FP32: stencil arithmetic and storage
 *                     in FP32 on the perturbations; time, dt and the
 *                     conservation sums in FP64.
 *   hyperdiffusion    1: hyper-diffusion and shock viscosity on; 0: ideal fluxes
 *   c2[6]             hyper-diffusion coefficient per conserved variable
 *   c_shk             shock-viscosity coefficient
 *   has_background    1: a static background (bg) is supplied to sac_set_state
 *   device            CUDA device ordinal
 *   stream            cudaStream_t the context enqueues on (NULL = default)
 *   gravity[2]        gravitational acceleration (g_x, g_y) (section 2's rho g
 *                     source).  The background is taken to be in
 *                     magnetohydrostatic balance (its own weight cancels), so the
 *                     perturbation gains rt g in the momentum equation and m.g in
 *                     the energy equation.  Nonzero gravity requires
 *                     has_background = 1 (a zero background array is allowed) and
 *                     is not supported by sac_batch_* or sac_step_noalloc.
 *   hd_single_face    0: the hyper-diffusion ratio takes the maxima of |d3| and
 *                     |d1| over the face and its two neighbours (default);
 *                     1: it uses the face itself (stencil radius 2), the
 *                     minimal form, for comparison.  FP32 supports 1 only
 *                     without background and gravity; not in sac_batch_* or
 *                     sac_step_noalloc.
 */
typedef struct {
    int nx, ny;
    double x0, x1, y0, y1;
    double gamma, courant;
    int bc_x, bc_y;
    int precision;
    int hyperdiffusion;
    double c2[6];
    double c_shk;
    int has_background;
    int device;
    void *stream;
    double gravity[2];
    int hd_single_face;
} sac_params;

/* Fill *p with defaults: 64x64 periodic on [0,1]^2, gamma 5/3, C 0.3, FP64,
 * HD on, c2 = (0.02, 0.1, 0.1, 0.02, 0.02, 0.02), c_shk = 0.5, no background,
 * device 0, default stream, no gravity. */
void sac_default_params(sac_params *p);

/* Validate *p, allocate the device buffers of one run and return a context in
 * *out (NULL on failure).  Errors: SAC_ERR_ARG, SAC_ERR_OOM, SAC_ERR_CUDA. */
int sac_init(const sac_params *p, sac_ctx **out);

/* Release every device and host resource of c (NULL is ignored). */
void sac_free(sac_ctx *c);

/* Text of the last error recorded in c ("" if none); static string for NULL. */
const char *sac_last_error(const sac_ctx *c);

/* Name of a status code. */
const char *sac_status_string(int code);

/*
 * Load the state at time t from HOST FP64 arrays: w [6][ny][nx] (required),
 * bg [4][ny][nx] (required iff has_background, else must be NULL).  Fills the
 * ghost cells (fixed sides are taken from this state and then held), resets
 * the step counter and error status and computes the signal speeds of this
 * state, so sac_dt() is valid.  Synchronous.
 */
int sac_set_state(sac_ctx *c, const double *w, const double *bg, double t);

/* Copy the current state to HOST FP64 w [6][ny][nx] and its time to *t (either
 * may be NULL).  Synchronous; reports a pending device error. */
int sac_get_state(sac_ctx *c, double *w, double *t);

/* As sac_set_state / sac_get_state with DEVICE arrays of the context's
 * precision (double for SAC_FP64, float for SAC_FP32), same packed layout, on
 * the context's device.  ASYNC on the context's stream (sac_get_state_dev
 * returns *t only after synchronising when t != NULL). */
int sac_set_state_dev(sac_ctx *c, const void *w_dev, const void *bg_dev, double t);
int sac_get_state_dev(sac_ctx *c, void *w_dev, double *t);

/*
 * One classical RK4 step (section 2).  dt > 0: take that step; dt <= 0: take
 * the CFL step C min(dx/cmax_x, dy/cmax_y) of the current state.  The signal
 * speeds of the step-start state scale the hyper-diffusion of all four
 * stages.  *dt_taken (may be NULL) receives the step size.  Synchronous.
 */
int sac_step(sac_ctx *c, double dt, double *dt_taken);

/* nsteps CFL steps.  ASYNC: no host synchronisation; errors surface at the
 * next synchronising call.  Steps are replays of a one-step and a 16-step
 * CUDA graph, both captured by the first call (and again after a change of
 * tile configuration or cell size), whatever its step count. */
int sac_steps(sac_ctx *c, long nsteps);

/*
 * Advance with CFL steps until t_end (the last step is clipped so that the
 * time lands exactly on t_end) or until max_steps steps (max_steps < 0: no
 * limit).  *steps_taken (may be NULL) receives the number of steps.  The host
 * polls the device every few steps; steps after t_end are skipped on the device.
 */
int sac_run_to(sac_ctx *c, double t_end, long max_steps, long *steps_taken);

/* Fixed step size for every later CFL step of this context (sac_steps,
 * sac_run_to, sac_step with dt <= 0): dt > 0 replaces the CFL step (the signal
 * speeds still scale the hyper-diffusion); dt <= 0 restores the CFL step.
 * ASYNC; stays in force until changed or until the next set_state. */
int sac_set_fixed_dt(sac_ctx *c, double dt);

/* CFL step the next sac_step(c, 0, ...) would take.  Synchronous. */
int sac_dt(sac_ctx *c, double *dt);

/* Time and steps taken since the last set_state.  Synchronous. */
int sac_time(sac_ctx *c, double *t, long *steps);

/* Maximum signal speeds |v_d| + c_fast of the current state.  Synchronous. */
int sac_cmax(sac_ctx *c, double *cmax_x, double *cmax_y);

/* Conservation sums over the interior of the current state, accumulated in
 * FP64 on the device: sums[f] = sum_ij w[f][j][i] for the six fields.
 * Synchronous. */
int sac_sums(sac_ctx *c, double sums[6]);

/* Discrete divergence of the total magnetic field B = B~ + B_b of the current
 * state (section 2's fourth-order central difference in x and y, the one the
 * flux derivatives use), evaluated in FP64 on the device from the stored
 * values.  A cell counts when its five-point stencil in each direction stays
 * inside the interior or wraps across a periodic side (non-periodic sides
 * drop two cells); a direction of one cell contributes no derivative.
 * max_abs = max |div B|, mean_abs = sum |div B| / ncells (0 when no cell
 * counts), ncells = the number of cells counted; any output may be NULL.
 * A NaN anywhere in the counted stencils makes both max_abs and mean_abs NaN.
 * Deterministic (fixed reduction order).  Synchronous.
 * Errors: SAC_ERR_ARG, SAC_ERR_STATE (no state set), SAC_ERR_CUDA. */
int sac_divb(sac_ctx *c, double *max_abs, double *mean_abs, long long *ncells);

/* Per-kernel timing: nsteps CFL steps launched kernel by kernel (no graph)
 * with CUDA events around every launch on the context's stream.  ms[0] is
 * the mean duration of the step-control kernel, ms[1..4] those of the RK
 * stage 1..4 kernels, in milliseconds.  Advances the state; synchronous. */
int sac_profile_stages(sac_ctx *c, int nsteps, double ms[5]);

/* Wait for the context's stream and report a pending device error. */
int sac_sync(sac_ctx *c);

/* Tile shapes of the FP32 stage kernels (not in the paper, which gives no
 * kernel design): a CTA stages a tile plus its 3-cell halo of the stage input
 * in shared memory (section 2's stencil reaches 3 cells) and updates the tile.
 * SAC_TILE_32x32: 32 x 32 cells, 256 threads, 2 CTAs per SM (the default);
 * SAC_TILE_64x16: 64 x 16 cells, 256 threads, 2 CTAs per SM;
 * SAC_TILE_32x16: 32 x 16 cells, 128 threads, 3 CTAs per SM.
 * SAC_TILE_KERNEL_GHOSTS + shape (3, 4, 5): the same shape, with the ghost
 * frame of every stage output (periodic and outflow copies) written by the
 * stage kernel itself after each tile next to a side, instead of by a separate
 * ghost-frame kernel after each stage (one launch per stage instead of two);
 * runs with a background, gravity or the single-face variant use the separate
 * kernel whatever the setting.
 * Every configuration gives bit-for-bit the same results (each cell's
 * arithmetic does not depend on where the tile boundaries fall, and the ghost
 * cells receive the same copies); they differ in halo overhead per cell, in
 * how evenly the tiles fill the GPU and in launches per step. */
enum { SAC_TILE_32x32 = 0, SAC_TILE_64x16 = 1, SAC_TILE_32x16 = 2, SAC_TILE_KERNEL_GHOSTS = 3 };

/* Use tile configuration `tile` (SAC_TILE_* shape, plus SAC_TILE_KERNEL_GHOSTS
 * for the in-kernel ghost frame) for the later steps of an FP32 context (the
 * gravity and single-face variants always run 32 x 32).  Waits for the
 * context's stream.  Errors: SAC_ERR_ARG (unknown configuration, FP64 context). */
int sac_set_tile(sac_ctx *c, int tile);

/* The context's current tile configuration.  Errors: SAC_ERR_ARG. */
int sac_get_tile(const sac_ctx *c, int *tile);

/* Autotuner of the tile configuration: for every shape, with and without the
 * in-kernel ghost frame (shapes only for runs with a background or the
 * single-face variant), one warm-up CFL step and
 * `trials` timed CFL steps (CUDA events on the context's stream) from the
 * current state, which is restored afterwards together with time, step count
 * and signal speeds; the fastest configuration is kept, reported in *tile (may be
 * NULL) with its mean step time in *ms (may be NULL), and remembered for
 * contexts of the same grid size, hyper-diffusion and background flags that
 * this process creates later (they start with it).  Allocates one state-sized
 * snapshot for the duration of the call.  Synchronous.
 * Errors: SAC_ERR_ARG (FP64 context, trials < 1), SAC_ERR_STATE (no state),
 * SAC_ERR_OOM, SAC_ERR_CUDA, or a device error pending before the call. */
int sac_tune(sac_ctx *c, int trials, int *tile, double *ms);

/* ---------------------------------------------------------------------------
 * Block decomposition (section 3 of the paper: the grid is split into equal
 * sub-domains, and before every RK stage each sub-domain receives from its
 * neighbours the boundary cells its stencil reaches; section 2's maximum wave
 * speed is a maximum over the whole domain).  A sub-domain is an ordinary
 * context of the block's size whose split sides are SAC_BC_FIXED (their ghost
 * cells are left to the caller); the calls below step it stage by stage, move
 * its 3-cell halo strips through caller-owned device buffers, and read or set
 * the running signal-speed maxima so that the caller can reduce them over all
 * sub-domains.  One RK step of a decomposed grid is, on every sub-domain:
 *   for stage 1..4: sac_stage(c, stage), then for each split direction (x
 *   first, then y): sac_halo_pack of the two sides, exchange with the
 *   neighbours, sac_halo_unpack of the two sides;
 *   after stage 4: sac_get_cmax_bits, a maximum over all sub-domains,
 *   sac_set_cmax_bits (also once after sac_set_state, with a halo exchange).
 * The x strips span the ghost-extended height and the y strips the
 * ghost-extended width, so exchanging x before y fills the corner ghosts.
 * These calls only enqueue work on the context's stream (ASYNC).
 * ------------------------------------------------------------------------- */

/* Cell size of the context's later steps (dx, dy > 0; default
 * (x1 - x0) / nx, (y1 - y0) / ny): a block of a decomposed grid takes the
 * grid's cell size bit for bit, which (x1 - x0) / nx of the block's own extent
 * cannot always give in FP64.  Also used by sac_divb.  Waits for the stream.
 * Errors: SAC_ERR_ARG. */
int sac_set_cell_size(sac_ctx *c, double dx, double dy);

/* Enqueue RK stage `stage` (1..4) of one step; stage 1 first starts the step
 * (CFL dt from the current signal-speed maxima, time advance), exactly as
 * sac_step does.  Stages must come in order.  ASYNC.
 * Errors: SAC_ERR_ARG, SAC_ERR_STATE (no state, or out of order), SAC_ERR_CUDA. */
int sac_stage(sac_ctx *c, int stage);

/* Number of elements (of the context's precision) of the packed strip of side
 * `side` (0 left, 1 right, 2 bottom, 3 top): 6 fields x 3 columns x (ny + 6)
 * rows for 0/1, 6 x (nx + 6) columns x 3 rows for 2/3, layout [6][rows][cols].
 * Errors: SAC_ERR_ARG (bad side, fewer than 3 cells across the strip). */
int sac_halo_size(sac_ctx *c, int side, long long *n);

/* Pack the 3 interior cells next to `side` of the latest stage output (the
 * step-start state after sac_set_state or a full step) into the DEVICE buffer
 * strip_dev; unpack a received strip into the 3 ghost cells beyond `side` of
 * that output.  ASYNC.  Errors: SAC_ERR_ARG, SAC_ERR_STATE, SAC_ERR_CUDA. */
int sac_halo_pack(sac_ctx *c, int side, void *strip_dev);
int sac_halo_unpack(sac_ctx *c, int side, const void *strip_dev);

/* Copy the two running signal-speed maxima (x, y) to / from a DEVICE buffer
 * of two 64-bit integers.  The keys are non-negative as signed 64-bit values,
 * order like the speeds, and a NaN speed gives the largest key, so the signed
 * maximum of the keys over sub-domains is the key of the global maximum (and
 * a NaN anywhere stays a NaN).  ASYNC.  Errors: SAC_ERR_ARG, SAC_ERR_STATE. */
int sac_get_cmax_bits(sac_ctx *c, void *bits_dev);
int sac_set_cmax_bits(sac_ctx *c, const void *bits_dev);

/* Test hook of the bounded device waits (FP32 contexts).  Each FP32 stage
 * kernel waits on an mbarrier for its staging copies and gives up after about
 * one second, recording SAC_ERR_TIMEOUT in the run's device status instead of
 * hanging.  With on != 0 the stage kernels issue no copies for their first
 * tile, so that wait runs out: the next step fails with SAC_ERR_TIMEOUT (the
 * remaining stages of that step return at once, and later steps are skipped)
 * until sac_set_state.  Call with on = 0 to clear it.  Nothing faults and no
 * copy is left in flight.  Errors: SAC_ERR_ARG (FP64 context), SAC_ERR_CUDA. */
int sac_debug_drop_copies(sac_ctx *c, int on);

/* ---------------------------------------------------------------------------
 * Batched runs: many independent runs of uneven grid size advanced together.
 * Each RK stage of all runs is ONE kernel launch over a shared queue of
 * tiles (persistent CTAs pulling tiles from an atomic counter, or one CTA per
 * tile; 32x32 tiles unless tuned), each run keeps its own CFL step, time and error status, and
 * each RK step of the whole batch is replayed from a CUDA graph.  Every run
 * must be SAC_FP32, on the same device and stream, with the same
 * hyperdiffusion and has_background flags.  The per-run arithmetic is that of
 * the single-run FP32 path (same tile code), so a batched run reproduces the
 * single-run result.
 * ------------------------------------------------------------------------- */
typedef struct sac_batch sac_batch;

/* Create a batch of 1 <= n <= 65535 runs from runs[0..n-1] (validated as
 * for sac_init).  Errors: SAC_ERR_ARG, SAC_ERR_OOM, SAC_ERR_CUDA. */
int sac_batch_init(const sac_params *runs, int n, sac_batch **out);
void sac_batch_free(sac_batch *b);
const char *sac_batch_last_error(const sac_batch *b);

/* State of run `run` (0-based), host FP64 arrays as sac_set_state /
 * sac_get_state.  Synchronous. */
int sac_batch_set_state(sac_batch *b, int run, const double *w, const double *bg, double t);
int sac_batch_get_state(sac_batch *b, int run, double *w, double *t);

/* nsteps CFL steps of every run (each with its own dt).  ASYNC.  The first
 * call captures the one-step and 16-step graphs it replays. */
int sac_batch_steps(sac_batch *b, long nsteps);

/* Wait for the batch's stream; report the first run in error. */
int sac_batch_sync(sac_batch *b);

/* Time and steps taken of one run.  Synchronous. */
int sac_batch_time(sac_batch *b, int run, double *t, long *steps);

/* Autotuner: times 36 launch configurations, the twelve launch modes (persistent
 * mode 0 = one CTA per tile, 1 = persistent CTAs taking tiles from an atomic
 * queue head, 2 = persistent CTAs walking the queue with a fixed stride;
 * ctas_per_sm 1 = one resident CTA per SM, 2 = as many as the tile shape
 * allows (two, or three for SAC_TILE_32x16); tile order 0 = runs as given,
 * 1 = largest run first, 2 = largest first with tiles interleaved across
 * runs: modes 0 and 2 at ctas_per_sm 2 and mode 1 at 1 and 2, each with all
 * three orders) for each of the three tile shapes (SAC_TILE_*), on `trials`
 * RK steps of the current states, keeps the fastest and restores the states
 * it advanced (every run must have a state).  config[3] (may be NULL)
 * receives (persistent, ctas_per_sm, order); ms (may be NULL) the mean time
 * of one batch RK step with that configuration; sac_batch_get_config also
 * reports the tile shape.  Synchronous. */
int sac_batch_tune(sac_batch *b, int trials, int config[3], double *ms);

/* Set the launch configuration directly (values as sac_batch_tune reports:
 * persistent 0..2, ctas_per_sm 1..2, order 0..2); the tile shape is kept.
 * Every configuration gives bitwise the same results.
 * Errors: SAC_ERR_ARG (out of range). */
int sac_batch_set_config(sac_batch *b, int persistent, int ctas_per_sm, int order);

/* Set the tile shape (SAC_TILE_*) of every run of the batch; the launch mode
 * is kept.  Bitwise the same results.  Errors: SAC_ERR_ARG. */
int sac_batch_set_tile(sac_batch *b, int tile);

/* The current configuration: config[4] = (persistent, ctas_per_sm, order,
 * tile shape).  Errors: SAC_ERR_ARG. */
int sac_batch_get_config(const sac_batch *b, int config[4]);

/* ---------------------------------------------------------------------------
 * Learned coarse-grid correction (not in the paper; a form built on the
 * section 2 method): a 4-layer periodic 3x3 convolutional network
 * f = conv(32->6) . ReLU . conv(32->32) . ReLU . conv(32->32) . ReLU . conv(8->32)
 * on 8 normalised features of the state (the six conserved fields, the kinetic
 * pressure p_k and the current j_z = D_x B_y - D_y B_x with the section 2
 * fourth-order difference, each divided by in_scale[c]).  After a coarse RK4
 * step the state is corrected by u_f <- u_f + out_scale[f] * f_f(features(u)).
 * Forward and backward run on BF16 tensor cores (weights and activations in
 * BF16, FP32 accumulation, FP32 master weights updated with Adam).
 * Parameters are FP32, flat, per layer W[cout][cin][3][3] then b[cout], layers
 * in order (sac_cnn_param_count() of them).  Device arrays are packed FP32
 * [6][ny][nx] conserved states (field order rho, m_x, m_y, e, B_x, B_y) on a
 * periodic nx x ny grid; pred is FP32 [ny*nx][8] (channels 6, 7 unused).
 * ------------------------------------------------------------------------- */
typedef struct sac_cnn sac_cnn;

long sac_cnn_param_count(void);
/* Network workspace for an nx x ny periodic grid (8 <= nx, ny <= 16384) on
 * `device`, enqueuing on `stream`.  Weights start at zero, scales at one. */
int sac_cnn_init(int nx, int ny, int device, void *stream, sac_cnn **out);
void sac_cnn_free(sac_cnn *c);
const char *sac_cnn_last_error(const sac_cnn *c);
/* Tensor-core path of the convolutions: 0 = mma.sync (warp-level BF16 MMA,
 * 8 x 16-pixel tiles); 1 = tcgen05 (5th-generation tensor cores: BF16 operands
 * staged in shared memory by 16-byte asynchronous copies, FP32 accumulators in
 * tensor memory, 4 rows x 128 pixels per tile); 2 = tcgen05 fed by tensor-map
 * copies, pipelined over two halo buffers and two accumulators (2 rows x 128
 * pixels per tile: a tile's MMAs run while the previous tile is written back
 * and the next one's halo is copied).  All accumulate in FP32 over the same tap and channel order
 * and store BF16 activations; on the B300 their outputs are bitwise equal.
 * Waits for the stream.  Errors: SAC_ERR_ARG (path not 0..2); SAC_ERR_CUDA (path 2 when the
 * driver could not encode the activations' tensor maps). */
int sac_cnn_set_tensor_path(sac_cnn *c, int path);
/* Limiter of the correction sac_cnn_apply adds (defaults: off).  clip > 0
 * clamps every network output to [-clip, clip] (a correction of at most clip
 * residual scales per field and step).  keep_positive = 1 drops the correction
 * of a cell whose corrected density or kinetic pressure would fall below half
 * of its value.  The per-field mean of the limited correction is removed, so
 * the correction still conserves every periodic sum.  Errors: SAC_ERR_ARG. */
int sac_cnn_set_limiter(sac_cnn *c, double clip, int keep_positive);
/* Wait for the network's stream and report a tensor-core accumulator wait
 * that gave up (about one second; SAC_ERR_TIMEOUT, flag cleared). */
int sac_cnn_sync(sac_cnn *c);
/* Host FP32 parameters in/out (n must equal sac_cnn_param_count()); setting
 * them also resets the optimiser state.  Synchronous. */
int sac_cnn_set_params(sac_cnn *c, const float *params, long n);
int sac_cnn_get_params(sac_cnn *c, float *params, long n);
/* Host feature scales [8] and output scales [6].  Synchronous. */
int sac_cnn_set_scales(sac_cnn *c, const float in_scale[8], const float out_scale[6]);
/* pred_dev <- f(features(w_dev)).  ASYNC. */
int sac_cnn_forward(sac_cnn *c, const float *w_dev, double gamma, double dx, double dy, float *pred_dev);
/* Training target: next_dev is the state the corrected step should reach (the
 * block-averaged fine run at the same time); the network's target is
 * t = (next - w) / out_scale per field.  Loss 0.5 * mean over 6 channels and all
 * pixels of (f(features(w)) - t)^2 and its gradient with respect to every
 * parameter (host FP32 grads may be NULL; loss may be NULL).  Synchronous when
 * either output is non-NULL. */
int sac_cnn_grads(sac_cnn *c, const float *w_dev, const float *next_dev, double gamma, double dx, double dy,
                  float *grads, double *loss);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) at learning rate lr on that loss.
 * *loss (may be NULL) receives the loss before the update. */
int sac_cnn_train_step(sac_cnn *c, const float *w_dev, const float *next_dev, double gamma, double dx, double dy,
                       double lr, double *loss);
/* Correct the current state of a periodic SAC_FP32 context of the network's
 * size in place: u += out_scale * (f(features(u)) - mean f), the per-field mean
 * taken over the grid so the correction conserves every periodic sum; ghosts
 * and the signal speed of the corrected state are refreshed so the next CFL
 * step uses them.  ASYNC. */
int sac_cnn_apply(sac_ctx *ctx, sac_cnn *c);
/* Training-input augmentation: out = w + amp[f] * xi with xi ~ U[-1, 1) from
 * SplitMix64 counters (seed, element index); w, out device [6][ny][nx] of the
 * network's grid (out may equal w).  Synchronous. */
int sac_cnn_perturb(sac_cnn *c, const float *w_dev, float *out_dev, const float amp[6], unsigned long long seed);
/* r x r block average of a packed FP32 device array [nfields][nyf][nxf] into
 * [nfields][nyf/r][nxf/r] (nxf, nyf multiples of r).  ASYNC on `stream`. */
int sac_block_average(const float *fine_dev, int nfields, int nxf, int nyf, int r, float *coarse_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free step.  The paper has no counterpart: this entry point serves
 * callers that cannot allocate device memory, for example a plug-in whose host
 * application owns all device memory through its own allocator, or a real-time
 * loop in which an allocation (which may synchronise the device and has no
 * latency bound) is not allowed.  It runs one SAC_FP32 RK4 step with the same
 * kernels as sac_step but keeps its working memory (ghost-padded RK registers
 * and step scalars) in a fixed array of 7,244,032 bytes compiled into the
 * library.  Every GPU that loads the library holds that array until the
 * process exits.
 *
 *   p         run parameters; precision must be SAC_FP32 and has_background 0
 *             (device and stream are used as given)
 *   w_in      DEVICE float [6][ny][nx], the state to advance (read only)
 *   w_out     DEVICE float [6][ny][nx], receives the new state (may equal w_in)
 *   dt        > 0: step size; <= 0: the CFL step of w_in
 *   dt_taken  host pointer or NULL.  Non-NULL: the call waits for the stream and
 *             stores the step taken.  NULL: the call only enqueues work.
 * The library cannot check the sizes of w_in and w_out: both must hold
 * 6 * nx * ny floats on p->device.
 * The grid must fit the fixed memory: its padded plane (as sac_init pads it)
 * holds at most 75,456 float2 elements (any grid up to 256 x 256 qualifies);
 * larger grids are rejected with SAC_ERR_TOO_LARGE before any GPU work.
 * Fixed boundaries hold the nearest interior cell of w_in.  The first call on a
 * device does a one-time set-up: it looks up the array's device address
 * (cudaGetSymbolAddress) and sets kernel attributes, under a lock, so first
 * calls from several host threads are safe; make that first call before any
 * stream capture.  No call allocates: no cudaMalloc/cudaFree and no allocating
 * library routine.  All calls share the one array: calls that overlap on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  The state is the only input: the array's previous contents are
 * overwritten (scalars reset) each call.
 * Returns SAC_OK, SAC_ERR_ARG, SAC_ERR_TOO_LARGE, SAC_ERR_CUDA, and, only when
 * dt_taken is non-NULL, SAC_ERR_NONFINITE (non-finite state or step) or
 * SAC_ERR_TIMEOUT (a stage kernel's bounded staging wait gave up).  After any
 * error the contents of w_out are undefined.
 * ------------------------------------------------------------------------- */
#define SAC_ERR_TOO_LARGE (-7)
int sac_step_noalloc(const sac_params *p, const float *w_in, float *w_out, double dt, double *dt_taken);

/* -------------------------------------------------------------------------
 * 3D form (the same method with three-component vectors; section 2 writes the
 * equations for vector fields and the paper runs them in 2D): eight conserved
 * fields rho, m_x, m_y, m_z, e, B_x, B_y, B_z on a periodic box, no background,
 * hyper-diffusion with the maxima over three faces, classical RK4, CFL step
 * dt = C min(min(dx/cmax_x, dy/cmax_y), dz/cmax_z).  FP64 agrees with the FP64
 * 3D oracle to rounding order; FP32 stores and computes in single precision.
 * All calls are synchronous.
 * ------------------------------------------------------------------------- */
typedef struct sac3_ctx sac3_ctx;

/*
 *   nx, ny, nz        interior cells, 1 .. 4096 each; periodic in every direction
 *   x0..z1            box; cell-centred grid
 *   gamma, courant    as in sac_params
 *   precision         SAC_FP64 or SAC_FP32
 *   hyperdiffusion    1: hyper-diffusion and shock viscosity on
 *   c2[8]             hyper-diffusion coefficient per field (rho, m_x, m_y, m_z, e, B_x, B_y, B_z)
 *   c_shk             shock-viscosity coefficient
 *   device, stream    CUDA device and stream (NULL = default)
 */
typedef struct {
    int nx, ny, nz;
    double x0, x1, y0, y1, z0, z1;
    double gamma, courant;
    int precision;
    int hyperdiffusion;
    double c2[8];
    double c_shk;
    int device;
    void *stream;
} sac3_params;

/* Defaults: 32^3 on [0,1]^3, gamma 5/3, C 0.3, FP64, HD on,
 * c2 = (0.02, 0.1, 0.1, 0.1, 0.02, 0.02, 0.02, 0.02), c_shk 0.5, device 0. */
void sac3_default_params(sac3_params *p);
/* Validate *p and allocate one run.  Errors: SAC_ERR_ARG, SAC_ERR_OOM, SAC_ERR_CUDA. */
int sac3_init(const sac3_params *p, sac3_ctx **out);
void sac3_free(sac3_ctx *c);
const char *sac3_last_error(const sac3_ctx *c);
/* State w: host FP64 array [8][nz][ny][nx] (copied; caller keeps ownership). */
int sac3_set_state(sac3_ctx *c, const double *w, double t);
int sac3_get_state(sac3_ctx *c, double *w, double *t);
/* One RK4 step: dt > 0 is used as given, dt <= 0 takes the CFL step;
 * *dt_taken (may be NULL) receives it.  SAC_ERR_NONFINITE if the state's signal
 * speeds or the step are not finite. */
int sac3_step(sac3_ctx *c, double dt, double *dt_taken);
/* n CFL steps. */
int sac3_steps(sac3_ctx *c, long n);
/* CFL steps until t_end (the last step is clipped so that the time lands
 * exactly on t_end) or until max_steps steps (max_steps < 0: no limit);
 * *steps_taken (may be NULL) receives the number of steps.  Errors:
 * SAC_ERR_ARG (t_end not finite), SAC_ERR_STATE, SAC_ERR_NONFINITE,
 * SAC_ERR_TIMEOUT, SAC_ERR_CUDA. */
int sac3_run_to(sac3_ctx *c, double t_end, long max_steps, long *steps_taken);
double sac3_time(const sac3_ctx *c);
/* Conservation sums over the interior of the current state, accumulated in
 * FP64 on the device in a fixed order: sums[f] = sum_ijk w[f][k][j][i] for the
 * eight fields.  Errors: SAC_ERR_ARG, SAC_ERR_STATE (no state), SAC_ERR_CUDA. */
int sac3_sums(sac3_ctx *c, double sums[8]);
/* Discrete divergence of B of the current state: Dx Bx + Dy By + Dz Bz with
 * section 2's fourth-order central difference (neighbours wrapped across the
 * periodic box), in FP64 from the stored values; max_abs = max |div B|,
 * mean_abs = mean |div B| over all cells (either may be NULL); a NaN anywhere
 * makes both NaN.  Deterministic.
 * Errors: SAC_ERR_ARG, SAC_ERR_STATE (no state), SAC_ERR_CUDA. */
int sac3_divb(sac3_ctx *c, double *max_abs, double *mean_abs);
/* Test hook of the bounded copy waits of the FP32 3D stage kernel (as
 * sac_debug_drop_copies): with on != 0 no copy is issued, each stage's wait
 * gives up after about one second and sac3_step returns SAC_ERR_TIMEOUT with
 * the state unchanged; on = 0 clears it.  Errors: SAC_ERR_ARG (FP64). */
int sac3_debug_drop_copies(sac3_ctx *c, int on);

#ifdef __cplusplus
}
#endif
#endif /* SAC_H */
