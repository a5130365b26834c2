/*
 * ac.h -- C ABI of libac.so: one third-order 2N-storage Runge-Kutta substep of
 * compressible non-ideal MHD with sixth-order central differences on a
 * periodic 3-D grid, fused into one CUDA kernel for GB300 (sm_103a).
 *
 * Paper: Pekkila, Vaisala, Kapyla, Rheinhardt, Lappi, "Scalable communication
 * for high-order stencil computations using CUDA-aware MPI" (arXiv:2103.01597).
 *   - problem statement (computational domain N, halo of radius r, grid
 *     M = N + 2r): Sec. 2, Eqs. 2-3;
 *   - stencil point set (axes and face diagonals, radius 3): Sec. 4, Eq. 13;
 *   - equations and fields: Appendix B, Eqs. B.1-B.4, Tables B.1-B.2;
 *   - time integration (Williamson third-order Runge-Kutta): Sec. 4;
 *   - periodic halo map s' = ((s - r) mod n) + r: Sec. 3.3;
 *   - single and double precision: Sec. 3.3.
 *
 * Conventions for every call:
 *   - Return value: AC_OK (0) or a negative AC_ERR_* code; no call throws, and
 *     ac_strerror() names a code.  After AC_ERR_CUDA, ac_last_cuda_error()
 *     gives the CUDA runtime's message.
 *   - Host buffers are owned by the caller and only read or written during the
 *     call.  Device buffers are owned by the library unless the caller binds
 *     its own with ac_bind_buffers(); bound buffers must outlive the handle.
 *   - Work is issued on the handle's CUDA stream (the one given to ac_init,
 *     or the legacy default stream for NULL).  ac_store() and ac_reduce()
 *     synchronise that stream before they return; every other call is
 *     stream-ordered and returns once its work is enqueued.
 *   - A handle is used by one host thread at a time.
 *   - Fields are stored as one array per field (structure of arrays), x
 *     fastest, in the order of Table B.1: ln rho, u_x, u_y, u_z, s, A_x, A_y,
 *     A_z.  Host arrays are always unpadded nx*ny*nz float64.
 */
#ifndef AC_H
#define AC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define AC_OK 0
#define AC_ERR_ARG (-1)       /* invalid argument (NULL, range, size)          */
#define AC_ERR_CUDA (-2)      /* a CUDA runtime call or kernel launch failed    */
#define AC_ERR_OOM (-3)       /* device or host allocation failed               */
#define AC_ERR_NONFINITE (-4) /* a reduction met a NaN or infinity              */
#define AC_ERR_TIMEOUT (-5)   /* a bounded device wait ran out                  */
#define AC_ERR_STATE (-6)     /* call out of order (e.g. substep s skipped)     */

/* ---- fields (Table B.1) ------------------------------------------------- */
#define AC_LNRHO 0
#define AC_UX 1
#define AC_UY 2
#define AC_UZ 3
#define AC_SS 4
#define AC_AX 5
#define AC_AY 6
#define AC_AZ 7
#define AC_NFIELDS 8
#define AC_ALL (-1)

/* ---- precision of device storage and arithmetic (Sec. 3.3 supports both) */
#define AC_FP64 0     /* fields, accumulator and arithmetic in binary64          */
#define AC_FP32 1     /* fields, accumulator and stencil arithmetic in binary32  */
#define AC_FP32_W64 2 /* binary32 fields and arithmetic, binary64 accumulator w */

/* ---- device layout ------------------------------------------------------ */
#define AC_LAYOUT_PERIODIC 0 /* nx*ny*nz per field; the periodic map of Sec. 3.3
                                is applied to every stencil load (no halo)    */
#define AC_LAYOUT_PADDED 1   /* (nx+6)(ny+6)(nz+6) per field with a radius-3
                                halo (grid M of Sec. 2) that ac_periodic_halo()
                                fills                                          */

/* ---- reductions ---------------------------------------------------------- */
#define AC_MAX 0
#define AC_MIN 1
#define AC_SUM 2 /* plain sum over cells (multiply by dx dy dz for integrals) */
#define AC_RMS 3 /* sqrt(sum q^2 / N)                                          */
/* quantities: 0..7 select a field; the rest are derived per cell (mu0 = 1): */
#define AC_Q_UMAG 8  /* |u|                                                    */
#define AC_Q_EKIN 9  /* rho |u|^2 / 2                                          */
#define AC_Q_EMAG 10 /* |B|^2 / 2, B = curl A with the sixth-order first derivative */
#define AC_Q_CFL 11  /* |u| + sqrt(c_s^2 + |B|^2 / rho): fastest signal speed  */

typedef struct {
    int nx, ny, nz;      /* computational domain N (Sec. 2); each >= 1           */
    double lx, ly, lz;   /* box lengths; grid spacing dx = lx / nx etc.          */
    int layout;          /* AC_LAYOUT_PERIODIC or AC_LAYOUT_PADDED               */
} ac_grid;

typedef struct {
    double nu;           /* kinematic viscosity (Eq. B.2)                        */
    double eta;          /* magnetic diffusivity (Eqs. B.3, B.4)                 */
    double cs0;          /* sound speed at s = 0, ln rho = lnrho0                */
    double gamma;        /* adiabatic index (> 1)                                */
    double cp;           /* specific heat at constant pressure (> 0)             */
    double lnrho0;       /* reference log density                                */
    double force_amp;    /* forcing amplitude f0 (0: no forcing)                 */
    unsigned long long seed; /* seed of the per-step forcing draw                */
    int precision;       /* AC_FP64, AC_FP32 or AC_FP32_W64                      */
} ac_params;

typedef struct ac_handle ac_handle; /* opaque; owned by the library */

/*
 * Create a handle for one grid on the current CUDA device.  Validates the
 * grid and parameters (AC_ERR_ARG), allocates small device work areas, and
 * leaves the state buffers unallocated: they are bound with
 * ac_bind_buffers() or allocated by the library on first use.  `stream` is a
 * cudaStream_t (NULL: legacy default stream).  The state starts at substep 0
 * of step 0 with all fields zero once buffers exist.
 */
int ac_init(ac_handle **h, const ac_grid *grid, const ac_params *params, void *stream);

/* Release the handle and every device buffer the library owns.  NULL is a no-op. */
int ac_quit(ac_handle *h);

/* Replace the handle's stream (cudaStream_t; NULL: legacy default stream). */
int ac_set_stream(ac_handle *h, void *stream);

/*
 * Bind caller-owned device memory for the state: dev_ptrs[0..7] and
 * [8..15] are the two state buffers that alternate between input and output
 * of a substep, dev_ptrs[16..23] the Runge-Kutta accumulator w (Williamson
 * 2N storage), one array per field.  Element type: double for AC_FP64, float
 * for AC_FP32 and AC_FP32_W64 (whose w arrays are double).  Each array holds
 * ac_field_elems() elements and must be 16-byte aligned.  Buffers the library
 * owned are freed.  The state is not cleared; dev_ptrs[0..7] become the
 * current state.
 */
int ac_bind_buffers(ac_handle *h, void *const dev_ptrs[24]);

/* Elements per device field array for this handle (padded size for
 * AC_LAYOUT_PADDED). */
int ac_field_elems(const ac_handle *h, size_t *elems);

/*
 * Copy the current state's field `field` (0..7, or AC_ALL for all eight
 * arrays back to back) from unpadded float64 host memory, converting to the
 * device precision (round to nearest).  Page-locked host memory makes the copy
 * asynchronous; pageable memory is copied synchronously.  Resets the substep
 * counter to 0 (a new step begins).
 */
int ac_load(ac_handle *h, int field, const double *host_src);

/* Copy the current state's field (or AC_ALL) to unpadded float64 host memory;
 * synchronises the stream. */
int ac_store(ac_handle *h, int field, double *host_dst);

/* Same as ac_load/ac_store for the accumulator w (checkpoint and resume). */
int ac_load_w(ac_handle *h, int field, const double *host_src);
int ac_store_w(ac_handle *h, int field, double *host_dst);

/* As ac_load / ac_store with float32 host memory (unpadded, x fastest, field
 * 0..7 or AC_ALL back to back).  For an AC_FP32 or AC_FP32_W64 state in the
 * periodic layout the copy moves the state's own bytes, half those of the
 * float64 format; otherwise the values pass through the staging buffer: a
 * float64 state takes the float32 values exactly on load and is rounded to
 * nearest on store.  ac_load_f32 resets the substep counter to 0; ac_store_f32
 * synchronises the stream. */
int ac_load_f32(ac_handle *h, int field, const float *host_src);
int ac_store_f32(ac_handle *h, int field, float *host_dst);

/*
 * One Runge-Kutta substep s of the step in progress (Sec. 4; Williamson's
 * third-order 2N-storage scheme):  w <- alpha_s w + dt RHS(f);  f <- f + beta_s w,
 * alpha = (0, -5/9, -153/128), beta = (1/3, 15/16, 8/15), with RHS the right-hand
 * side of Eqs. B.1-B.4 evaluated with sixth-order central differences on the
 * points of Eq. 13, the periodic map of Sec. 3.3 at the domain boundary, and the
 * step's forcing term added to du/dt when force_amp != 0.  One fused kernel
 * reads f and w and writes the new f (into the other state buffer, which then
 * becomes current) and w.  At s = 0, w is not read.  s must follow the previous
 * substep ((previous + 1) mod 3, starting at 0): otherwise AC_ERR_STATE.
 * dt must be finite.  With AC_LAYOUT_PADDED the halo is refreshed first.
 * At s = 0 with forcing on, the step's forcing is drawn (ac_forcing_draw with
 * the handle's seed and step counter) unless ac_set_forcing() fixed it.  After
 * s = 2 the step counter advances.
 */
int ac_integrate_substep(ac_handle *h, double dt, int s);

/*
 * The terms of Eqs. B.2-B.3 that the base configuration sets to zero: thermal
 * conductivity K (constant), bulk viscosity zeta (kinematic, as written in
 * Eq. B.2: du/dt gains zeta grad(div u), rho T ds/dt gains zeta rho (div u)^2),
 * and explicit heating H and cooling C (uniform rates: rho T ds/dt gains
 * H - C).  Conduction: div(K grad T) = K T (lap xi + |grad xi|^2) with
 * xi = gamma s / c_p + (gamma - 1)(ln rho - ln rho0) (grad T = T grad xi), the
 * gradient and Laplacian of xi taken with the stencils of s and ln rho.
 * All four must be finite and >= 0 (AC_ERR_ARG otherwise); default 0.  Any
 * non-zero term selects kernels that evaluate them (binary64, binary32 and
 * the integer-sum path alike); the batched ensemble keeps the base terms.
 */
int ac_set_entropy_terms(ac_handle *h, double K, double zeta, double heat, double cool);

/*
 * Stencil order (Sec. 4 uses sixth order, radius 3, on the points of Eq. 13;
 * orders 2, 4 and 8 use the same kind of point set out to radius 1, 2, 4:
 * the axes and the face diagonals).  Central weights of order 2r: first
 * derivative sum_m w_m (f_m - f_-m) / dx, second derivative
 * [a_0 f_0 + sum_m a_m (f_m + f_-m)] / dx^2, mixed derivative
 * sum_m a_m S_m / (4 dx_a dx_b) on the diagonal sums S_m.  Default 6.  Order 8
 * needs the periodic layout (the padded layout's halo is 3 cells).  Only at a
 * step boundary (AC_ERR_STATE otherwise); AC_ERR_ARG for other orders, or for
 * an order other than 6 while AC_STENCIL_FIXED is set.  Binary32 handles use
 * the shared-memory tiled kernel at order 6 and the direct-load kernel
 * otherwise; reductions (E_M's curl) use the same order.
 */
int ac_set_stencil_order(ac_handle *h, int order);
int ac_get_stencil_order(const ac_handle *h, int *order);

/*
 * Arithmetic of the stencil sums for AC_FP64.  AC_STENCIL_AUTO (default): exact
 * integer sums whenever they apply (binary64 fields, periodic layout, equal
 * spacing dx = dy = dz, stencil order 6, a step dt with |dt| in [1e-100, 1e100]:
 * those kernels fold dt into their coefficients), plain binary64 sums
 * otherwise.  With
 * integer sums every field is first written, on the device before each
 * substep, as int64 fixed point about its own offset: F = round((f - c)
 * 2^(50 - E)), c the midpoint of the field's range and 2^E above its
 * half-range, so |F| <= 2^50 + 2 and each input is resolved to 2^-51 of the
 * field's own range (the weights of every Eq. 13 stencil sum to zero, so the
 * offset changes no derivative).  Every stencil numerator and every sum of
 * numerators with a common coefficient is then exact and only one int64 ->
 * binary64 conversion and one multiplication per derivative term run on the
 * FP64 pipe.  The device picks, per substep, one of three modes (counted by
 * ac_get_stencil_modes): AC_STENCIL_MODE_GROUP when the exponents E of the
 * components of u (and of A) lie within one binade of each other (they share
 * the largest, so a component keeps at least 49 bits of its own range, and the
 * cross-component sums stay single integers); AC_STENCIL_MODE_FIELD otherwise
 * (each field keeps its own scale; the sums across components are added in
 * binary64); AC_STENCIL_MODE_PLAIN when the
 * state holds a NaN or an infinity or a range outside [2^-960, 2^960) (plain
 * binary64 stencils, the AC_STENCIL_FP64 arithmetic, so non-finite values
 * propagate as the definition does and show in ac_last_cfl).  The result stays
 * within the 1e-12 relative bound of the exact-rounding definition.
 * AC_STENCIL_FP64: binary64 arithmetic throughout.  AC_STENCIL_FIXED: integer
 * sums, AC_ERR_ARG where they do not apply.  Extra device memory for integer
 * sums: one int64 copy of the eight fields, allocated on first use.
 */
#define AC_STENCIL_AUTO 0
#define AC_STENCIL_FP64 1
#define AC_STENCIL_FIXED 2
int ac_set_stencil_mode(ac_handle *h, int mode);
/* *fixed = 1 if the next substeps use integer stencil sums. */
int ac_get_stencil_path(const ac_handle *h, int *fixed);
/*
 * counts[m] = substeps the integer-sum path has run in mode m since the
 * handle's first integer-sum substep (all 0 before it).  Synchronises the
 * handle's stream.
 */
#define AC_STENCIL_MODE_GROUP 0
#define AC_STENCIL_MODE_FIELD 1
#define AC_STENCIL_MODE_PLAIN 2
int ac_get_stencil_modes(ac_handle *h, unsigned long long counts[3]);

/* Substeps 0, 1, 2 with the same dt (one full Runge-Kutta step). */
int ac_integrate_step(ac_handle *h, double dt);

/*
 * Kernel timing (no counterpart in the paper; for the roofline of the substep
 * kernel).  While on, every ac_integrate_substep records CUDA events on the
 * handle's stream around its preparation kernels (on the integer-sum path: the
 * field extremes, the plan and the quantisation) and around the substep kernel
 * itself, for up to AC_TIMING_MAX substeps after the call that switched it on.
 * ac_kernel_timings waits for the last recorded substep and returns, per
 * substep index s, the average preparation and kernel times in milliseconds and
 * how many substeps were recorded; it then clears the records.  Turning timing
 * on creates 3 * AC_TIMING_MAX events (freed by ac_quit).
 */
#define AC_TIMING_MAX 1024
int ac_set_kernel_timing(ac_handle *h, int on);
int ac_kernel_timings(ac_handle *h, double prep_ms[3], double kernel_ms[3], int count[3]);

/*
 * Largest CFL speed |u| + sqrt(c_s^2 + |B|^2 / rho) over the cells of the state
 * that the last substep 0 read (the state at the start of the step), computed
 * by the substep kernel itself in the field precision (quantity AC_Q_CFL of
 * ac_reduce, without a separate pass).  Synchronises the stream;
 * AC_ERR_NONFINITE if a cell gave NaN or infinity.  0 before any substep 0.
 * Not in the paper (constant dt, Sec. 5): for a CFL check of dt.
 */
int ac_last_cfl(ac_handle *h, double *out);

/*
 * Fill the radius-3 halo of the current state (AC_LAYOUT_PADDED) with the
 * periodic map of Sec. 3.3, s' = ((s - r) mod n) + r per axis: the six sides,
 * twelve edges and eight corners.  A no-op for AC_LAYOUT_PERIODIC.
 */
int ac_periodic_halo(ac_handle *h);

/*
 * Reduce a quantity of the current state over all cells in binary64
 * (AC_MAX, AC_MIN, AC_SUM, AC_RMS; quantity 0..7 or AC_Q_*), write the result
 * to *out (host memory) and synchronise.  AC_ERR_NONFINITE if any per-cell
 * value met is NaN or infinite (*out is still written).  Not in the paper (its
 * timestep is constant, Sec. 5): energies and the CFL speed for monitoring.
 */
int ac_reduce(ac_handle *h, int op, int quantity, double *out);

/*
 * The forcing of step `step` for seed `seed` (not in the paper): wave vector
 * k with 2 <= |k| <= 3, unit polarisation e perpendicular to k, phase phi in
 * [0, 2 pi), drawn with the SplitMix64 counter generator.  The forcing adds
 * force_amp * e * cos(2 pi sum_a k_a i_a / n_a + phi) to du/dt at cell i.
 */
int ac_forcing_draw(unsigned long long seed, unsigned long long step, int k[3], double e[3],
                    double *phi);

/* Fix the forcing for the following substeps (instead of the per-step draw);
 * k == NULL returns to the per-step draw. */
int ac_set_forcing(ac_handle *h, const int k[3], const double e[3], double phi);

/* Step counter (completed full steps) and the next expected substep. */
int ac_get_step(const ac_handle *h, unsigned long long *step, int *next_substep);

/* Position the handle at substep `next_substep` (0..2) of step `step`, e.g. to
 * resume from a checkpoint: load f with ac_load and w with ac_load_w first
 * (ac_load resets the substep to 0).  The step's forcing is drawn again for
 * `step` at the next substep. */
int ac_set_step(ac_handle *h, unsigned long long step, int next_substep);

/* Number of kernels the handle has launched so far. */
int ac_launch_count(const ac_handle *h, unsigned long long *count);

/* ---- batched ensemble ------------------------------------------------------
 * Independent periodic boxes of uneven size integrated together (the paper
 * notes that parameter scans inflate problem sizes, Sec. 4).  Each box carries
 * its own grid and nu, eta; the other constants come from `common`.  One
 * persistent kernel launch per substep covers every box: work items are
 * (box, column tile, z range), taken largest first from a device
 * counter; each item computes exactly what the single-box binary32 kernel
 * computes for those cells (same substep as ac_integrate_substep, no forcing),
 * whatever its tile shape: 32 x 8 or 16 x 16 cells per tile, chosen per box.
 * State: binary32 fields (AC_FP32, or AC_FP32_W64 with a binary64 accumulator);
 * device memory is owned by the batch.  Limits: 1..AC_BATCH_MAX_BOXES boxes,
 * 1..4096 cells per axis, nx a multiple of 4; force_amp must be 0.
 */
#define AC_BATCH_MAX_BOXES 128

typedef struct {
    int nx, ny, nz;      /* cells per axis                                       */
    double lx, ly, lz;   /* box lengths                                          */
    double nu, eta;      /* this box's viscosity and magnetic diffusivity        */
} ac_box;

typedef struct ac_batch ac_batch; /* opaque; owned by the library */

/* Create a batch of `nbox` boxes (`boxes`: host array, copied) sharing the
 * constants and precision of `common` (its force_amp must be 0); *b receives
 * the handle, freed by ac_batch_quit (NULL is accepted there).  `stream`
 * (cudaStream_t, may be NULL) orders every later call of the batch.
 * AC_ERR_ARG outside the limits above, AC_ERR_OOM if device memory runs out. */
int ac_batch_init(ac_batch **b, int nbox, const ac_box *boxes, const ac_params *common,
                  void *stream);
int ac_batch_quit(ac_batch *b);
/* Host float64 <-> one box's current state (field 0..7 or AC_ALL, unpadded,
 * x fastest) or accumulator; store synchronises the stream, load resets the
 * substep counter to 0. */
int ac_batch_load(ac_batch *b, int box, int field, const double *host_src);
int ac_batch_store(ac_batch *b, int box, int field, double *host_dst);
int ac_batch_load_w(ac_batch *b, int box, int field, const double *host_src);
int ac_batch_store_w(ac_batch *b, int box, int field, double *host_dst);
/* The same state copies with float32 host memory: the batch's state is binary32,
 * so each call is one copy of the box's own bytes (load resets the substep
 * counter, store synchronises the stream). */
int ac_batch_load_f32(ac_batch *b, int box, int field, const float *host_src);
int ac_batch_store_f32(ac_batch *b, int box, int field, float *host_dst);
/* Substep s of every box (order rules of ac_integrate_substep). */
int ac_batch_integrate_substep(ac_batch *b, double dt, int s);
/* Substeps 0, 1, 2 of every box; with the graph enabled, the three launches
 * (and the counter resets) are captured once per (dt, state buffer) into a
 * CUDA graph and replayed. */
int ac_batch_integrate_step(ac_batch *b, double dt);
/* Enable (non-zero) or disable (0, the default) the graph of ac_batch_integrate_step. */
int ac_batch_set_graph(ac_batch *b, int enable);
/* Tile shapes of the work items (one per box). */
#define AC_TILE_32X8 0
#define AC_TILE_16X16 1

/* Autotuner of the work split: times whole steps (substeps 0, 1, 2, each
 * candidate from the same state: the state is saved on the device first and
 * restored afterwards, so the call leaves it unchanged and w is rewritten by
 * the next substep 0) for work items of z extent 8, 16, 32, 64 and 128 with
 * every box on one tile shape, for both shapes; then, for each class of boxes
 * of equal nx and ny (largest total cells first), tries the other shape and
 * keeps it if the step gets faster by more than 0.3%.  *zc_out receives the
 * chosen z extent (ac_batch_get_tiling gives the shapes and the step times).
 * With a cache path, the choice for this device, precision and set of box
 * sizes is read from, or added to, a JSON object file written by this call:
 * one line per entry, "<signature>": {"zc": Z, "tiles": "<one digit per box>",
 * "ms_default": T0, "ms_tuned": T1}; a file holding anything else is read but
 * never rewritten.  Temporarily allocates one state pool.  Must be called at a
 * step boundary (AC_ERR_STATE otherwise). */
int ac_batch_tune(ac_batch *b, double dt, const char *cache_path, int *zc_out);
/* Set the work split by hand: z extent 1..4096 and `shapes` (nbox entries of
 * AC_TILE_*, or NULL for all AC_TILE_32X8).  Results do not depend on it. */
int ac_batch_set_tiling(ac_batch *b, int zc, const int *shapes);
/* The current split (z extent, nbox shapes) and, after a tuning, the step time
 * (ms) of the default split (z extent 64, all 32 x 8) and of the tuned one
 * (0 where unknown).  Any output may be NULL. */
int ac_batch_get_tiling(const ac_batch *b, int *zc, int *shapes, float tune_ms[2]);
/* Reduction of one box's state, as ac_reduce. */
int ac_batch_reduce(ac_batch *b, int box, int op, int quantity, double *out);
/* Total cells, work items, z extent of an item, persistent CTAs, launches so far. */
int ac_batch_info(const ac_batch *b, long long *cells, int *items, int *zc, int *ctas,
                  unsigned long long *launches);

/* Device pointers of the current state's eight field arrays, with the
 * handle's precision, layout and grid size (any of the outputs may be NULL). */
int ac_get_state(const ac_handle *h, void *dev_ptrs[8], int *precision, int *layout, int n[3]);

/* ---- learned closure for a 2x-coarser grid ---------------------------------
 * The paper only mentions machine-learned reconstruction of turbulent flows
 * from low-resolution data (Sec. 6); this closure is a reading of that remark:
 * a three-layer 3-D conv net (8 -> 32 -> 32 -> 8 channels, 3x3x3 kernels,
 * circular padding, ReLU after layers 1 and 2) maps a coarse state f (binary32,
 * periodic layout, eight device arrays) to a correction
 *     delta[c] = out_scale[c] * net(f / in_scale)[c].
 * Convolutions run on the tensor cores with bfloat16 weights and activations
 * and binary32 accumulation; master weights, gradients and Adam moments are
 * binary32.  Parameters are one binary32 array of AC_CLOSURE_NPARAMS values:
 * W1[32][8][3][3][3], b1[32], W2[32][32][3][3][3], b2[32], W3[8][32][3][3][3],
 * b3[8]; a weight W[co][ci][kz][ky][kx] multiplies input channel ci at
 * (z + kz - 1, y + ky - 1, x + kx - 1) (periodic).  Loss: mean squared error of
 * the scaled output against target / out_scale over all cells and channels.
 */
#define AC_CLOSURE_NPARAMS 41544
typedef struct ac_closure ac_closure; /* opaque; owned by the library */

/* Create a closure for a coarse periodic grid of nx x ny x nz cells with zero
 * parameters and unit scales; *c receives the handle, freed by ac_closure_quit
 * (NULL is accepted there).  `stream` (cudaStream_t, may be NULL) orders every
 * later call.  AC_ERR_ARG for sizes outside 1..2^20, AC_ERR_OOM if device
 * memory runs out. */
int ac_closure_init(ac_closure **c, int nx, int ny, int nz, void *stream);
int ac_closure_quit(ac_closure *c);
/* Host binary32 parameters in/out (set also clears the Adam moments). */
int ac_closure_set_params(ac_closure *c, const float *host_params);
int ac_closure_get_params(ac_closure *c, float *host_params);
/* Gradients of the last ac_closure_backward, same layout as the parameters. */
int ac_closure_get_grads(ac_closure *c, float *host_grads);
/* Per-channel input and output scales (positive, finite). */
int ac_closure_set_scales(ac_closure *c, const float in_scale[8], const float out_scale[8]);
/* Correction of the coarse state `in` into `out` (device arrays, may not alias;
 * out == NULL keeps the result inside the closure). */
int ac_closure_forward(ac_closure *c, const float *const in[8], float *const out[8]);
/* As ac_closure_forward (out required), and ms[0..4] receives the device time
 * of each of its launches (input pack, convolution layers 1, 2, 3, output
 * scaling) from CUDA events on the closure's stream; synchronises.  On the
 * tcgen05 path layer 3 scales in its epilogue and ms[4] is the empty interval. */
int ac_closure_forward_timings(ac_closure *c, const float *const in[8], float *const out[8],
                               float ms[5]);
/* Forward, loss against `target` (physical units, device arrays) and
 * gradients of every parameter; *loss (if non-NULL) synchronises. */
int ac_closure_backward(ac_closure *c, const float *const in[8], const float *const target[8],
                        double *loss);
/* One Adam step (Kingma and Ba, bias-corrected) with the last gradients. */
int ac_closure_adam_step(ac_closure *c, float lr, float beta1, float beta2, float eps);
/* Add the correction of a binary32 periodic handle's current state to it, but
 * only if every correction value is finite and at most `limit` in magnitude
 * (the guard runs on the device; *applied, if non-NULL, synchronises). */
int ac_closure_apply(ac_closure *c, ac_handle *h, double limit, int *applied);
/* Number of kernels the closure has launched so far. */
int ac_closure_launch_count(const ac_closure *c, unsigned long long *count);
/* Convolution kernels of the forward pass run by ac_closure_forward and
 * ac_closure_apply.  AC_CONV_TCGEN05 (the default): tcgen05.mma with the
 * accumulator in tensor memory, on channels-last activations, persistent CTAs
 * holding one layer's weights in shared memory.  AC_CONV_MMA_SYNC: the
 * warp-level mma.sync kernels on channel-major activations that
 * ac_closure_backward always uses.  AC_CONV_TCGEN05_PAIR: the tcgen05 kernel
 * on clusters of two CTAs (cta_group::2, M = 256), each CTA holding half of a
 * layer's weights.  All take the same bfloat16 operands and accumulate in
 * binary32, in different orders.  Any other value: AC_ERR_ARG. */
#define AC_CONV_TCGEN05 0
#define AC_CONV_MMA_SYNC 1
#define AC_CONV_TCGEN05_PAIR 2
int ac_closure_set_conv_path(ac_closure *c, int path);
int ac_closure_get_conv_path(const ac_closure *c, int *path);
/* Reads and clears the device error word of the tcgen05 kernels
 * (synchronises the closure's stream): AC_ERR_TIMEOUT if one of their bounded
 * mbarrier waits ran out since the last call (the outputs of that call are
 * then undefined), else AC_OK. */
int ac_closure_status(ac_closure *c);
/* Diagnostic of the bounded device waits that the tcgen05 kernels use: one CTA
 * waits, through the same bounded mbarrier wait, on a phase that nothing
 * completes, gives up after `polls` polls (1 <= polls <= 2^18, the kernels'
 * own bound, about one second; else AC_ERR_ARG), records that in a device word
 * and returns.  The expected result is AC_ERR_TIMEOUT, with the context still
 * usable; AC_OK would mean the wait completed.  `stream` may be NULL;
 * synchronises it. */
int ac_diag_wait_timeout(unsigned polls, void *stream);
/* Diagnostic of the table-driven binary64 exp that the binary64 substep
 * kernels use for exp(-ln rho), exp(xi) and exp(-xi) (Tang's method with a
 * 256-entry table; the library exp where |x| >= 700 or x is not finite).
 * `x`: n device binary64 values; `y`: 4n device binary64 values, written as
 * y[i] = the table exp of x[i], y[n + i] = CUDA's exp(x[i]), y[2n + i] and
 * y[3n + i] = exp(x[i]) and exp(-x[i]) from the paired evaluation.  Both
 * buffers belong to the caller.  n < 0, or a NULL pointer with n > 0, is
 * AC_ERR_ARG; n == 0 does nothing.  `stream` may be NULL; synchronises it. */
int ac_diag_exp_table(const double *x, long long n, double *y, void *stream);

/* Global-index checks of a library built with AC_BOUNDS_CHECK (a separate,
 * slower build for tests): every index the stencil, substep and convolution
 * kernels form is compared with its array's extent, and an index outside it is
 * recorded (bit 63 set, a kind tag in bits 48-62, the index's low 48 bits) and
 * redirected or skipped instead of performed.  Writes the first recorded word
 * since the last call to *first (0: none) and clears them all; AC_OK.  In the
 * normal build *first = 0 and the result is AC_ERR_STATE (nothing is checked).
 * Synchronises the device. */
int ac_bounds_check_take(unsigned long long *first);
/* Self-test of those checks (checked build): one kernel computes two checked
 * indices without using them, -5 and 3 against an extent of 10, and writes
 * them to out: expected 0 (redirected, and recorded with tag 7 for the next
 * ac_bounds_check_take) and 3.  AC_ERR_STATE in the normal build. */
int ac_bounds_check_selftest(long long out[2]);

/*
 * Domain decomposition with halo exchange (Sec. 3.2-3.3, Fig. "concurrency"):
 * the periodic grid (AC_LAYOUT_PERIODIC; n_a divisible by p_a, n_a / p_a >= 6)
 * is split into p[0] x p[1] x p[2] subdomains of n' = n / p cells, each held
 * with a radius-3 halo.  Subdomains are ordered in Z-order (their coordinates
 * sorted by Morton code, bits of x, y, z interleaved with x lowest:
 * ac_decomp_coord), the order in which they would be assigned to devices.
 * Every substep (ac_decomp_integrate_substep) runs the iteration of Sec. 3.3:
 * pack the outbound halo segments (6 sides and 12 edges per subdomain; the 8
 * corners are never read by the Eq. 13 stencil and are not sent) into
 * contiguous message buffers, deliver the messages, unpack them into the
 * receivers' halos, and update the outer segments; the inner segment
 * (interior cells at least 3 from the subdomain's faces, whose stencils read
 * no halo cell) is updated on the caller's `stream` while the exchange runs on
 * a second, higher-priority stream.  ac_decomp_set_overlap(d, 0) runs pack,
 * exchange, unpack and one whole-subdomain update in sequence instead.  All
 * subdomains live on the current device, so a message is a device-local copy.
 * Arithmetic: plain binary64 (AC_FP64) or binary32 stencils of order 6, the
 * same per-cell code as the undecomposed padded-layout substep, so the result
 * equals ac_integrate_substep on an AC_LAYOUT_PADDED handle (or, in binary64,
 * an AC_STENCIL_FP64 periodic one) bitwise.  Forcing is drawn per step from
 * (seed, step) as ac_integrate_substep draws it.  ac_decomp_load/_store take
 * the whole unpadded host array (x fastest) and are synchronous; substeps are
 * stream-ordered and checked in order (AC_ERR_STATE).
 */
typedef struct ac_decomp ac_decomp;
int ac_decomp_init(ac_decomp **d, const ac_grid *grid, const ac_params *params, const int p[3],
                   void *stream);
int ac_decomp_quit(ac_decomp *d);
int ac_decomp_load(ac_decomp *d, int field, const double *host_src);
int ac_decomp_store(ac_decomp *d, int field, double *host_dst);
int ac_decomp_load_w(ac_decomp *d, int field, const double *host_src);
int ac_decomp_store_w(ac_decomp *d, int field, double *host_dst);
int ac_decomp_integrate_substep(ac_decomp *d, double dt, int s);
int ac_decomp_integrate_step(ac_decomp *d, double dt);
int ac_decomp_set_overlap(ac_decomp *d, int on);
/* Partition, local size, message count (18 per subdomain) and kernel launches. */
int ac_decomp_info(const ac_decomp *d, int p[3], int nloc[3], int *messages,
                   unsigned long long *launches);
/* Host-only schedule (no device call).  ac_decomp_partition: the paper's
 * partition of a power-of-two device count, P = morton^-1(count - 1) +
 * (1, 1, 1).  ac_decomp_coord: coordinates of the subdomain with Z-order
 * position `rank` in a p grid.  ac_decomp_segment: halo segment `seg` (0..17:
 * sides x-, x+, y-, y+, z-, z+, then the edges in lexicographic order of the
 * direction) of a subdomain of nloc cells: its direction d, the origin of the
 * receiver's halo box (dst_b0) and of the cells of the neighbour at +d that
 * fill it (src_b0), both in padded coordinates (interior from 3 to 3 + n' - 1),
 * and the box's extent; src = ((dst - 3) mod n') + 3 per axis (Sec. 3.3). */
int ac_decomp_partition(int count, int p[3]);
int ac_decomp_coord(const int p[3], int rank, int coord[3]);
int ac_decomp_segment(const int nloc[3], int seg, int dir[3], int src_b0[3], int dst_b0[3],
                      int ext[3]);

/* Arithmetic-rate probe (no counterpart in the paper; the denominator of the
 * binary64 substep's roofline): *fma_per_s = thread-level fused multiply-adds
 * per second of the library's own FMA-chain kernel (8 independent chains per
 * thread, 8 CTAs of 256 threads per SM, each timed launch about 50 ms, best of
 * several) in binary64 (AC_FP64: the FP64 pipe) or binary32 (AC_FP32: the
 * FP32 pipes) on the current device.  Synchronises `stream`.  AC_ERR_ARG for
 * another precision. */
int ac_diag_fma_rate(int precision, double *fma_per_s, void *stream);

/* Full-weighting restriction of eight fine fields (nx, ny, nz even; binary64
 * for AC_FP64, binary32 otherwise; periodic layout) to eight binary32 coarse
 * arrays: coarse(I) = sum over d in {-1,0,1}^3 of prod_a w(d_a) fine(2I + d),
 * w = (1/4, 1/2, 1/4).  Asynchronous on `stream`. */
int ac_restrict(const void *const fine[8], int fine_precision, int nx, int ny, int nz,
                float *const coarse[8], void *stream);

/*
 * Allocation-free reduction (the paper has no counterpart; it exists for
 * callers that cannot allocate device memory -- for example an application
 * that owns all device memory through its own pool and only lends the library
 * its field arrays, and so cannot create an ac_handle, whose work areas are
 * allocated with cudaMalloc).
 *
 * Same result as ac_reduce (op, quantity, binary64 accumulation, per-cell
 * quantities evaluated the same way at stencil order 6) for the state held in
 * `fields`: eight device arrays in the field order of the AC_LNRHO..AC_AZ
 * constants above, each laid out for `grid` (padded layout: the halo must
 * already hold the periodic images) with elements of `params->precision`
 * (double for AC_FP64, float otherwise).  The curl of A in AC_Q_EMAG and
 * AC_Q_CFL always uses the sixth-order first derivative, so those two match
 * ac_reduce only on handles at stencil order 6.  `grid` and `params` are
 * checked as ac_init checks them.  The partial sums go to a fixed device array
 * inside the library (one slot per z-plane, at most AC_NOALLOC_MAX_NZ planes:
 * larger nz is rejected with AC_ERR_ARG); nothing is allocated.  The result is
 * written to host memory *out and `stream` (cudaStream_t, NULL: legacy default
 * stream) is synchronised; AC_ERR_NONFINITE if a NaN or infinity was met.
 * Only the summation order differs from ac_reduce, so sums and rms agree to
 * rounding and max/min exactly.
 *
 * The fixed array has one copy per device; each call uses the copy of the
 * device current on the calling thread (looked up on every call), so `stream`
 * and the field arrays must belong to that device.  Every call shares the
 * array: calls whose work overlaps on the GPU (other streams or host threads)
 * race on it and must be serialised by the caller.
 */
#define AC_NOALLOC_MAX_NZ 8192
int ac_reduce_noalloc(const void *const fields[8], const ac_grid *grid, const ac_params *params,
                      int op, int quantity, double *out, void *stream);

/* Text of an AC_* code; message of the last CUDA error seen by this thread. */
const char *ac_strerror(int code);
const char *ac_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AC_H */
