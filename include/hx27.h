/*
 * hx27 -- wavelength-adaptive 27-point Helmholtz operator and solver (C ABI).
 *
 * Method: Aghamiry, Gholami, Combe & Operto, "Accurate 3D frequency-domain
 * seismic wave modeling with the wavelength-adaptive 27-point finite-difference
 * stencil" (arXiv 2108.08730).  The discrete problem is [M + S] p = s (Eq. 3)
 * on a regular grid with PML (Eqs. 1.1-1.4), constant density (Section 3.1),
 * stiffness weights (ws1, ws2, ws3) and consistent-mass weights (wm1..wm4)
 * picked per row from a Tikhonov-smoothed table by the row's own
 * G = v / (f h) (Section 2.2; the GA stencil of Section 3.1).
 *
 * Conventions shared by every entry point:
 *  - Grids are row-major with x fastest: index = ix + nx*(iy + ny*iz).
 *    Velocity is float32 v[nz][ny][nx] in m/s.  Wavefields are interleaved
 *    complex (re, im): complex64 = 2 x float32, complex128 = 2 x float64,
 *    laid out [nrhs][nz][ny][nx].
 *  - Pointers named *_dev are device pointers on the context's device,
 *    *_host are host pointers.  All buffers passed in are owned by the
 *    caller; the library never frees or retains them past the call (device
 *    work is enqueued on `stream` and may still be running when the call
 *    returns, like any CUDA launch).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - The context owns its caches (weight table on the device, PML
 *    coefficient arrays, multigrid hierarchies, Krylov workspaces) and frees
 *    them in hx_ctx_destroy.  A context is not thread-safe; use one per host
 *    thread.
 *  - Every call returns an hx_status; on failure it also records a message
 *    retrievable with hx_last_error.  Nothing throws across the ABI.
 *  - Kernels are launched with programmatic dependent launch: a kernel's
 *    CTAs may become resident while its predecessor on the same stream
 *    drains, and wait for it in hardware before touching memory.  Setting
 *    the environment variable HX_PDL=0 before the first launch turns this
 *    off (results are bit-identical either way).
 */
#ifndef HX27_H
#define HX27_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HX_OK = 0,
  HX_ERR_ARG = -1,            /* invalid argument (message says which)          */
  HX_ERR_OOM = -2,            /* device or host allocation failed               */
  HX_ERR_NOT_CONVERGED = -3,  /* solve stopped at its iteration cap; the best
                                 iterate is in the output and the report filled */
  HX_ERR_NUMERIC = -4,        /* NaN/Inf or breakdown detected                  */
  HX_ERR_TIMEOUT = -5,        /* a bounded device wait ran out                  */
  HX_ERR_CUDA = -6,           /* a CUDA runtime call failed                     */
  HX_ERR_STATE = -7,          /* call order (e.g. no weight table set yet)      */
  HX_ERR_CANCELLED = -8       /* stopped by its cancel flag (hx_solve_opts.cancel,
                                 hx_server_cancel); the best iterate so far is in
                                 the output when the solve had started           */
} hx_status;

typedef struct hx_ctx hx_ctx;

/* Grid, frequency and PML of one problem.  PML nodes are part of the grid
 * (npml nodes at each face).  The damping follows the reading
 * gamma(d) = gamma0 (d/L)^2, gamma0 = 3 v_ref / (2 L) ln(1/r_coef), with d the
 * distance from the inner PML face and L = npml h; xi = 1 + i gamma/omega
 * (Eqs. 1.1-1.4, exp(-i omega t)).  Outside the grid the field is zero. */
typedef struct {
  int nx, ny, nz;      /* nodes per axis incl. PML, each >= 3              */
  double h;            /* grid interval (m), > 0                            */
  double f;            /* frequency (Hz), > 0                               */
  int npml[6];         /* x_lo, x_hi, y_lo, y_hi, z_lo, z_hi; 0 <= npml < n/2 */
  double v_ref;        /* PML reference speed (m/s), > 0; normally max(v)   */
  double r_coef;       /* PML target reflection coefficient in (0, 1)      */
} hx_grid;

/* A grid-node point source (Section 3.1: s = delta(x - x_s)) of complex
 * amplitude (amp_re, amp_im) for right-hand side `rhs`.  Several sources may
 * feed the same rhs.  Injected as amp / h^3 at the node, or spread over the 27
 * nodes with the row's consistent-mass weights when hx_solve_opts.source_spread
 * is 1 (a reading: it cancels the 1/(1-(kh)^2/12) far-field amplitude bias of
 * the plain delta).  Sources must lie inside the grid. */
typedef struct {
  int ix, iy, iz;
  int rhs;
  double amp_re, amp_im;
} hx_source;

/* ---------------------------------------------------------------- weights */

/* Fit the adaptive weight table (Section 2.2): for 1/G on the uniform grid
 * 0, d_inv_g, ..., inv_g_max (n_g = round(inv_g_max/d_inv_g) + 1 nodes) and
 * plane waves at every (theta, phi) pair of the given angle lists (degrees),
 * minimise ||H w - g||^2 + lambda ||D P w||^2 over the 5 free weights per
 * node, with H, g of Eq. linear_basic (H2 with the constant term derived from
 * Eq. vtilde), D the first-order forward difference along 1/G of each weight
 * series and P the series-major permutation.  Solved in FP64 by sequential
 * Givens QR of the stacked banded system (no normal equations).
 *   table_out: caller-owned host array of capacity doubles; receives
 *              n_g rows of 7: [ws1, ws2, ws3, wm1, wm2, wm3, wm4] with
 *              PER-POINT mass weights (wm1 + 6 wm2 + 12 wm3 + 8 wm4 = 1).
 *   n_g_out:   receives n_g (also when capacity is too small, with HX_ERR_ARG).
 * Needs no context and no GPU.  Errors: HX_ERR_ARG (bad sizes, lambda <= 0,
 * capacity < 7 n_g), HX_ERR_NUMERIC (rank-deficient system). */
int hx_build_weight_table(const double* theta_deg, int n_theta,
                          const double* phi_deg, int n_phi,
                          double inv_g_max, double d_inv_g, double lambda,
                          double* table_out, int capacity, int* n_g_out);

/* Non-adaptive weights (Eq. eq_cost of Section 2.2): ONE weight vector fitted
 * to the plane waves of all n listed 1/G values (and all angle pairs) --
 * the paper's G4 stencil for {1/4} and Gm for {1/4, 1/6, 1/8, 1/10}.  Minimum-
 * norm least squares (a single G leaves a 2-dimensional family of minimisers).
 *   w7_out: caller-owned [7] = [ws1, ws2, ws3, wm1, wm2, wm3, wm4], per-point
 *           mass weights as in hx_build_weight_table.
 * A table whose every row is w7 (hx_set_table) makes every operator call
 * use that fixed stencil.  Needs no context and no GPU.  Errors: HX_ERR_ARG
 * (1/G outside (0, 0.5], empty lists), HX_ERR_NUMERIC. */
int hx_fit_joint_weights(const double* inv_g, int n, const double* theta_deg, int n_theta,
                         const double* phi_deg, int n_phi, double* w7_out);

/* ---------------------------------------------------------------- context */

/* Create a context bound to CUDA device `device`.  *out is NULL on failure. */
int hx_ctx_create(hx_ctx** out, int device);
void hx_ctx_destroy(hx_ctx* ctx);
/* Message of the last failed call on ctx (static "" when none; "no context"
 * for ctx == NULL).  Valid until the next call on ctx. */
const char* hx_last_error(const hx_ctx* ctx);

/* Install the weight table used by every later operator call on ctx:
 * table_host [n_g][7] as produced by hx_build_weight_table, nodes at
 * 1/G = i * d_inv_g.  Copied (FP64 and FP32 forms) to the device; the host
 * array may be freed on return.  Synchronous.  Errors: HX_ERR_ARG (n_g < 2,
 * d_inv_g <= 0, non-finite entries), HX_ERR_OOM, HX_ERR_CUDA. */
int hx_set_table(hx_ctx* ctx, const double* table_host, int n_g, double d_inv_g);

/* Roles of a table in hx_set_table_ex. */
enum { HX_TABLE_BOTH = 0, HX_TABLE_OPERATOR = 1, HX_TABLE_PRECONDITIONER = 2 };

/* hx_set_table for one role: HX_TABLE_OPERATOR sets the table of the operator
 * itself (hx_apply_operator, hx_row_coefficients, hx_assemble_csr, the Krylov
 * operator and FP64 residual of hx_solve) and leaves hx_solve's multigrid
 * preconditioner on the table it used so far; HX_TABLE_PRECONDITIONER sets the
 * preconditioner's only (the operator table must exist); HX_TABLE_BOTH is
 * hx_set_table.  Lets a fixed stencil -- the paper's non-adaptive G4 or Gm
 * (hx_fit_joint_weights) -- be solved with the adaptive preconditioner,
 * which only has to approximate A^-1.  Errors as hx_set_table, plus
 * HX_ERR_STATE. */
int hx_set_table_ex(hx_ctx* ctx, const double* table_host, int n_g, double d_inv_g, int which);

/* Weights of an operator row (hx_set_operator_form). */
enum { HX_WEIGHTS_GA = 0, HX_WEIGHTS_GAM = 1 };

/* Operator variants of the paper for every later call on ctx that forms the
 * operator itself (hx_apply_operator, hx_stencil_sweep, hx_row_coefficients,
 * hx_assemble_csr, hx_assemble_csr_noalloc, and the Krylov operator and FP64
 * residual of hx_solve; hx_solve's multigrid preconditioner stays GA with the
 * second mass form, it only has to approximate A^-1):
 *   weights   HX_WEIGHTS_GA (default): each row takes the weights of its own
 *             G (Section 3.1, GA); HX_WEIGHTS_GAM: the mean of the weights of
 *             the stencil points inside the grid, each at its own G (GAm);
 *   mass_form 2 (default): the second form of Eq. 8, omega^2/kappa at the
 *             collocation point; 1: the first form, omega^2/kappa_j at each
 *             of the 27 points.
 * A variant other than (GA, 2) runs on the one-thread-per-row kernels (the
 * fields of a launch back to back), slower than the z-marching kernels.
 * hx_apply_batched refuses variants.  Errors: HX_ERR_ARG. */
int hx_set_operator_form(hx_ctx* ctx, int weights, int mass_form);

/* Heterogeneous density and attenuation (Eq. 2 and Eqs. 1.1-1.4; the paper's
 * benchmarks use b = 1 and no attenuation, Section 3.1) for every later call
 * on ctx that forms the operator itself (the calls listed under
 * hx_set_operator_form; hx_solve's preconditioner keeps b = 1, no Q):
 *   buoyancy_dev: float32 [nz][ny][nx] b = 1/rho per node, > 0, in any unit
 *                 (the operator is linear in b); NULL = 1.  Each second
 *                 difference becomes the conservative form with b at the half
 *                 nodes (the mean of the two nodes; the node's own b where the
 *                 other lies outside the grid) and the mass omega^2 b / v^2;
 *   inv_q_dev:    float32 [nz][ny][nx] 1/Q per node, >= 0; NULL = no
 *                 attenuation.  The velocity becomes c* = v (1 - i/(2Q)), so
 *                 waves decay as exp(-Im(omega/c*) r) (exp(-i omega t)); the
 *                 weights still follow the real G = v / (f h).
 * The arrays are caller-owned and read by those calls with the call's grid
 * size: keep them alive and sized for every grid used until
 * hx_set_medium(ctx, NULL, NULL).  A medium runs on the one-thread-per-row
 * kernels; hx_apply_batched refuses it.  Errors: HX_ERR_ARG (null ctx). */
int hx_set_medium(hx_ctx* ctx, const float* buoyancy_dev, const float* inv_q_dev);

/* ---------------------------------------------------------------- operator */

/* Flag or-ed into hx_apply_operator's precision argument (see there). */
#define HX_APPLY_DIRECT 0x100

/* y = A x for nrhs right-hand sides, A the impedance matrix [M + S] of Eq. 3
 * built on the fly per row (Eqs. 4-8 with the GA weight selection): the row's
 * 1/G = f h / v is looked up in the table by linear interpolation (clamped to
 * the table), the stiffness is sum_d T_d[delta_d p] (stretched second
 * differences averaged over the transverse 3x3 plane with weights
 * ws1 + 2ws2/3 + ws3/2, ws2/12, ws3/8) and the mass is the second form of
 * Eq. 8 with kappa at the collocation point.  shift_beta != 0 replaces
 * omega^2 by (1 + i shift_beta) omega^2 (the complex-shifted operator of the
 * preconditioner; 0 gives the paper's operator).
 *   precision 32: x, y complex64, arithmetic FP32 (table in FP32);
 *   precision 64: x, y complex128, arithmetic FP64;
 *   | HX_APPLY_DIRECT: use the one-thread-per-row kernel (coefficients formed
 *   per row, neighbours through the read-only cache) that the multigrid uses
 *   on small coarse grids, instead of the tiled z-marching kernel.
 *   x_dev, y_dev: [nrhs][nz][ny][nx], must not overlap.
 * Velocities are not validated here (see hx_solve).  Asynchronous on stream.
 * Errors: HX_ERR_ARG, HX_ERR_STATE (no table), HX_ERR_CUDA. */
int hx_apply_operator(hx_ctx* ctx, const hx_grid* grid, const float* v_dev,
                      double shift_beta, const void* x_dev, void* y_dev,
                      int nrhs, int precision, void* stream);

/* Kinds of hx_stencil_sweep. */
enum { HX_SWEEP_RESIDUAL = 1, HX_SWEEP_JACOBI = 2 };

/* The two stencil sweeps of the multigrid preconditioner, exposed for
 * callers that build their own smoothers (not in the paper, whose solver is
 * direct).  A_beta is the operator of hx_apply_operator with shift_beta.
 *   HX_SWEEP_RESIDUAL: y = b - A_beta x   (b_dev NULL: y = -A_beta x);
 *   HX_SWEEP_JACOBI:   y = x + omega D^-1 (b - A_beta x), D the diagonal of
 *                      A_beta (b_dev required).
 * precision 32 (complex64, FP32) or 64 (complex128, FP64); x_dev, b_dev,
 * y_dev are [nrhs][nz][ny][nx]; y must overlap neither x nor b.
 * Asynchronous on stream.  Errors: HX_ERR_ARG, HX_ERR_STATE, HX_ERR_CUDA. */
int hx_stencil_sweep(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta,
                     int kind, const void* x_dev, const void* b_dev, void* y_dev, int nrhs,
                     int precision, double omega, void* stream);

/* hx_apply_operator (kind 0) and hx_stencil_sweep (kind HX_SWEEP_RESIDUAL /
 * HX_SWEEP_JACOBI), complex64 only, on fields whose x rows are padded to
 * `pitch` elements: element (ix, iy, iz) of field r sits at
 * r * pitch * ny * nz + (iz * ny + iy) * pitch + ix.  The paper has no
 * counterpart: this is the layout hx_solve keeps its complex64 fields in
 * (pitch = nx rounded up to a multiple of 4), exposed for callers that hold
 * wavefields the same way.  An even pitch (16-byte rows) runs the kernel that
 * moves each plane tile with one tensor-memory-access copy; pitch = nx (any
 * nx) is the same as hx_apply_operator / hx_stencil_sweep.  Padding elements
 * are neither read nor written.  x, b 16-byte aligned, y 8-byte aligned; b
 * may be NULL for the residual (b = 0).  Asynchronous on stream.
 * Errors: HX_ERR_ARG (pitch odd and != nx, or < nx; alignment), HX_ERR_STATE,
 * HX_ERR_CUDA. */
int hx_stencil_pitched(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, double shift_beta,
                       int kind, const void* x_dev, const void* b_dev, void* y_dev, int nrhs,
                       int64_t pitch, double omega, void* stream);

/* One problem of hx_apply_batched: y = A x on its own grid and velocity. */
typedef struct {
  hx_grid grid;
  const float* v_dev;       /* velocity [nz][ny][nx]                              */
  const void* x_dev;        /* complex64 [nrhs][nz][ny][nx], 16-byte aligned      */
  void* y_dev;              /* complex64 [nrhs][nz][ny][nx], not overlapping x    */
  int nrhs;
} hx_apply_item;

/* hx_apply_operator (precision 32) for n problems of different sizes in ONE
 * persistent launch (not in the paper; it batches the subdomains and
 * requests a server or a domain-decomposed caller holds at once).  The work
 * is cut into items (problem, 32 x 8 column tile, z-chunk, block of RHS),
 * largest problems first; resident CTAs take items from a device counter
 * until none is left, so uneven sizes balance across the SMs.  Every output
 * equals hx_apply_operator's for the same kernel configuration on grids
 * where hx_apply_operator runs the same z-marching kernel (odd nx; with even
 * nx it takes the tensor-copy kernel, whose results differ only in FP32
 * rounding order).  The configuration is the context's forced one (ids 0-2),
 * else the default for the smallest nrhs.  shift_beta as in
 * hx_apply_operator, common to all.
 * The plan is staged through a pinned host buffer and a device buffer owned
 * by ctx, sized by the first call (later calls with no more work reuse them;
 * such calls can be recorded into a CUDA graph: a call made while the stream
 * is being captured and needing larger buffers fails with HX_ERR_STATE; a
 * recorded graph reads the plan from the staging buffer when it runs, so
 * replay it while no other hx_apply_batched call on ctx intervenes).
 * Asynchronous on stream.  Errors: HX_ERR_ARG, HX_ERR_STATE, HX_ERR_OOM,
 * HX_ERR_CUDA. */
int hx_apply_batched(hx_ctx* ctx, const hx_apply_item* items, int n, double shift_beta, void* stream);

/* The 27 complex128 coefficients of every row of A (same definition as
 * hx_apply_operator, FP64), written to coef_dev as [N][27][2] doubles in
 * offset order (dk, dj, di) with each of dk, dj, di running -1, 0, 1
 * (di fastest).  Entries whose neighbour lies outside the grid are written as
 * 0.  For tests and for users who assemble the matrix themselves.  Async. */
int hx_row_coefficients(hx_ctx* ctx, const hx_grid* grid, const float* v_dev,
                        double shift_beta, double* coef_dev, void* stream);

/* Assemble A as CSR on the host (complex128, lexicographic rows, columns
 * sorted, entries outside the grid omitted).  Caller-owned host arrays:
 * rowptr [N+1], col [nnz_cap], val [2*nnz_cap] (interleaved re, im);
 * nnz_cap >= 27 N always suffices.  v_dev is on the device; the call
 * synchronises `stream`.  Errors: HX_ERR_ARG (nnz_cap too small), others as
 * above. */
int hx_assemble_csr(hx_ctx* ctx, const hx_grid* grid, const float* v_dev,
                    double shift_beta, int64_t* rowptr, int32_t* col,
                    double* val, int64_t nnz_cap, int64_t* nnz_out, void* stream);

/* Largest grid (nx*ny*nz) hx_assemble_csr_noalloc accepts: a 27^3 grid. */
#define HX_NOALLOC_MAX_POINTS 19683

/* hx_assemble_csr for callers that may not allocate device memory.  The
 * paper has no counterpart: this is a deployment convenience.  Some callers
 * cannot call cudaMalloc/cudaFree where they need the matrix -- their device
 * memory belongs to another allocator, they must avoid the device-wide
 * synchronisation of cudaFree, or their memory budget is fixed after
 * start-up.  hx_assemble_csr allocates a temporary device buffer for the
 * coefficients; this entry point allocates nothing and uses a fixed scratch
 * array compiled into the library (about 8.7 MB held on every GPU that loads
 * the library, until the process exits).
 *   Same arguments, output and result as hx_assemble_csr, for grids of at
 *   most HX_NOALLOC_MAX_POINTS points (HX_ERR_ARG with a message otherwise).
 *   The first call on each device looks up the scratch array's device address
 *   (cudaGetSymbolAddress) while the context's device is current, and later
 *   calls reuse that address; make that first call before any stream
 *   capture, and do not reset the device (cudaDeviceReset) between calls.
 *   All calls share the one device scratch array and one host staging copy,
 *   on every GPU: two calls whose work overlapped would race and return each
 *   other's coefficients.  The library therefore holds a process-wide lock
 *   for the whole call (upload, kernel, stream synchronisation, CSR fill), so
 *   calls from any host threads or GPUs run one at a time.  The scratch keeps
 *   the last call's contents; every entry a call reads is written by that
 *   call first.  Synchronises `stream`. */
int hx_assemble_csr_noalloc(hx_ctx* ctx, const hx_grid* grid, const float* v_dev,
                            double shift_beta, int64_t* rowptr, int32_t* col,
                            double* val, int64_t nnz_cap, int64_t* nnz_out, void* stream);

/* ---------------------------------------------------------------- tuning */

/* The complex64 operator (hx_apply_operator with precision 32,
 * hx_stencil_sweep, hx_stencil_pitched and every complex64 stencil sweep of
 * hx_solve on grids above the direct-kernel size) runs on one of two
 * z-marching kernels, each in several launch configurations:
 *   ids 0-2: any row pitch (the only kernel for odd pitches, e.g. odd nx);
 *            per-thread asynchronous copies, x/y-PML rows in the same tiles;
 *            1, 2, 4 RHS per CTA;
 *   ids 3-8: even row pitch (16-byte rows: even nx, or the padded layout
 *            hx_solve uses); one tensor-memory-access copy per plane tile,
 *            the x/y-PML rows in a separate kernel; (8 rows, 1 / 2 / 4 / 8
 *            RHS) and (16 rows, 2 / 4 RHS) per CTA.
 * The automatic choice for an even pitch is the second kernel.  All compute
 * the same operator (results differ only in FP32 rounding order); their
 * speed depends on the grid and nrhs (the first is faster on small grids with
 * thick PML, where the second kernel's separate PML rows weigh more).  A
 * configuration that does not serve a launch's layout is replaced by the
 * automatic choice.  The
 * paper has no counterpart (its solver is a sparse direct factorisation);
 * this only chooses between launch shapes.  hx_kernel_config_info returns
 * the number of configurations and, for a valid cfg, writes its rows per
 * thread (1 for all) and RHS per CTA (either pointer may be NULL).  Needs no
 * context. */
int hx_kernel_config_info(int cfg, int* rows_per_thread, int* rhs_per_cta);

/* Force configuration cfg for every later complex64 launch on ctx; cfg = -1
 * restores the automatic choice (the hx_autotune result recorded for the
 * launch's grid size and nrhs, else a default by nrhs).  Errors: HX_ERR_ARG. */
int hx_set_kernel_config(hx_ctx* ctx, int cfg);

/* Time every configuration of the complex64 apply that serves this grid's
 * own layout (pitch = nx: all ids for even nx, 0-2 for odd nx; shifted form,
 * nrhs fields, one warm-up then ncalls launches each, CUDA events on stream;
 * configurations with at least twice nrhs RHS per CTA are skipped) on this
 * grid and velocity, and record the fastest for (nx, ny, nz, nrhs) in ctx;
 * later hx_apply_operator / hx_solve launches of that size use it (hx_solve
 * tunes its own padded layout itself when this size has no entry).  The
 * damped-Jacobi sweep of the shifted operator is timed the same way and its
 * fastest configuration recorded apart, for the sweeps (hx_stencil_sweep and
 * the solver's smoother); best_cfg and ms_out report the apply.
 *   best_cfg: receives the chosen configuration (may be NULL);
 *   ms_out:   receives up to ms_cap per-launch times in ms, by configuration
 *             id (1e300 for configurations not timed; may be NULL).
 * Allocates two temporary complex64 fields (nrhs * N each) and frees them;
 * synchronises stream; refuses to run while stream is being captured
 * (HX_ERR_STATE).  Errors: HX_ERR_ARG, HX_ERR_STATE, HX_ERR_OOM, HX_ERR_CUDA. */
int hx_autotune(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, int nrhs, int ncalls,
                int* best_cfg, double* ms_out, int ms_cap, void* stream);

/* ---------------------------------------------------------------- solve */

enum { HX_SOLVE_MIXED = 0, HX_SOLVE_FP64 = 1 };

/* Options of hx_solve (hx_solve_default_opts fills the defaults shown). */
typedef struct {
  int mode;              /* HX_SOLVE_MIXED (default): complex64 Krylov + multigrid
                            inner solves inside FP64 iterative refinement;
                            HX_SOLVE_FP64: the same Krylov + multigrid in FP64   */
  double tol;            /* stop when every RHS has ||s - A x|| <= tol ||s||,
                            residual computed in FP64 (default 1e-10)            */
  double inner_tol;      /* relative residual reduction of each complex64 inner
                            solve (mixed mode; default 1e-4)                    */
  int max_outer;         /* refinement steps (default 12)                         */
  int max_iter;          /* BiCGStab iterations per inner solve (default 2000)    */
  double shift_beta;     /* complex shift of the preconditioner (default 1.0)    */
  int mg_levels;         /* multigrid levels incl. the fine grid; 0 = automatic   */
  int nu_pre, nu_post;   /* damped-Jacobi sweeps before / after coarse correction
                            (default 3, 3)                                        */
  int coarse_sweeps;     /* damped-Jacobi sweeps on the coarsest level when it is
                            not solved exactly (default 4)                        */
  double omega_jacobi;   /* Jacobi damping (default 0.6)                          */
  int source_spread;     /* 0: grid delta (default); 1: consistent-mass spread    */
  int initial_guess;     /* 1: wavefield_dev holds the starting iterate           */
  int check_every;       /* iterations between host convergence checks (2)       */
  int coarse_galerkin;   /* 1: coarse operators R A P (Galerkin); 0 (default):
                            the stencil rediscretised at 2^l h                    */
  double pml_cap;        /* the preconditioner's PML damping is capped at
                            gamma <= cap * omega.  pml_cap > 0: cap = pml_cap;
                            0: no cap; < 0 (default -15): cap =
                            min(1, |pml_cap| omega / gamma0), gamma0 the
                            largest damping of the grid's PML faces (tighter
                            for thin, strongly damped layers at low
                            frequency).  Damped Jacobi diverges where the
                            stretching rotates one axis's coefficients far from
                            the others; the preconditioner only has to
                            approximate A^-1, and the Krylov operator keeps the
                            true PML.                                           */
  int use_graphs;        /* 1 (default): each block of check_every Krylov
                            iterations is captured once per call as a CUDA graph
                            and replayed (not while hx_profile timing is on);
                            0: direct launches                                    */
  int autotune;          /* 1 (default): the first mixed solve of a grid size and
                            nrhs with at least 2^18 point*RHS times the complex64
                            kernel configurations on the fine level (using the
                            solver's own buffers, before the solve) and keeps the
                            fastest in the context (see hx_autotune); 0: no     */
  double time_limit_s;   /* > 0: stop at the first convergence check after this
                            many seconds of solving and return
                            HX_ERR_NOT_CONVERGED with the best iterate (a
                            deadline for serving); 0 (default): no limit        */
  const int* cancel;     /* non-NULL: a host int read (atomically) where the host
                            synchronises anyway; once non-zero the solve stops
                            with HX_ERR_CANCELLED and the best iterate.  Another
                            thread may set it at any time.  NULL (default)     */
  int nu_coarse;         /* > 0 (default 2): damped-Jacobi sweeps before and after
                            the coarse correction on the levels below the fine
                            one (the fine level keeps nu_pre / nu_post); 0:
                            nu_pre / nu_post on every level                     */
  double bicg_kappa;     /* BiCGStab's omega safeguard (Sleijpen and van der
                            Vorst, 1995): where |cos| of the angle between t and
                            s is below kappa, omega = (t, s) / (t, t) is scaled
                            by kappa / |cos|, which keeps the minimal-residual
                            step from stalling the Bi-CG part on strongly
                            complex spectra.  0 (default) disables; 0.7 is the
                            published choice; must be in [0, 1).  It removes
                            stalls on strongly heterogeneous models (5-7x
                            fewer iterations there) but costs 5-15 % more
                            iterations on smooth ones                         */
  int coarse_velocity;   /* the preconditioner's coarse-level velocity, from the
                            next finer level: 0 (default) injection (the fine
                            node under the coarse one); 1 the full-weighting
                            average of 1/v^2 over its 27 fine neighbours      */
} hx_solve_opts;

typedef struct {
  int status;               /* same as the return value                          */
  int outer_iters;          /* FP64 residual evaluations after the first          */
  int inner_iters;          /* BiCGStab iterations summed over inner solves       */
  int mg_levels;            /* levels used                                        */
  double rel_residual;      /* max over RHS of ||s - A x|| / ||s|| (FP64)         */
  double setup_ms, solve_ms;
} hx_solve_report;

void hx_solve_default_opts(hx_solve_opts* opts);

/* ---------------------------------------------------------------- profiling */

/* Kernel classes timed by the profiler. */
enum {
  HX_PROF_APPLY32 = 0,   /* fine-level y = A x, complex64 (Krylov operator)      */
  HX_PROF_SMOOTH32 = 1,  /* fine-level Jacobi / residual sweeps, complex64       */
  HX_PROF_APPLY64 = 2,   /* fine-level FP64 operator (residual or Krylov)        */
  HX_PROF_SMOOTH64 = 3,  /* fine-level Jacobi / residual sweeps, complex128      */
  HX_PROF_KINDS = 4
};

/* Enable (1) or disable (0) per-launch timing of the fine-level operator
 * kernels inside hx_solve and reset the counters.  When enabled, each such
 * launch is bracketed by a CUDA event pair on the solve's stream and its
 * duration, launch count and algorithmic bytes (x, b read + y written once,
 * v read once: (8|16) * (2|3) * N * nrhs + 4 N) are accumulated; read them
 * with hx_profile_read.  Also counts every kernel the library launches.
 * While timing is on, hx_solve launches kernels directly instead of replaying
 * CUDA graphs.  enable = 0 resets the counters and turns timing off (the
 * launch count of kind -1 keeps counting). */
int hx_profile(hx_ctx* ctx, int enable);

/* kind in [0, HX_PROF_KINDS): launches, summed duration (ms) and summed
 * algorithmic bytes of that class since hx_profile(ctx, 1).  kind = -1:
 * launches = all kernels launched by the library on this context (any
 * class, also when timing is off), total_ms = bytes = 0. */
int hx_profile_read(hx_ctx* ctx, int kind, int64_t* launches, double* total_ms,
                    double* algo_bytes);

/* Measured FP64 fused-multiply-add throughput of the context's GPU, in
 * GFLOP/s (2 flops per FMA).  The paper has no counterpart: this is the
 * roofline of the complex128 kernels (the plain FP64 solve and the FP64
 * residual of the mixed form), which run on the FP64 units and are bounded by
 * their rate rather than by HBM.  Launches a short kernel of independent FMA
 * chains (one warm-up launch, then the best of three, CUDA events on stream),
 * allocates and frees an 8-byte-per-block sink, synchronises stream.
 * Errors: HX_ERR_ARG (null gflops), HX_ERR_CUDA. */
int hx_measure_fp64_peak(hx_ctx* ctx, double* gflops, void* stream);

/* Solve [M + S] p = s (Eq. 3) for nrhs right-hand sides built from point
 * sources (Section 3.1), GA weights per row, with the given grid/PML.
 * Method (not in the paper, which uses a sparse direct solver): BiCGStab
 * right-preconditioned by a V-cycle of the complex-shifted operator
 * (omega^2 -> (1 + i beta) omega^2) on vertex-centred grids coarsened by 2,
 * with Galerkin coarse operators R A P (or, with coarse_galerkin = 0, the
 * same stencil and PML profile rediscretised at 2^l h on injected
 * velocities, 1/G clamped to the table), damped-Jacobi smoothing,
 * full-weighting restriction, trilinear prolongation and an exact dense solve
 * of the coarsest level (at most 512 nodes).  Mixed mode runs that in
 * complex64 and corrects an FP64 iterate with FP64 residuals until opts.tol.
 *   v_dev: float32 [nz][ny][nx], every value finite, > 0 and with
 *          f h / v <= the table's largest 1/G (HX_ERR_ARG otherwise).
 *   src:   host array of nsrc sources; every rhs in [0, nrhs) must have one.
 *   wavefield_dev: complex128 [nrhs][nz][ny][nx], receives p (and holds the
 *          initial guess when opts->initial_guess).
 *   opts:  NULL = defaults.  report: may be NULL.
 * The ctx keeps the workspaces for the grid size and nrhs (reused by later
 * calls).  Synchronises `stream` (convergence checks read norms on the host).
 * Errors: HX_ERR_ARG, HX_ERR_STATE, HX_ERR_OOM, HX_ERR_CUDA, HX_ERR_NUMERIC
 * (breakdown / non-finite residual), HX_ERR_NOT_CONVERGED (best iterate kept). */
int hx_solve(hx_ctx* ctx, const hx_grid* grid, const float* v_dev, const hx_source* src,
             int nsrc, int nrhs, void* wavefield_dev, const hx_solve_opts* opts,
             hx_solve_report* report, void* stream);

/* ---------------------------------------------------------------- serving */

/* A request-serving engine for hx_solve (not part of the paper, whose solves
 * run one at a time under a direct solver).  It keeps `slots` worker threads,
 * each with its own context and CUDA stream on one device, so the solves of
 * different requests overlap on the GPU; a request is admitted as soon as a
 * slot is free and its estimated device memory fits in the budget next to
 * the requests in flight (in the configured order: the selected request waits
 * while it does not fit, and so do the requests behind it).  Velocity models stay
 * resident on the device by model id, and every worker keeps its latest
 * solver workspace (multigrid hierarchy and Krylov vectors) across requests of
 * the same grid size and nrhs, so a model served at a new frequency only
 * rebuilds its PML coefficients and coarsest inverse.  Every request is
 * solved exactly as a lone hx_solve with the same options would solve it
 * (options are taken as given, hx_solve_opts.autotune is forced to 0 so that
 * no result depends on timing), so results do not depend on the mix. */
typedef struct hx_server hx_server;

typedef struct {
  int device;               /* CUDA device                                        */
  int slots;                /* concurrent requests (worker threads), >= 1         */
  double mem_budget;        /* bytes of device memory for admitted requests and
                               resident models; <= 0: 85% of the free memory at
                               creation                                          */
  const double* table;      /* weight table [n_g][7] (hx_build_weight_table),
                               copied at creation                                 */
  int n_g;
  double d_inv_g;
  int order;                /* admission order: 0 first come, first served; 1 the
                               smallest queued request (grid points x nrhs)
                               first, which keeps small requests from waiting
                               behind large ones under load                       */
  double max_wait_s;        /* order 1: a request that has waited this long or
                               longer is admitted before the others, oldest
                               first (bounds how long a large request can be
                               passed over); 0: no bound                         */
} hx_server_config;

typedef struct {
  uint64_t model_id;        /* velocity model identity: requests with the same id
                               (and grid size) share one device copy             */
  const float* v_host;      /* velocity [nz][ny][nx]; read when the model is not
                               resident; must stay valid until the request ends  */
  hx_grid grid;
  const hx_source* src;     /* copied at submission                               */
  int nsrc, nrhs;
  void* wavefield_host;     /* complex128 [nrhs][nz][ny][nx], written when the
                               request completes; must stay valid until then     */
  const hx_solve_opts* opts;/* NULL = hx_solve_default_opts; copied at submission;
                               the server sets autotune = 0 and its own cancel
                               flag (see hx_server_cancel)                        */
} hx_request;

typedef struct {
  int status;               /* hx_solve's status (or HX_ERR_OOM / HX_ERR_ARG from
                               admission)                                         */
  hx_solve_report report;
  double queue_ms;          /* submission -> start on a worker                    */
  double run_ms;            /* start -> wavefield on the host                     */
  double latency_ms;        /* submission -> completion                           */
  int worker;               /* slot that served it                                */
} hx_request_result;

typedef struct {
  int64_t submitted, completed, failed;
  double p50_ms, p99_ms, max_ms;   /* latency percentiles of completed requests   */
  double point_rhs;                /* sum of N * nrhs over completed requests     */
  double busy_s;                   /* first submission -> last completion (s)     */
  double peak_committed;           /* peak bytes committed by admission           */
  int max_concurrent;              /* most requests on the GPU at once            */
  int64_t cancelled;               /* requests ended by hx_server_cancel (also
                                      counted in failed)                          */
} hx_server_stats;

/* Create the engine (starts the worker threads).  Errors: HX_ERR_ARG,
 * HX_ERR_CUDA, HX_ERR_OOM; *out is NULL on failure. */
int hx_server_create(hx_server** out, const hx_server_config* cfg);
/* Queue a request; returns at once with *ticket (>= 0).  Errors: HX_ERR_ARG
 * (invalid grid, sources, buffers; the request is not queued), HX_ERR_OOM
 * (the request alone exceeds the memory budget). */
int hx_server_submit(hx_server* srv, const hx_request* req, int64_t* ticket);
/* Wait until request `ticket` completes (timeout_s < 0: no limit) and fill
 * *res (may be NULL).  Returns the request's status, or HX_ERR_TIMEOUT when
 * timeout_s passed first (the request keeps running), HX_ERR_ARG for an
 * unknown ticket.  A ticket can be waited for once. */
int hx_server_wait(hx_server* srv, int64_t ticket, double timeout_s, hx_request_result* res);
/* Statistics since creation (or the last reset).  reset = 1 clears them. */
int hx_server_get_stats(hx_server* srv, hx_server_stats* st, int reset);

/* Cancel a submitted request.  A queued request is removed and completes at
 * once with status HX_ERR_CANCELLED (its wavefield is not written); a running
 * one stops at its solve's next convergence check (see hx_solve_opts.cancel)
 * and completes with HX_ERR_CANCELLED, its best iterate written.  The result
 * is still collected with hx_server_wait.  Errors: HX_ERR_ARG (unknown or
 * already collected ticket), HX_ERR_STATE (already finished). */
int hx_server_cancel(hx_server* srv, int64_t ticket);
/* Finish the queued requests, stop the workers and free everything. */
void hx_server_destroy(hx_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* HX27_H */
