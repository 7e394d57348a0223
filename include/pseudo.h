/*
 * pseudo.h -- C ABI of the B300 (sm_103a) pseudospectra library.
 *
 * The library evaluates sigma_min(C - zI) at every point z of a grid, for a
 * dense square complex matrix C given through its complex Schur factor T
 * (C = Q T Q^H, T upper triangular; Sec. 2.1 and SM2.1 of the paper:
 * M = T, S = I, so sigma(C - zI) = sigma(T - zI) and no QR per point is needed).
 * The epsilon-pseudospectrum is {z : sigma_min(C - zI) < eps} (Sec. 1, eq.
 * (defSquareSVD)); the library also returns that membership per level.
 *
 * Two methods are exposed (pseudo_opts.mode):
 *   PSEUDO_INVLANC  inverse Lanczos on N(z)^{-1}, N(z) = (T - zI)^H (T - zI),
 *                   per point, through triangular solves with T - zI
 *                   (Sec. 1; the EigTool core the paper compares against).
 *   PSEUDO_RECYCLE  singular-subspace recycling (Alg. 3, psTriRecy): a fast
 *                   Rayleigh--Ritz-SVD on a recycled basis V (Alg. 1) with a
 *                   backward-stability test (eq. (tolC)); rejected points are
 *                   refined by LOBPCG-SVD on (T - zI)^{-H} (Alg. SM1.2) and
 *                   their singular vectors update V (Alg. 2).
 *
 * Conventions for every entry point:
 *   - Complex numbers are pseudo_c64 {re, im} (layout of cuDoubleComplex and
 *     of torch.complex128).
 *   - Return value: PSEUDO_OK (0), a positive warning (results written), or a
 *     negative error (nothing valid written).  pseudo_last_error() gives a
 *     thread-local message for the last non-zero return.
 *   - "device" pointers are CUDA device memory of the handle's device;
 *     "host" pointers are ordinary host memory.  Which one a pointer is
 *     is never guessed: it is stated per argument or by a flag.
 *   - All work is enqueued on the CUDA stream passed in (cudaStream_t cast to
 *     void*; NULL = legacy default stream).  Calls that return results to
 *     host memory synchronise that stream before returning.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef PSEUDO_B300_H
#define PSEUDO_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pseudo_ctx *pseudo_handle;
typedef struct { double re, im; } pseudo_c64;

enum {
    PSEUDO_OK = 0,
    PSEUDO_WARN_NOT_CONVERGED = 1, /* all outputs written; some points flagged */
    PSEUDO_ERR_ARG = -1,           /* invalid argument (null, size, range) */
    PSEUDO_ERR_UNSUPPORTED = -2,   /* e.g. m != n (rectangular input) */
    PSEUDO_ERR_CUDA = -3,          /* a CUDA call failed; see pseudo_last_error */
    PSEUDO_ERR_WORKSPACE = -4,     /* workspace too small or misaligned */
    PSEUDO_ERR_NONFINITE = -5,     /* NaN/Inf in T or z */
    PSEUDO_ERR_TIMEOUT = -6        /* an iteration cap was hit in a fatal place */
};

enum { PSEUDO_INVLANC = 0, PSEUDO_RECYCLE = 1 };
enum { PSEUDO_FP64 = 0, PSEUDO_MIXED = 1 };
/* pseudo_solve / pseudo_matvec only: the CUDA-core kernels instead of the tensor-core ones */
enum { PSEUDO_MIXED_CUDACORE = 2 };
/* pseudo_solve only: the solve in double-single arithmetic on the FP32 units */
enum { PSEUDO_DOUBLE_SINGLE = 3 };
/* pseudo_opts.fp32_solver: chosen per matrix order from the tuned table */
enum { PSEUDO_SOLVER_AUTO = 2 };
/* pseudo_opts.fp32_solver: the tensor-core solve in a fixed form, 16 right-hand
 * sides per CTA (2-stage copy ring, two CTAs per SM) or 32 (4-stage ring, one
 * CTA per SM); plain 0 takes the 32-column form from padded order 4096 up */
enum { PSEUDO_SOLVER_TC16 = 3, PSEUDO_SOLVER_TC32 = 4 };

/* grid traversal of the recycling path (pseudo_opts.traversal):
 * BATCH_ZIGZAG = the batch-zigzag order of Sec. 2.3 with column batches of
 * batch_b points (default); HILBERT, MORTON = the Hilbert curve and the
 * Z-order that Sec. 5 names as locality-preserving alternatives, on the
 * smallest 2^q x 2^q square holding the grid, points outside it skipped. */
enum { PSEUDO_TRAVERSE_BATCH_ZIGZAG = 0, PSEUDO_TRAVERSE_HILBERT = 1, PSEUDO_TRAVERSE_MORTON = 2 };

/* per-point flags (flags_out) */
enum {
    PSEUDO_PT_ACCEPTED = 1,      /* recycled Ritz value accepted (no refinement) */
    PSEUDO_PT_REFINED = 2,       /* refined by LOBPCG-SVD / Lanczos */
    PSEUDO_PT_NOT_CONVERGED = 4, /* iteration cap hit; best estimate returned */
    PSEUDO_PT_IR_FALLBACK = 8,   /* mixed precision: kappa too large for the FP32 solves; the
                                    point was redone in FP64 (or found singular to working
                                    precision, PSEUDO_PT_SINGULAR) */
    PSEUDO_PT_SINGULAR = 16      /* sigma_min(T - zI) is below FP64 working precision (z on a
                                    diagonal entry of T, or deep inside the pseudospectrum of a
                                    strongly nonnormal T): sigma_out is an upper bound at the
                                    rounding level and res_out = sigma_out / (||T||_2,est + |z|) */
};

/* Options; pseudo_opts_default() fills the paper's parameters (Sec. 4):
 * r = 6, eta = 1e-4, eps shift = 1e-14 ||C||^2, tau = 1e-10, omega = 1.6,
 * p_max = 60, b = 20. */
typedef struct {
    int mode;           /* PSEUDO_INVLANC | PSEUDO_RECYCLE */
    int precision;      /* PSEUDO_FP64 | PSEUDO_MIXED (FP32 solves + FP64 refinement) */
    int r;              /* LOBPCG block size r (paper 6) */
    int p_max;          /* cap on recycled blocks; k_max = p_max * r */
    int grid_nx, grid_ny; /* Cartesian layout of z[] (row-major, x fastest); 0 = unordered */
    int batch_b;        /* column-batch size b of the batch-zigzag traversal (paper 20) */
    int lanes;          /* independent recycle lanes processed side by side (0 = auto) */
    int shift_batch;    /* INVLANC: shifts per launch wave (0 = auto); RECYCLE: points each lane
                           takes per round (0 = 1: V is updated after every refined point) */
    double eps_shift_rel; /* epsilon = eps_shift_rel * ||T||_2^2 (paper 1e-14) */
    double tau;         /* eigen-gap tolerance of eq. (tau) (paper 1e-10) */
    double omega;       /* pruning threshold of eq. (omegaCond) (paper 1.6) */
    double eta;         /* backward-stability tolerance of eqs. (tolC), (tolSVD) (paper 1e-4) */
    double rtol;        /* accuracy target on sigma: points are accepted/converged only when
                           the a-posteriori relative error estimate is <= rtol/4; 0 = paper
                           tests only */
    int maxiter_lanczos; /* Lanczos steps cap (1 .. 64) */
    int maxiter_lobpcg;  /* LOBPCG iterations cap */
    int max_ir;          /* iterative-refinement steps cap per solve (mixed precision) */
    int io_host;        /* 1: z/sigma/res/flags/member pointers of pseudo_grid are host memory */
    uint64_t seed;      /* seed of the random start vectors */
    int profile;        /* 1: time every hot-kernel launch with CUDA events (pseudo_kernel_stats) */
    int fp32_solver;    /* mixed precision: the FP32 triangular solves run on 0 = the tensor
                           cores (tcgen05, operands split hi + lo into TF32, 3 products;
                           16 or 32 right-hand sides per CTA by order), PSEUDO_SOLVER_TC16 /
                           PSEUDO_SOLVER_TC32 = the tensor cores in that form, 1 = the CUDA
                           cores (FP32 FMA), PSEUDO_SOLVER_AUTO (default) = the choice of the
                           library's tuned table for the matrix order (pseudo_tuned_config) */
    int traversal;      /* RECYCLE on a Cartesian grid: the visiting order, PSEUDO_TRAVERSE_* */
    int device_loop;    /* INVLANC: 1 (default) = the Lanczos driver's loop runs on the device,
                           captured once per call as a CUDA graph whose conditional nodes
                           decide every step, finish and stop (no host round trip per step);
                           0 = the host reads the slot counts back after every step.  Kernel
                           profiling (profile = 1) always takes the host loop. */
} pseudo_opts;

typedef struct {
    int64_t sv_R;        /* triangular solves with T - zI or its adjoint, one per column */
    int64_t mv_M;        /* products of T (or T^H) with a vector, one per column */
    int64_t mv_M_fp64_refine; /* FP64 products spent in iterative refinement */
    int64_t n_points;
    int64_t n_accepted;  /* recycle mode: accepted from the recycled subspace */
    int64_t n_refined;   /* refined points (= recycling points) */
    int64_t n_not_converged;
    int64_t n_updates;   /* updateRecy calls */
    int64_t lanczos_steps;
    int64_t lobpcg_iters;
    int64_t n_fallback;  /* mixed precision: points handed to the FP64 pass (PSEUDO_PT_IR_FALLBACK) */
    /* device time in ms, summed over calls: the recycling path's phases in the
     * paper's breakdown (recySing; LOBPCG-SVD refinement with its start block;
     * values and residuals of the refined points; updateRecy), each from events
     * on the call's stream around the phase (0 in inverse-Lanczos mode), and
     * whole pseudo_grid calls in either mode */
    double ms_recysing, ms_refine, ms_update, ms_polish, ms_total;
    int64_t n_singular;  /* of those, points found singular to working precision (PSEUDO_PT_SINGULAR) */
    int64_t n_rtilde_capped; /* recycle mode: recySing evaluations whose r~ of eq. (tau) exceeded the
                                16 columns the second Rayleigh--Ritz step keeps */
    int64_t n_graph_launches; /* launches of the device-driven Lanczos loop's graph (device_loop) */
    int64_t n_graph_builds;   /* of those graphs, captured and instantiated (the others were cached:
                                 a call with the same workspace, inputs, outputs and options) */
    double ms_graph_build;    /* host time spent capturing and instantiating them */
} pseudo_stats_t;

/* Per-kernel-class accounting (filled when pseudo_opts.profile = 1): launches,
 * device time from CUDA events recorded on the launching stream around each
 * launch, and the algorithmic work of those launches (flops: real floating-point
 * operations of the textbook algorithm, 8 per complex multiply-add; bytes: the
 * operands each launch must read and write at least once). */
enum {
    PSEUDO_K_TRSV32 = 0,  /* multi-shift triangular solve, FP32 arithmetic */
    PSEUDO_K_TRSV64,      /* multi-shift triangular solve, FP64 */
    PSEUDO_K_TRMV64,      /* triangular product / residual, FP64 */
    PSEUDO_K_TRMV_DS,     /* triangular product / residual, double-single on FP32 units */
    PSEUDO_K_RECYSING,    /* recycled Rayleigh--Ritz-SVD + residual, one CTA per point */
    PSEUDO_K_LANCZOS,     /* Lanczos reorthogonalisation */
    PSEUDO_K_TRSV_DS,     /* multi-shift triangular solve, double-single on FP32 units */
    PSEUDO_K_RECT_QR,     /* rectangular pencil: per-point QR of [T - zI; B], FP64 */
    PSEUDO_K_COUNT
};
typedef struct {
    int64_t launches;
    double ms, flops, bytes;
} pseudo_kstat;
int pseudo_kernel_stats(pseudo_handle h, int kclass, pseudo_kstat *out);

/* Fill *o with defaults. Returns PSEUDO_OK or PSEUDO_ERR_ARG (o == NULL). */
int pseudo_opts_default(pseudo_opts *o);

/* Create a handle from the output of the preliminary reduction (SM2).
 * Square C (SM2.1: M = T, S = I): m = n, T is the upper-triangular Schur factor.
 * Rectangular C with m_C >= 2n rows (SM2.2: M = [C_u; R_l], S = [I; 0]): m = 2n,
 *   rows 0..n-1 hold an upper-triangular T and rows n..2n-1 an upper-triangular
 *   B such that [T - zI; B] has the singular values of C - zI for every z (for
 *   example T = U^H C_u U from the Schur form of the top block and B the
 *   triangular factor of R_l U; the host reduction of the package's workloads
 *   module computes them).  Such a handle runs mode INVLANC in precision FP64
 *   only: every point factors its own pencil (Alg. 3's QR of eq. (triGen)).
 *   T         : column-major complex m x n with leading dimension ldT >= m;
 *               only the upper triangle of each n x n block (i <= j) is read.
 *   t_on_host : 1 if T is host memory, 0 if device memory.
 *   m, n      : m = n or m = 2n (any other m -> PSEUDO_ERR_UNSUPPORTED; m = 2n
 *               needs n <= 14000, else UNSUPPORTED).
 *   stream    : cudaStream_t for the set-up copies/kernels.
 * The library copies T (and B) into handle-owned device buffers (packed FP64
 * and FP32 panels of T and T^H; for m = 2n also FP64 panels of B and B^H and
 * the dense 2n x n pencil) -- the only device allocations the library makes;
 * the caller may free T on return.  Also computes ||M||_F and a 2-norm
 * estimate of M.  Errors: ARG (null/size), UNSUPPORTED (m not n or 2n),
 * NONFINITE, CUDA. */
int pseudo_create(const pseudo_c64 *T, int64_t ldT, int64_t m, int64_t n, int t_on_host,
                  void *stream, pseudo_handle *out);

/* Bytes of caller-provided device workspace that pseudo_grid needs for npts
 * points under options o.  Errors: ARG. */
int pseudo_workspace_bytes(pseudo_handle h, const pseudo_opts *o, int64_t npts, size_t *bytes);

/* sigma_min(T - z_j I) for j < npts (0 <= npts <= 2^31 - 1).
 *   z          : npts complex shifts (device, or host if o->io_host).
 *   eps_levels : host array of neps (<= 32) levels; may be NULL if neps == 0.
 *   sigma_out  : npts doubles (device/host as z).
 *   res_out    : npts doubles or NULL: ||N(z)x - s^2 x|| / (s * (||T||_2,est + |z|)) for the
 *                returned unit vector x and value s (the quantity eq. (tolC) bounds by eta).
 *   flags_out  : npts int32 PSEUDO_PT_* bits, or NULL.
 *   member_out : npts uint32 words, bit i set iff sigma < eps_levels[i] (strict), or NULL.
 *   workspace  : device memory of >= pseudo_workspace_bytes(...) bytes, 256-byte aligned.
 * Device arrays must be naturally aligned (z 16 bytes, sigma/res 8, flags/member
 * 4): a misaligned one gives PSEUDO_ERR_ARG before any work (host arrays, with
 * o->io_host, need no alignment).
 * Outputs are in the caller's order of z.  No device memory is allocated.
 * Returns OK, WARN_NOT_CONVERGED, or an error. */
int pseudo_grid(pseudo_handle h, const pseudo_c64 *z, int64_t npts, const double *eps_levels,
                int neps, const pseudo_opts *o, double *sigma_out, double *res_out,
                int32_t *flags_out, uint32_t *member_out, void *workspace,
                size_t workspace_bytes, void *stream);

/* Many independent problems in one call (a batch of matrices of uneven size,
 * each with its own grid): the same result as pseudo_grid on every (hs[m],
 * z[m], npts[m]) in turn, but the matrices run concurrently on the device so
 * that small ones, which cannot fill the GPU alone, fill it together.
 *   hs          : nmat distinct handles (host array).
 *   z, sigma_out, res_out, flags_out, member_out : host arrays of nmat
 *                 pointers, each as in pseudo_grid (res/flags/member arrays
 *                 and their entries may be NULL).
 *   npts        : host array of nmat point counts (0 allowed).
 *   eps_levels, neps, o : shared by all matrices, as in pseudo_grid, except that
 *                 every matrix's inverse-Lanczos loop is driven from its worker
 *                 thread (o->device_loop is not used): replayed conditional-node
 *                 graphs on the workers' streams overlapped less on the device
 *                 than host-driven loops did (measured).
 *   workspace   : device memory of >= pseudo_grid_batch_workspace_bytes(...).
 * Matrices are assigned to the workers by a fixed rule (largest first, balanced
 * by n^2 x npts), so repeated calls repeat the assignment.
 * Work is ordered after prior work on `stream`; later work on `stream` waits
 * for all of it.  Returns the largest non-negative status over the matrices,
 * or the first error (the message names the matrix). */
int pseudo_grid_batch_workspace_bytes(const pseudo_handle *hs, int nmat, const int64_t *npts,
                                      const pseudo_opts *o, size_t *bytes);
int pseudo_grid_batch(const pseudo_handle *hs, int nmat, const pseudo_c64 *const *z, const int64_t *npts,
                      const double *eps_levels, int neps, const pseudo_opts *o, double *const *sigma_out,
                      double *const *res_out, int32_t *const *flags_out, uint32_t *const *member_out,
                      void *workspace, size_t workspace_bytes, void *stream);

/* Recycle mode: where the lanes' recycled subspaces (Alg. 2 state) sit in the
 * workspace after pseudo_grid returns, for inspection.  out[11] = {lanes, k_max,
 * row stride of V and W (complex elements), byte offsets of V, W1 = T V,
 * W3 = T^H T V, W4 = T^H V (n x lanes*k_max row-major, lane l in columns
 * [l k_max, l k_max + k_max)), H1 = W1^H W1, H2 = W1^H V, L (k_max x k_max per
 * lane, row-major) and p (int per lane, blocks in use; k = p r columns valid)}.
 * Errors: ARG. */
int pseudo_recycle_state_layout(pseudo_handle h, const pseudo_opts *o, int64_t npts, int64_t *out);

/* The order in which the recycling path (PSEUDO_RECYCLE) visits the points of
 * a Cartesian grid.  PSEUDO_TRAVERSE_BATCH_ZIGZAG: the batch-zigzag traversal
 * of Sec. 2.3, eq. (batch): the grid is cut into column batches of b
 * vertically adjacent points (the top batch row is shorter when b does not
 * divide grid_ny); batch rows are taken from the bottom, swept in a row-wise
 * zigzag (the first left to right, the next right to left, and so on), and
 * the points of each batch are visited bottom to top.  PSEUDO_TRAVERSE_HILBERT
 * and PSEUDO_TRAVERSE_MORTON (Sec. 5): the Hilbert curve from (0, 0) to
 * (2^q - 1, 0), resp. the Z-order (x in the low bit), on the smallest 2^q x
 * 2^q square holding the grid, with the points outside the grid skipped.
 * The recycling path splits this sequence into `lanes` contiguous segments.
 *   npts             : number of points; must equal grid_nx * grid_ny when
 *                      grid_nx > 0 (at most 2^31 - 1).
 *   grid_nx, grid_ny : the layout of pseudo_opts (z[iy * grid_nx + ix]);
 *                      grid_nx = 0 means unordered points, visited in index
 *                      order.
 *   batch_b          : b >= 1 (pseudo_opts.batch_b; used by the batch zigzag).
 *   traversal        : PSEUDO_TRAVERSE_* (pseudo_opts.traversal).
 *   order            : caller-owned host array of npts int32, written with the
 *                      point indices in visiting order.
 * Host-only: needs no handle and no device.  Errors: ARG. */
int pseudo_traversal_order(int64_t npts, int grid_nx, int grid_ny, int batch_b, int traversal,
                           int32_t *order);

/* The library's tuned choices for a matrix of order n (the autotuner of the
 * multi-matrix batching; the paper has no counterpart): the FP32 solver kernel
 * that pseudo_opts.fp32_solver = PSEUDO_SOLVER_AUTO selects (0 tensor cores in
 * the form the order picks, PSEUDO_SOLVER_TC16 / TC32 tensor cores in that
 * form, 1 CUDA cores) and the number of Lanczos slots (shifts per solve launch)
 * that shift_batch = 0 selects in inverse-Lanczos mode.  The table comes from
 * an offline sweep on this part, per bucket of n.  Either pointer may be NULL.
 * Host-only.  Errors: ARG (n < 1). */
int pseudo_tuned_config(int64_t n, int *fp32_solver, int *slots);

/* Counters and phase timings accumulated since create or the last reset. */
int pseudo_stats(pseudo_handle h, pseudo_stats_t *out);
int pseudo_stats_reset(pseudo_handle h);

/* Problem facts of the handle: n, ||T||_F and the 2-norm estimate. */
int pseudo_info(pseudo_handle h, int64_t *n, double *norm_fro, double *norm2_est);

/* Release the handle and its device buffers.  NULL-safe. */
void pseudo_destroy(pseudo_handle h);

/* Thread-local message describing the last non-OK return ("" if none). */
const char *pseudo_last_error(void);

/* Number of CUDA kernel launches the library has made in this process (all
 * handles, all threads); differences around a call count its launches. */
int64_t pseudo_launch_count(void);

/* ---- kernel-level entry points (used by the tests; same rules as above) ----
 * All three need a square handle (m = n); a rectangular one gives UNSUPPORTED.
 *
 * pseudo_solve: X[:, c] <- (T - z_c I)^{-1} X[:, c] (adjoint = 0) or
 *               (T - z_c I)^{-H} X[:, c] (adjoint = 1) for c < ncols: the
 *               multi-shift triangular solve that applies R(z)^{-1} and R(z)^{-*}
 *               (Alg. 3, lobpcgSvd on R(z)^{-*}; sv_R in Table 2).
 *   X   : device, row-major n x ncols complex (element (i, c) at X[i*ncols + c]).
 *   z   : device, ncols complex shifts, one per column.
 *   precision : PSEUDO_FP64 (all FP64), PSEUDO_MIXED (FP32 arithmetic on the tensor
 *               cores), PSEUDO_MIXED_CUDACORE (FP32 on the CUDA cores) or
 *               PSEUDO_DOUBLE_SINGLE (double-single arithmetic on the CUDA cores,
 *               about 2^-46 relative per operation).
 *   workspace : device, >= pseudo_solve_workspace_bytes bytes, 256-byte aligned.
 *   X and z must be 16-byte aligned (PSEUDO_ERR_ARG otherwise).
 * pseudo_matvec: Y[:, c] <- B[:, c] - (T - z_c I)^{op} X[:, c] (subtract = 1) or
 *   Y[:, c] <- (T - z_c I)^{op} X[:, c] (subtract = 0, B ignored and may be NULL); the
 *   refinement residual of a shifted solve and the products T V, T^H V of Alg. 2.
 *   precision PSEUDO_FP64: IEEE double arithmetic; PSEUDO_MIXED: on the tensor cores,
 *   T and X split into 7 exact bf16 slices each (per-row / per-column power-of-two
 *   scaling), slice products accumulated exactly per level in FP32 and summed in
 *   double-single (about 2^-50 relative to the row and column maxima);
 *   PSEUDO_MIXED_CUDACORE: double-single arithmetic on the FP32 units (T split into
 *   two FP32 planes, exact products and two-sums; relative error about 2^-46).
 *   X, Y, B device row-major n x ncols complex (16-byte aligned, as is z); Y must not
 *   alias X. z may be NULL (z = 0).
 *   workspace : device, >= pseudo_matvec_workspace_bytes bytes, 256-byte aligned (used
 *   by PSEUDO_MIXED). */
int pseudo_matvec_workspace_bytes(pseudo_handle h, int64_t ncols, size_t *bytes);
int pseudo_solve_workspace_bytes(pseudo_handle h, int64_t ncols, size_t *bytes);
int pseudo_solve(pseudo_handle h, pseudo_c64 *X, const pseudo_c64 *z, int64_t ncols, int adjoint,
                 int precision, void *workspace, size_t workspace_bytes, void *stream);
int pseudo_matvec(pseudo_handle h, const pseudo_c64 *X, const pseudo_c64 *B, pseudo_c64 *Y,
                  const pseudo_c64 *z, int64_t ncols, int adjoint, int subtract, int precision,
                  void *workspace, size_t workspace_bytes, void *stream);

/* pseudo_set_wait_limit: the limit, in nanoseconds, of every bounded wait of
 * the tensor-core kernels of this handle (the mixed-precision solves and
 * products; default 10^9 = 1 s).  A wait that runs out makes its kernel stop,
 * let the copies and MMAs it has in flight finish, release its tensor memory
 * and record the failure; the call then returns PSEUDO_ERR_TIMEOUT with its
 * outputs invalid, and the handle stays usable.  0 makes any wait that is not
 * already satisfied give up at once (for testing that path).  No
 * counterpart in the paper: it is part of the library's failure handling.
 * Errors: ARG (h NULL). */
int pseudo_set_wait_limit(pseudo_handle h, uint64_t ns);

/* pseudo_solve_noalloc: the FP64 form of pseudo_solve without a workspace, for
 * callers that cannot allocate device memory (a process that reserved its whole
 * device-memory budget at start-up, or a latency-critical loop that must not
 * call cudaMalloc/cudaFree because they can synchronise the device).  The paper
 * has no counterpart: it is a library-usage entry point.
 *   X, z, ncols, adjoint, stream : as for pseudo_solve (X device, in place; z device;
 *   both 16-byte aligned).
 * Scratch: a fixed 16 MiB array inside the library (2^20 complex doubles), held
 * by every GPU that loads the library until the process exits.  The solve needs
 * ceil(ncols / 8) * n_pad * 8 of its elements (n_pad = n rounded up to 128), so
 * n = 2000 allows up to 512 columns per call; larger calls (and any ncols
 * above 2^20) return PSEUDO_ERR_ARG with a message and launch nothing.
 * The first call on a device looks up the array's device address (with the
 * handle's device current, which the call requires); make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: after a device reset (cudaDeviceReset, or anything else that tears
 * down the primary context) it is stale, so do not call this entry point
 * again in that process.  All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and corrupt each
 * other's results, so serialise them.  The array keeps the last call's
 * contents; the solve writes every scratch row before reading it, so nothing
 * has to be cleared.  No device memory is allocated or freed. */
int pseudo_solve_noalloc(pseudo_handle h, pseudo_c64 *X, const pseudo_c64 *z, int64_t ncols, int adjoint,
                         void *stream);


#ifdef __cplusplus
}
#endif
#endif
