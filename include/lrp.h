/*
 * lrp.h - C ABI of the GB300 (sm_103a) library for Parareal with low-rank
 * coarse solvers (Gander, Ohlberger, Rave, arXiv 2508.08873).
 *
 * Problem (Sec. 2): a linear semi-discretisation u_t = -A u + f on [0, T] is
 * split into N coarse intervals of M backward-Euler steps each (dt = T/(N M)).
 * The fine solver of interval i is F_i v = F_i' v + b_i (Eq. F_n_affine).
 * The coarse solver is the rank-R truncated SVD of F_i' plus b_i
 * (Eq. spectral_G), computed by the randomized SVD of Sec. 2.1, and Parareal
 * (Eq. def_Parareal) corrects the fine solves with it.
 *
 * Conventions shared by every entry point:
 *  - Intervals are 0-based: interval i maps t_i to t_{i+1} (the paper's n=i+1).
 *  - A vector of length n is contiguous; a batch of vectors is row-major
 *    (vector v occupies [v*n, (v+1)*n)).
 *  - Sources are separable, f(t, x) = sum_{q<Q} c_q(t) g_q(x): g is Q x n,
 *    and c holds c_q at the end of every fine step, c[(J-1)*Q + q] at
 *    t = J*dt for J = 1..N*M (fully implicit Euler samples f at t_{j+1});
 *    operators with an SDIRK stepper take two samples per step, at its stage
 *    times (lrp_operator_set_stepper).
 *  - Every pointer argument may be host memory or device memory of the
 *    context's device; the library detects which.  The caller owns all
 *    buffers it passes; the library owns the handles it returns and the device
 *    memory behind them.  Host outputs are complete when the call returns;
 *    device outputs are complete in stream order on the context's stream.
 *  - Errors are returned as lrp_status; nothing is thrown across the ABI.
 *    lrp_last_error() gives a message for the last failure on a context.
 *  - A context is used by one host thread at a time.
 *  - The inner product is the Euclidean one on the coefficient vectors, so
 *    the adjoint of F_i' is its transpose (Sec. 2.1, step 3).
 */
#ifndef LRP_H
#define LRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRP_OK = 0,
  LRP_EINVAL = 1,      /* bad argument (size, null pointer, unsupported shape) */
  LRP_ENOMEM = 2,      /* device allocation failed or the HBM budget is exceeded */
  LRP_ENOTCONV = 3,    /* an iteration cap was hit; outputs hold the last iterate */
  LRP_EBREAKDOWN = 4,  /* a zero pivot or a breakdown in an iterative solver */
  LRP_ETIMEOUT = 5,    /* a bounded device wait expired */
  LRP_ECUDA = 6,       /* a CUDA runtime error; see lrp_last_error() */
  LRP_EBUSY = 7,       /* the request queue is full */
  LRP_PENDING = 8      /* a served request has not finished yet */
} lrp_status;

/* Arithmetic of the coarse-solver build (rSVD steps 1-6).
 * LRP_PREC_F64:   sketches, orthonormalisation, SVD and factors in FP64.
 * LRP_PREC_MIXED: sketch propagation and orthonormalisation in FP32, the small
 *                 SVD in FP64, factors kept in FP32 and FP64.
 * Parareal fine solves, corrections and bounds are FP64 in both modes. */
typedef enum { LRP_PREC_F64 = 0, LRP_PREC_MIXED = 1 } lrp_precision;

typedef struct lrp_ctx lrp_ctx;
typedef struct lrp_operator lrp_operator;
typedef struct lrp_coarse lrp_coarse;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = no cap beyond the free memory).  The
 * context creates its own non-blocking stream. */
lrp_status lrp_create(lrp_ctx** out, int device, size_t hbm_budget_bytes);
void lrp_destroy(lrp_ctx* ctx);
/* Use the caller's cudaStream_t (passed as void*) for all later work; NULL
 * returns to the context's own stream.  The caller keeps ownership. */
lrp_status lrp_set_stream(lrp_ctx* ctx, void* cuda_stream);
void* lrp_get_stream(lrp_ctx* ctx);
/* Wait until all work of the context's stream has finished. */
lrp_status lrp_synchronize(lrp_ctx* ctx);
const char* lrp_status_string(lrp_status s);
const char* lrp_last_error(lrp_ctx* ctx);
/* Device bytes currently held by the context. */
size_t lrp_bytes_in_use(lrp_ctx* ctx);
/* Number of kernels the context has launched so far (all kernel families). */
long lrp_launch_count(lrp_ctx* ctx);

/* Launch tuning (0 = automatic, the default):
 *   "sweep_rows":    rows of a vector per CTA in the coarse sweep (128..2048,
 *                    a power of two; default 1024);
 *   "tri_cluster":   CTAs per tridiagonal system for small batches (1..8);
 *   "tri_chunk":     rows per chunk of the cluster tridiagonal kernel (8, 16);
 *   "tri_warp":      1 disables the one-warp-per-CTA FP64 cluster kernel that
 *                    FP64 batches with 256 < n <= 4096 and up to about 7
 *                    warps per SM sub-partition use by default, 2 uses it for
 *                    every FP64 batch with n <= 4096;
 *   "tri_wchunk":    rows per chunk of the one-warp FP64 cluster kernel (8 to
 *                    16; 0 = automatic);
 *   "tri_wblock":    one system per CTA of C warps (the one-warp kernel's
 *                    steps with the exchange in shared memory): 0 = automatic
 *                    (FP32 batches that do not take a cluster, and FP64
 *                    constant-coefficient batches beyond the cluster kernels'
 *                    range), 1 = always (FP64: at most 8 warps, else
 *                    LRP_EINVAL), 2 = never;
 *   "tri_wtoep":     the constant-coefficient variant of the one-warp kernels
 *                    (operators whose lo[1..n-1], di and up[0..n-2] are each
 *                    one value, no source term, n mod MM in {0, MM - 1}):
 *                    0 = automatic, 1 = always (LRP_EINVAL where it does not
 *                    apply), 2 = never;
 *   "tri_wsplit":    where the one-warp kernel runs the chunk-interior solve
 *                    of the next step: 0 = all of it between the cluster
 *                    barrier's arrive and wait, 1 (default) = its last third
 *                    of backward rows after the wait, beside the super system;
 *   "tri_spt":       systems per thread of the cluster tridiagonal kernel (1, 2);
 *   "tri_group":     systems per CTA of the one-CTA-per-system tridiagonal
 *                    kernel (1..16, at most 512 threads per CTA);
 *   "queue_cluster": CTAs per cluster of the batched 2D work queue (1..16,
 *                    a power of two);
 *   "orth_tc":       1 (default) orthonormalises the FP32 sketches of the mixed
 *                    mode by CholeskyQR2 on the tensor cores and lifts the
 *                    singular vectors there (sketch width <= 64, intervals
 *                    whose Gram passes the conditioning test); 0 uses
 *                    Gram-Schmidt and the SIMT lift throughout;
 *   "orth_cluster":  CTAs per interval of the shared-memory CGS2 kernel (a power
 *                    of two up to 16; -1 selects the one-CTA kernel);
 *   "krylov_cluster": CTAs per cluster of the 2D propagator (1..16, a power
 *                    of two; default: the most CTAs in flight whose Krylov
 *                    workspaces fit in 96 MB);
 *   "krylov_onchip": 0 (default) runs the conjugate gradients of symmetric
 *                    5-point operators with every Krylov vector on chip
 *                    (registers and shared memory of one thread-block
 *                    cluster per system) where the grid allows it (at most
 *                    512 columns and 512 rows in FP32, 256 rows in FP64;
 *                    time-dependent operators in FP32, every step on its
 *                    own couplings); 2 always uses the kernel with its
 *                    Krylov vectors in global memory;
 *   "krylov_block":  0 (default) or 4: propagations of two or more systems
 *                    without a source on symmetric 5-point operators (at
 *                    most 512 columns in FP32, 256 in FP64, 512 rows) solve
 *                    every step by block conjugate gradients over groups of
 *                    four consecutive systems (the paper's Sec. 2.2 remark
 *                    that the R + p sketch vectors can be propagated
 *                    together; one block Krylov space per group, fewer
 *                    iterations than four separate solves, block vectors in
 *                    a device workspace of the operator);
 *   "krylov_block_clusters": clusters in flight of the block CG (0 =
 *                    automatic: workspaces within 96 MB);
 *   "krylov_refine": FP64 steps of 5-point operators by
 *                    mixed-precision iterative refinement (FP64 residual,
 *                    FP32 correction from zero -- CG on the on-chip kernel
 *                    for symmetric operators, BiCGStab on the global-memory
 *                    kernel otherwise -- FP64 update, repeated until the
 *                    FP64 test of the Krylov kernels passes or the residual
 *                    reaches its rounding level 8 u_64 ||D^1/2 (|d| +
 *                    |B||x|)||; at most 60 rounds per step, else
 *                    LRP_ENOTCONV): 0 (default) or 1: nonsymmetric
 *                    operators always, symmetric ones wherever the FP32
 *                    on-chip kernel takes the grid (and the block CG was not
 *                    requested); 2 never (the FP64 Krylov kernels: on chip
 *                    where the grid fits, else in global memory).  The
 *                    batched solves (lrp_parareal_solve_batch) refine inside
 *                    their persistent queue kernel unless 2.  SDIRK steps
 *                    refine each stage solve on its stage matrix;
 *                    time-dependent operators refine when symmetric (their
 *                    nonsymmetric steps keep the FP64 Krylov kernels);
 *   "krylov_refine_digits": relative tolerance 10^-digits (1..7) of the FP32
 *                    correction solves (0 = automatic: 1e-3);
 *   "krylov_stage":  1 stages the stencil input of every FP32 pass of the
 *                    global-memory Krylov kernel (the CTA's rows and a halo
 *                    row on each side) in shared memory by one bulk copy of
 *                    the TMA engine per pass, completion on an mbarrier with
 *                    bounded waits (LRP_ETIMEOUT); results are bitwise those
 *                    of 0 (default: the stencil reads global memory through
 *                    L1), and on GB300 it measured no faster;
 *   "tri_refine":    1 computes the backward-Euler steps of FP64
 *                    propagations of time-invariant tridiagonal operators
 *                    to about 48 bits instead of in FP64 (n <= 4096,
 *                    forward, no source term) from FP32 solves: per step one
 *                    FP32 solve, then "tri_refine_rounds" corrections, each
 *                    the FP32 solve of the residual x_j - B y formed in pairs
 *                    of FP32 numbers (exact products by FMA, two-sum
 *                    additions, B's FP64 entries as hi + lo pairs), the state
 *                    carried as a pair (about 48 bits).  One system per CTA.
 *                    Results are not those of the FP64 kernels: after 256
 *                    steps of the adr1d operator (n = 4095) they differ by
 *                    2.7e-12 relative with one round, 1.4e-12 with two
 *                    (the 48-bit pair form of B enters every step alike).
 *                    Each round gains about u_32 kappa(B) on a step's error
 *                    and no residual test follows the last round, so it is
 *                    meant for well-conditioned steps, such as the
 *                    diagonally dominant backward-Euler matrices of
 *                    diffusion-advection-reaction operators.
 *                    0 (default) keeps the FP64 kernels;
 *   "tri_refine_rounds": correction rounds per step of tri_refine (1..3,
 *                    default 2);
 *   "tri_refine_cluster": 0 (default) one CTA of up to 16 warps per system
 *                    (block barriers), 1 a cluster of one-warp CTAs per
 *                    system for constant-coefficient operators (cluster
 *                    barriers; measured slower on GB300: 0.73 against
 *                    0.47 ms per 62-system launch of adr1d).
 * Results do not depend on these settings beyond rounding (the block
 * solver stops every system on the same residual test as the others). */
lrp_status lrp_set_param(lrp_ctx* ctx, const char* name, int value);
/* lrp_get_param reads the parameters above and, read-only, the launch shape
 * of the last on-chip CG launch of the context: "krylov_onchip_rows" (grid
 * rows per thread), "krylov_onchip_cs" (CTAs per cluster) and
 * "krylov_onchip_clusters" (clusters in flight); of the last 2D propagation,
 * whether it ran on the block CG: "krylov_block_last_systems" (systems per
 * block, 0 when it did not), "krylov_block_last_cs" (CTAs per cluster),
 * "krylov_block_last_clusters" (clusters in flight); 0 before the first
 * one.  A bounded wait of the block CG that expires returns LRP_ETIMEOUT. */
lrp_status lrp_get_param(lrp_ctx* ctx, const char* name, int* value);

/* Per-kernel timing with CUDA events recorded around every launch of the
 * named kernel family on the context's stream (off by default).  Families:
 * "propagate_f64" and "propagate_f32" (the batched fine propagator in each
 * arithmetic), "sweep" (the coarse sweep), "orth", "svd", "lift".  lrp_kernel_time returns the launches and the summed
 * event time (ms) since the last reset; it synchronises the stream. */
lrp_status lrp_set_kernel_timing(lrp_ctx* ctx, int enable);
lrp_status lrp_kernel_time(lrp_ctx* ctx, const char* family, int* launches, double* total_ms);
lrp_status lrp_reset_kernel_time(lrp_ctx* ctx);

/* ---- operators (the semi-discretisation A; inputs, copied to the device) -- */

/* Tridiagonal A, row i: lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] (lo[0] and
 * up[n-1] are ignored).  I + dt*A must be diagonally dominant: the
 * propagator eliminates without pivoting.  2 <= n <= 16384.  The call reads
 * the arrays back once to note whether the coefficients are constant (the
 * propagator has faster kernels for that case; "tri_wtoep"). */
lrp_status lrp_operator_tridiag(lrp_ctx* ctx, int n, const double* lo, const double* di,
                                const double* up, lrp_operator** out);
/* Time-dependent tridiagonal operator (Experiment 2 of Sec. 4: coefficients
 * that vary in time, so that the fine solvers F_n of the intervals differ):
 * lo, di, up are nJ x n (host or device), row J holding A(t_{J+1}) for fine
 * step J = 0..nJ-1 of the whole time grid (backward Euler is fully implicit).
 * Interval i of a coarse build or Parareal solve runs steps i M .. i M + M - 1
 * (N M <= nJ, else LRP_EINVAL); its adjoint applies the transposed steps in
 * reversed order.  lrp_propagate runs steps 0..M-1 on every vector.  n <= 1024
 * (each step is solved by parallel cyclic reduction within one CTA).  The
 * classical comparator takes time-invariant operators only; SDIRK steps take
 * the stage-sampled constructor lrp_operator_tridiag_td_sdirk. */
lrp_status lrp_operator_tridiag_td(lrp_ctx* ctx, int n, int nJ, const double* lo,
                                   const double* di, const double* up, lrp_operator** out);
/* 5-point A on an mx x my grid of interior nodes, node p = iy*mx + ix:
 * (A x)_p = C[p] x_p + W[p] x_{p-1} + E[p] x_{p+1} + S[p] x_{p-mx} + N[p] x_{p+mx};
 * coefficients that reach outside the grid are ignored (homogeneous Dirichlet). */
lrp_status lrp_operator_stencil5(lrp_ctx* ctx, int mx, int my, const double* C,
                                 const double* W, const double* E, const double* S,
                                 const double* N, lrp_operator** out);
/* Time-dependent 5-point operator (Experiment 3 of Sec. 4: a conductivity
 * that varies in time; Sec. 2: every interval its own F_n): C, W, E, S, N are
 * nJ x (mx my) (host or device), row J holding the stencil of A(t_{J+1}) for
 * fine step J = 0..nJ-1 of the whole time grid, each row as in
 * lrp_operator_stencil5.  Interval i of a coarse build or Parareal solve runs
 * steps i M .. i M + M - 1 (N M <= nJ, else LRP_EINVAL); its adjoint applies
 * the transposed steps in reversed order.  lrp_propagate runs steps 0..M-1
 * on every vector.  Every step is solved by Jacobi-preconditioned CG when
 * every step's stencil is symmetric, else by BiCGStab, with the controls of
 * lrp_operator_set_krylov.  The library keeps the step matrices of every
 * (dt, adjoint) pair it has propagated with: 13 (n + 2 mx) nJ values in FP64
 * and FP32 each.  nJ <= 65535 and mx my nJ <= 2^28.  The classical
 * comparator and the batched builds take time-invariant operators only;
 * SDIRK steps take the stage-sampled constructor
 * lrp_operator_stencil5_td_sdirk. */
lrp_status lrp_operator_stencil5_td(lrp_ctx* ctx, int mx, int my, int nJ, const double* C,
                                    const double* W, const double* E, const double* S,
                                    const double* N, lrp_operator** out);
void lrp_operator_free(lrp_operator* op);
int lrp_operator_size(const lrp_operator* op);
/* Krylov iterations spent so far by 2D propagations with this operator. */
unsigned long long lrp_operator_krylov_iterations(const lrp_operator* op);

/* Linear solver controls of 2D operators.  Each implicit-Euler step is solved
 * by Jacobi-preconditioned conjugate gradients when the stencil is symmetric
 * (W[p] = E[p-1] and S[p] = N[p-mx] for all interior couplings), else by
 * Jacobi-preconditioned BiCGStab, warm-started from the previous step, to
 * ||d - B x||_2 <= rtol ||d||_2 (B = I + dt A, d the step's right-hand side).
 * Arguments: the relative tolerances for FP64 and FP32 propagation and the
 * iteration cap per step (reaching it makes the call return LRP_ENOTCONV with
 * the outputs written).  Defaults: 1e-12, 1e-6, 20000. */
lrp_status lrp_operator_set_krylov(lrp_operator* op, double rtol_f64, double rtol_f32,
                                   int max_iter);

/* ---- the batched fine propagator (Sec. 4: backward Euler) ---------------- */

/* Apply M backward-Euler steps (I + dt A) x_{j+1} = x_j + dt f(t_{j+1}) to each
 * of nvec vectors.  x_in, x_out: nvec x n (may alias).  adjoint != 0 applies
 * the transpose solves (F'^*; requires Q = 0).  Q > 0 adds the source: g is
 * Q x n and c is nvec x M x Q (the source samples of each vector's steps).
 * prec selects FP64 or FP32 arithmetic (LRP_PREC_MIXED = FP32). */
lrp_status lrp_propagate(lrp_ctx* ctx, const lrp_operator* op, double dt, int M, int adjoint,
                         int nvec, const double* x_in, double* x_out, int Q, const double* g,
                         const double* c, lrp_precision prec);

/* The Gaussian sketch vectors of rSVD step 1 (Sec. 2.1) exactly as the build
 * draws them in its kernels: out[c*n + r] = omega_{interval, c}[r] for
 * c < ncol, r < n.  prec selects the FP64 or the FP32 deviate.  out: host or
 * device, ncol x n doubles. */
lrp_status lrp_gaussian(lrp_ctx* ctx, uint64_t seed, int interval, int ncol, int n,
                        lrp_precision prec, double* out);

/* Allocation-free variant of lrp_propagate (the paper has no counterpart).
 * It exists for callers that cannot allocate device memory: hosts that forbid
 * allocation after start-up (real-time and embedded deployments), frameworks
 * that own every device byte through their own memory pool, and latency-
 * sensitive callers that must avoid cudaFree, which synchronises the whole
 * device.  It takes no context and calls no cudaMalloc, cudaFree or
 * allocating library routine.  The operator (lo, di, up as in
 * lrp_operator_tridiag), x_in (nvec x n, or NULL for zero initial values),
 * x_out (nvec x n) and, when Q > 0, g (Q x n) and c (nvec x M x Q) must all be
 * DEVICE pointers of `device`; the caller allocates them.  Work is queued on
 * `stream` (a cudaStream_t, NULL = the default stream); the call waits on that
 * stream for the factorisation's pivot check and returns with the
 * propagation queued behind it.
 * The factorisation of I + dt*A is written to one fixed device array of
 * 300 KiB per GPU (held by every GPU that loads the library until the process
 * exits), so n is limited to LRP_NOALLOC_MAX_N; larger n returns LRP_EINVAL.
 * The first call on a device looks up that array's device address (a one-time
 * set-up per device).  Every call shares the array and overwrites the previous
 * call's factorisation: calls that overlap on the GPU (several streams or host
 * threads) race and must be serialised by the caller.  The calling thread's
 * current device is the same after the call as before it.  Returns
 * LRP_EBREAKDOWN on a zero pivot. */
#define LRP_NOALLOC_MAX_N 4096
lrp_status lrp_propagate_noalloc(int device, void* stream, int n, const double* lo,
                                 const double* di, const double* up, double dt, int M,
                                 int adjoint, int nvec, const double* x_in, double* x_out,
                                 int Q, const double* g, const double* c, lrp_precision prec);

/* ---- coarse solvers (Sec. 2.1, randomized SVD steps 1-6) ----------------- */

/* Build G_i' = U_i diag(S_i) V_i^T for i = 0..N-1 from rank + oversample
 * Gaussian sketch vectors per interval (Philox4x32-10 keyed by seed; counter
 * (row, column, interval, 0); Box-Muller).  The factors stay on the device. */
lrp_status lrp_build_coarse(lrp_ctx* ctx, const lrp_operator* op, double dt, int M, int N,
                            int rank, int oversample, uint64_t seed, lrp_precision prec,
                            lrp_coarse** out);

/* Build variants (flags of lrp_build_coarse_ex). */
enum { LRP_BUILD_INDEPENDENT_ADJOINT = 1 };
/* lrp_build_coarse with flags.  LRP_BUILD_INDEPENDENT_ADJOINT: the variant
 * mentioned in Sec. 2.2 that evaluates F_i'^* on an independent set of
 * 2 (rank + oversample) Gaussian vectors Psi (Philox stream 3) instead of on
 * the basis W, so that the forward and adjoint sketches have no dependence
 * (one sequential round instead of two) at some cost in accuracy: with
 * Y = F'Omega, Z = F'^* Psi, Q = orth(Y), the core X = (Psi^T Q)^+ Psi^T F'
 * is a least-squares estimate of Q^T F', and the factors are those of the
 * SVD of Q X.  Other arguments, outputs and errors as lrp_build_coarse;
 * LRP_EBREAKDOWN when Psi^T Q is rank deficient. */
lrp_status lrp_build_coarse_ex(lrp_ctx* ctx, const lrp_operator* op, double dt, int M, int N,
                               int rank, int oversample, uint64_t seed, lrp_precision prec,
                               int flags, lrp_coarse** out);
void lrp_coarse_free(lrp_coarse* co);
/* R_i (kept rank), the dimensions of the deflated bases of steps 2 and 4, all
 * singular values of the small matrix of step 5 (N x (rank+oversample),
 * zero-padded), delta = max_i sigma_{i,1} and eps = max_i sigma_{i,R_i+1}
 * (Eq. bounds_delta_eps).  Any output pointer may be NULL. Host outputs. */
lrp_status lrp_coarse_info(const lrp_coarse* co, int* R_i, int* rank_w, int* rank_v,
                           double* sigma, double* delta, double* eps);
/* How the bases of rSVD steps 2 and 4 (Sec. 2.1, orthonormal bases of the
 * sketches) were computed: tc_w / tc_v = number of intervals whose basis W /
 * V^ came from CholeskyQR2 with the Gram products and triangular applies on
 * the tensor cores (TF32 operands split into two terms, FP32 accumulation;
 * mixed precision, sketch width <= 64, well-conditioned sketches); the other
 * intervals used Gram-Schmidt applied twice with deflation.  Host outputs,
 * either may be NULL. */
lrp_status lrp_coarse_orth_method(const lrp_coarse* co, int* tc_w, int* tc_v);
/* Copy the factors of interval i: U and V are R_i x n (row r = psi_r / phi_r),
 * S has R_i entries (host or device outputs). */
lrp_status lrp_coarse_factors(const lrp_coarse* co, int interval, double* U, double* S,
                              double* V);

/* Checkpoint of a coarse handle (the factors depend on the operator and the
 * time grid only, so a saved handle serves later solves with any source).
 * meta_i[6] = {M, N, rank, oversample, n, precision}, meta_d[3] = {dt, delta,
 * eps}; R_i, rank_w, rank_v: N ints; sigma: N x (rank+oversample); U, V:
 * N x max(rank,1) x n; S: N x max(rank,1) (all host or device memory).  The
 * export fills what is not NULL; the import creates a handle for `op`
 * (whose size must be n) from the same arrays. */
lrp_status lrp_coarse_export(const lrp_coarse* co, int* meta_i, double* meta_d, uint64_t* seed,
                             int* R_i, int* rank_w, int* rank_v, double* sigma, double* U,
                             double* S, double* V);
lrp_status lrp_coarse_import(lrp_ctx* ctx, const lrp_operator* op, const int* meta_i,
                             const double* meta_d, uint64_t seed, const int* R_i,
                             const int* rank_w, const int* rank_v, const double* sigma,
                             const double* U, const double* S, const double* V,
                             lrp_coarse** out);

/* ---- Parareal (Eq. def_Parareal) ----------------------------------------- */

typedef struct {
  int k_done;          /* iterations performed */
  int fine_evals;      /* fine evaluations per interval in this solve (b_i + k) */
  int converged;       /* 1 if the tol criterion was met */
  double final_bound;  /* max_n a posteriori bound of the last iterate */
  double scale;        /* max_n ||u^k_n|| of the last iterate */
  double device_ms;    /* device time of the solve (events on the stream) */
} lrp_solve_stats;

/* Solve with coarse solvers `co` from u0 (n) and the source (Q, g, c as in
 * the conventions; Q = 0 for f = 0).  Runs at most K_max iterations (clamped
 * to N: u^N equals the fine solution).  If tol > 0 it stops at the first
 * k >= 1 with max_n bound_n^k <= tol * max_n ||u^k_n||, bound_n^k being the
 * a posteriori bound eps sum_{m=1}^{n-1} delta^{n-m-1} ||u^k_m - u^{k-1}_m||
 * (Eq. apost_bound).  Outputs: u_out ((N+1) x n, the last iterate),
 * bound_out (K_max x (N+1), row k-1 = bound of iterate k, may be NULL),
 * k_done and stats (may be NULL).  Returns LRP_ENOTCONV when tol > 0 was not
 * met within K_max iterations (outputs are valid). */
lrp_status lrp_parareal_solve(lrp_ctx* ctx, const lrp_coarse* co, const double* u0, int Q,
                              const double* g, const double* c, int K_max, double tol,
                              double* u_out, double* bound_out, int* k_done,
                              lrp_solve_stats* stats);

/* Fine time stepper of an operator's propagations (all of lrp_propagate,
 * the sketches of lrp_build_coarse, the fine solves of lrp_parareal_solve and
 * lrp_fine_solution): backward Euler (the default), or the two-stage SDIRK
 * methods of Sec. 4 (effect of the time discretisation), SDIRK2 (gamma = 1,
 * a21 = -1, b = (1/2, 1/2); not L-stable) and SDIRK2-L (gamma = (2-sqrt 2)/2,
 * a21 = 1 - gamma, b = (1 - gamma, gamma); L-stable), each step two solves
 * with I + gamma dt A.  SDIRK steppers: time-invariant tridiagonal operators
 * with n <= 4096 and 5-point operators (their steps on the Krylov kernel with
 * the vectors in global memory; not in batched builds); LRP_EINVAL
 * otherwise.  With a source f(t, x) = sum_q c_q(t) g_q(x) an
 * SDIRK step takes two samples of every c_q, at its stage times t + c_1 dt
 * and t + c_2 dt (c = (1, 0) for SDIRK2, (gamma, 1) for SDIRK2-L), so that
 * the c arrays of lrp_propagate, lrp_parareal_solve and lrp_fine_solution
 * hold 2 Q values per fine step, c[((J - 1) * 2 + i) * Q + q] for stage i of
 * step J; the classical comparator and the server take sources with
 * backward-Euler steps only.  Coarse handles must be built with the stepper
 * their solves use.  The allocation-free entry point always uses backward
 * Euler. */
typedef enum {
  LRP_STEP_BACKWARD_EULER = 0,
  LRP_STEP_SDIRK2 = 1,
  LRP_STEP_SDIRK2_L = 2
} lrp_stepper;
lrp_status lrp_operator_set_stepper(lrp_operator* op, int stepper);

/* SDIRK steppers on time-dependent operators (Sec. 4, effect of the time
 * discretisation, run on Experiment 3's time-dependent operator): every
 * stage of a step solves with the operator at its own stage time, so the
 * coefficient arrays hold two rows per fine step, 2 nJ rows in all: row
 * 2J + s = A(t_J + c_s dt) for stage s = 0, 1 of step J (t_J = J dt the
 * start of step J; c = (1, 0) for SDIRK2, (gamma, 1) for SDIRK2-L), each row
 * laid out as in lrp_operator_tridiag_td / lrp_operator_stencil5_td.
 * stepper: LRP_STEP_SDIRK2 or LRP_STEP_SDIRK2_L (LRP_EINVAL otherwise); the
 * operator keeps it (lrp_operator_set_stepper accepts only the same one).
 * Sources take two samples per step at the same stage times, as for
 * time-invariant operators.  The adjoint propagation applies the transpose
 * of every step map in reversed step order (stage-2 matrix first).  Limits
 * as for the backward-Euler constructors, with 2 nJ rows in place of nJ. */
lrp_status lrp_operator_tridiag_td_sdirk(lrp_ctx* ctx, int n, int nJ, int stepper,
                                         const double* lo, const double* di, const double* up,
                                         lrp_operator** out);
lrp_status lrp_operator_stencil5_td_sdirk(lrp_ctx* ctx, int mx, int my, int nJ, int stepper,
                                          const double* C, const double* W, const double* E,
                                          const double* S, const double* N, lrp_operator** out);

/* Classical Parareal for comparison (the method of the dashed curves in the
 * paper's numerical experiments, Sec. 4): Eq. def_Parareal with the coarse
 * solver G_i = one backward-Euler step of size M*dt over interval i, the
 * source sampled at the interval's end t_{i+1}; the same fine solver as
 * lrp_parareal_solve (M steps of size dt).  No coarse factors are built.
 * Stops after K_max iterations (clamped to N) or, when tol > 0, at the first
 * k >= 1 with max_n ||u^k_n - u^{k-1}_n|| <= tol * max_n ||u^k_n|| (the
 * classical coarse solver has no a posteriori bound).  u0 (n), g (Q x n),
 * c ((N*M) x Q) host or device; u_out ((N+1) x n) the last iterate;
 * incr_out (K_max, may be NULL): the relative increment of every iteration.
 * Workspace is allocated per call on the context.  Returns LRP_ENOTCONV when
 * tol > 0 was not met (outputs valid). */
lrp_status lrp_parareal_solve_classical(lrp_ctx* ctx, const lrp_operator* op, double dt, int M,
                                        int N, const double* u0, int Q, const double* g,
                                        const double* c, int K_max, double tol, double* u_out,
                                        double* incr_out, int* k_done, lrp_solve_stats* stats);

/* The sequential fine solution u_{i+1} = F_i u_i (Sec. 2), (N+1) x n, with the
 * same propagator: the fixed point Parareal converges to. */
lrp_status lrp_fine_solution(lrp_ctx* ctx, const lrp_operator* op, double dt, int M, int N,
                             const double* u0, int Q, const double* g, const double* c,
                             double* u_out);

/* ---- many 2D problems of uneven size at once ------------------------------ */

/* Coarse solvers for `count` 5-point operators (grids may differ) sharing the
 * time grid, rank, oversampling, seed and precision.  Each propagation stage
 * of the randomized SVD runs as one persistent launch over a device work
 * queue of (problem, system) items, largest grids first, and the whole build
 * is captured into one CUDA graph and launched once.  out[p] receives the
 * handle of problem p (free each with lrp_coarse_free).  The queue's cluster
 * size is the "queue_cluster" parameter (default 4). */
lrp_status lrp_build_coarse_batch(lrp_ctx* ctx, int count, lrp_operator* const* ops, double dt,
                                  int M, int N, int rank, int oversample, uint64_t seed,
                                  lrp_precision prec, lrp_coarse** out);
/* Parareal (f = 0) for `count` 2D problems with handles from any build of
 * equal N, M, rank and precision: per iteration the fine solves of all
 * unconverged intervals of all problems run as one queue launch and the coarse
 * sweeps are batched per grid size.  u0[p]: n_p values; u_out[p]: (N+1) x n_p
 * (host or device); k_done[p]: iterations of problem p (tol as in
 * lrp_parareal_solve, per problem). */
lrp_status lrp_parareal_solve_batch(lrp_ctx* ctx, int count, lrp_coarse* const* cos,
                                    const double* const* u0, int K_max, double tol,
                                    double* const* u_out, int* k_done);

/* ---- serving: continuous batching over resident coarse solvers ----------- */

/* The coarse solvers depend on the operator and the time grid only (Sec. 2.1,
 * Remark rem:affine_g_n), so built handles serve a stream of solves with new
 * u0 and new sources.  A server works on the device of `ctx`; the requests
 * of each coarse handle form a group with its own worker thread and its own
 * stream, whose priority is higher the cheaper the handle's fine solves are
 * (n N M row-steps: the highest up to 1e5, one level lower per factor of
 * ten), so that short requests do not wait behind long ones of another
 * handle.  Requests are admitted into slots (device memory for the iterate,
 * F outputs, b_i and the source of one request; at most max_slots per
 * coarse handle and as many as half the free HBM -- and the budget, if
 * nonzero -- allow); waiting requests stay queued.  Each tick of a group runs
 * one Parareal iteration for every admitted request: the fine solves of all
 * their unconverged intervals in one launch and all their coarse sweeps in
 * one batched launch; requests arriving meanwhile join at the next tick.
 * max_terms bounds Q (the number of source terms) of a request. */
typedef struct lrp_server lrp_server;
typedef struct {
  int k_done;           /* Parareal iterations performed */
  int status;           /* LRP_OK, LRP_ENOTCONV (tol not met by K_max), or an error */
  double final_bound;   /* max_n a posteriori bound of the returned iterate */
  double scale;         /* max_n ||u^k_n|| of the returned iterate */
  double queue_ms;      /* submit -> admitted into a slot */
  double latency_ms;    /* submit -> result ready on the host */
} lrp_request_info;
typedef struct {
  unsigned long long completed, ticks;
  size_t queued;
  int active, slots, error;
  double busy_ms;       /* worker time spent in ticks */
} lrp_server_stats;

lrp_status lrp_server_create(lrp_ctx* ctx, int max_slots, int max_terms,
                             size_t hbm_budget_bytes, lrp_server** out);
/* Stop the worker (requests still queued or running are abandoned) and free
 * the server.  Coarse handles in use must outlive the server. */
void lrp_server_destroy(lrp_server* srv);
/* Queue a solve with coarse solvers `co` (same arguments as
 * lrp_parareal_solve; host pointers; copied before the call returns).  The
 * first request of a handle creates its group (LRP_ENOMEM when not one slot
 * fits).  Returns LRP_EBUSY when the queue is full, or when the handle has a
 * latency target and the request's estimated latency exceeds it. */
lrp_status lrp_server_submit(lrp_server* srv, const lrp_coarse* co, const double* u0, int Q,
                             const double* g, const double* c, int K_max, double tol,
                             uint64_t* ticket);
/* Non-blocking: LRP_PENDING while the request runs; otherwise its status,
 * with u_out ((N+1) x n, host, may be NULL) and info filled.  A finished
 * request can be fetched once. */
lrp_status lrp_server_poll(lrp_server* srv, uint64_t ticket, double* u_out,
                           lrp_request_info* info);
/* Blocking variant; timeout_s <= 0 waits without limit, else LRP_ETIMEOUT. */
lrp_status lrp_server_wait(lrp_server* srv, uint64_t ticket, double timeout_s, double* u_out,
                           lrp_request_info* info);
lrp_status lrp_server_stats_get(lrp_server* srv, lrp_server_stats* stats);
/* Admission control: requests on `co` whose estimated latency (submit ->
 * result) exceeds target_ms are turned away with LRP_EBUSY (0: no target,
 * the default).  Estimate, with A the requests active or queued on `co`
 * plus the new one: (ticks a request spends in a slot) x (tick time with
 * min(A, slots) requests active) x ceil(A / slots), the first an average
 * over finished requests, the second a line in the number of active
 * requests fitted to the group's ticks with exponential forgetting; while
 * the group has finished no request the estimate is 0 and requests are
 * admitted. */
lrp_status lrp_server_set_latency_target(lrp_server* srv, const lrp_coarse* co, double target_ms);
/* The current latency estimate (ms) of a request on `co` (0 without history). */
lrp_status lrp_server_estimate(lrp_server* srv, const lrp_coarse* co, double* latency_ms);

#ifdef __cplusplus
}
#endif
#endif /* LRP_H */
