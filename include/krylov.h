/*
 * libkrylov: DCGS2 Arnoldi-QR on one GB300 GPU (C ABI).
 *
 * Method: "Low-Synch Gram-Schmidt with Delayed Reorthogonalization for Krylov Solvers"
 * (Bielich, Langou, Thomas, Swirydowicz, Yamazaki, Boman).  The hot path is the DCGS2
 * Arnoldi step of Algorithm 4 (Section 4): one sparse matvec on the pending unnormalised
 * vector w, ONE fused reduction [Q, w]^T [w, A w], the delayed normalisation (Pythagorean
 * trick), Stephen's trick (eq. 30), the projection update and the lagged Hessenberg
 * correction.  Baselines: CGS2-Arnoldi (Algorithm 3) and MGS-Arnoldi (Section 2).
 * Drivers: restarted GMRES (Section 1 problem (1)), Krylov-Schur (problem (2)), FP32/BF16
 * inner solves in FP64 iterative refinement, and flexible GMRES with a learned
 * convolutional right preconditioner.
 *
 * Conventions for every entry point
 *  - All array arguments are DEVICE pointers owned by the caller unless stated otherwise;
 *    the library never frees them.  The library allocates only its context workspace.
 *  - Work is enqueued on the context's stream and is asynchronous, except where a function
 *    returns a host scalar (it then synchronises that stream once at the end).
 *  - Errors are returned as kc_status; kc_last_error() gives the message of the context's
 *    last failure.  No C++ exception crosses the ABI.
 *  - Index convention (0-based): H[i + j*ldh] is the coefficient of q_i in A q_j, so that
 *    A Q_n = Q_{n+1} H_n ((n+1) x n, eq. "arnoldi").  The paper's 1-based j maps to k = j-1.
 */
#ifndef KRYLOV_H
#define KRYLOV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KC_OK = 0,
  KC_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or dtype combination */
  KC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  KC_ERR_OOM = 3,           /* context workspace allocation failed */
  KC_ERR_BREAKDOWN = 4,     /* alpha_k <= 1e-13 * ||H(:,k-1)||: invariant subspace found */
  KC_ERR_NOT_CONVERGED = 5, /* iteration limit reached before the tolerance */
  KC_ERR_NONFINITE = 6,     /* NaN/Inf in a reduction result */
  KC_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  KC_ERR_PYTHAGORAS_NEG = 8 /* beta - C^T C <= 0 in the delayed normalisation */
} kc_status;

typedef enum { KC_F64 = 0, KC_F32 = 1, KC_BF16 = 2 } kc_dtype;

typedef struct kc_ctx kc_ctx;

/* The operator A (m x m), in one of two forms chosen by grid[0]:
 *
 *  - CSR matrix (grid[0] == 0; a zero-initialised struct is a CSR): int32 indices
 *    (nnz < 2^31), caller-owned device arrays.  row_ptr[m+1] non-decreasing with
 *    row_ptr[0] = 0, col_idx[nnz] in [0, m), val[nnz] of type val_dtype (KC_F64 or KC_F32).
 *
 *  - Matrix-free 7-point stencil (grid[0] > 0; row_ptr, col_idx, val and nnz are ignored):
 *    on an nx x ny x nz grid, grid = {nx, ny, nz}, m = nx ny nz, row i = ix + nx (iy + ny iz)
 *    (x fastest), with zero (homogeneous Dirichlet) values outside the grid:
 *      (A x)_i = c0 x_i + c1 x_{i-1} + c2 x_{i+1} + c3 x_{i-nx} + c4 x_{i+nx}
 *              + c5 x_{i-nx ny} + c6 x_{i+nx ny},   stencil = {c0, ..., c6},
 *    each neighbour term present only when that neighbour lies in the grid.  This is the
 *    constant-coefficient form of the h^2-scaled upwind convection-diffusion operators
 *    (2D with nz = 1) and of the Manteuffel matrix of Section 6.1; with it the basis
 *    generation v = A w of Algorithm 4 reads w once and writes v once instead of streaming
 *    the matrix.  val_dtype KC_F64: FP64 vectors, seven FP64 FMAs per row in both FP64
 *    modes (an error in v, unlike one in S or Q C, is not removed by the next
 *    reorthogonalisation: it enters A Q = Q H); KC_F32: FP32 vectors, coefficients rounded
 *    to FP32.  Accepted wherever a kc_csr is, except by the entry points that read the
 *    matrix entries themselves (fgmres_solve, kc_cnn_train_step_residual,
 *    dcgs2_arnoldi_step_noalloc), which return KC_ERR_INVALID_ARG for a stencil. */
typedef struct {
  int64_t m;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const void* val;
  int32_t val_dtype;
  int32_t grid[3];
  double stencil[7];
} kc_csr;

/* Arnoldi state (caller-owned device buffers).
 *  Q     basis, column-major: column j starts at element j*ldq; ldq >= m and even,
 *        Q 16-byte aligned.  Element type q_dtype (KC_F64 with FP64 vectors; KC_F32 or
 *        KC_BF16 with FP32 vectors).  ncap columns (the basis holds at most ncap columns,
 *        i.e. at most ncap-1 DCGS2 steps before the finish); 2 <= ncap <= 128.
 *  w, v  m-vectors (FP64 when q_dtype is KC_F64, else FP32), 16-byte aligned: w is the
 *        pending vector, v the matvec workspace.
 *  H     FP64, column-major, ldh >= ncap, at least ldh*(ncap-1) entries.
 *  K     FP64 workspace, ncap*(ncap-1) entries, column-major with ld ncap: column j holds
 *        the partial Hessenberg column that the next step completes (Algorithm 4).
 *  k     number of final basis columns; written by the library (read-only for callers).
 *  nsteps_since_init  written by the library. */
typedef struct {
  void* Q;
  int64_t ldq;
  int32_t ncap;
  int32_t q_dtype;
  void* w;
  void* v;
  double* H;
  int32_t ldh;
  double* K;
  int32_t k;
  int32_t finished;
} kc_arnoldi;

/* ---- context ------------------------------------------------------------------------ */

/* Create a context on `device` that enqueues on `cuda_stream` (a cudaStream_t, or NULL for
 * the legacy default stream).  Allocates the reduction workspace (a few hundred KB). */
kc_status kc_create(kc_ctx** ctx, int device, void* cuda_stream);
kc_status kc_destroy(kc_ctx* ctx);
kc_status kc_set_stream(kc_ctx* ctx, void* cuda_stream);
/* Message of the last failed call on this context (static storage inside ctx). */
const char* kc_last_error(const kc_ctx* ctx);
/* FP64 arithmetic mode of the DCGS2 step (default 1).
 *  0: every product of the two basis passes in FP64 FMAs.
 *  1: FP64 with offload: C = Q^T w and the projection v/alpha - Q T stay in FP64; the
 *     first-projection coefficients S = Q^T v and the product Q C use float-float
 *     arithmetic (about 2^-44 relative) on the FP32/INT pipes.  An error d in S is
 *     removed by the next step's delayed reorthogonalisation (it returns as -d/alpha in
 *     the next C and cancels in H = K + C, Section 4), and Q C is scaled by the tiny C,
 *     so Q and H keep FP64 accuracy while half of the FP64 FMAs leave the FP64 pipe.
 *  2: as 1, but the fused reduction (C, S, beta, s: the single reduction of Algorithm 4) runs on the
 *     tensor cores as exact integer dot products of fixed-point digit expansions (the
 *     Ozaki scheme: basis entries as round(q 2^56), w and v scaled per 512-row chunk,
 *     FP16 digits, FP32 accumulators that stay exact, one FP64 rounding per chunk), with
 *     no FP64 arithmetic per basis entry; steps with more than 59 basis columns, or a
 *     basis, w or v not 16-byte aligned (odd leading dimension), use mode 1's reduction.
 *     A basis entry of magnitude >= 2 or a non-finite operand sets KC_ERR_NONFINITE.
 * Other values return KC_ERR_INVALID_ARG. */
kc_status kc_set_fp64_mode(kc_ctx* ctx, int mode);
int kc_get_fp64_mode(const kc_ctx* ctx);
/* Kernel variants of the FP64 basis passes (bit flags; same arithmetic either way):
 *  1: the DCGS2 update stages basis tiles in shared memory with bulk asynchronous copies
 *     (one producer thread and an mbarrier ring per SM);
 *  2: the fused DCGS2 reduction stages 2D tiles of the basis with tensor-memory copies
 *     (cp.async.bulk.tensor, one producer thread, sixteen consumer warps per SM);
 *  4: FP64 mode 1 / 2 without the bounded FP32 products and the float-float first
 *     projection: Q C of the update and of the CGS2 finish's projections then always
 *     take float-float (update) or FP64 (finish), instead of FP32 products on the
 *     launches whose error bound, (k + 3) 2^-24 ||C||_1 <= 2^-53 ||w - Q C||, holds; and
 *     the finish's first projection C1 = Q^T w is summed in FP64 instead of float-float
 *     (its error is removed by the second projection either way);
 *  8: fused first steps: in FP64 mode 1 the steps with k <= 4 basis columns form
 *     v = A w and the fused reduction in one pass (one thread per row, one launch fewer,
 *     w and v read once; the pass stays bound by its FP64 operations, so it is not the
 *     default);
 * 0 streams both passes through registers, with the bounded FP32 products. */
kc_status kc_set_staged(kc_ctx* ctx, int flags);
/* Kernel of the network's 32 -> 32 convolutions: 0 mma.sync (m16n8k16, registers);
 * 1 tcgen05 (default: tensor-copy fed, accumulator in tensor memory, operands in shared
 * memory).  Same arithmetic: BF16 products, FP32 accumulation (summation order differs). */
kc_status kc_set_conv_kernel(kc_ctx* ctx, int kind);
/* Execution path of an FP64 gmres_solve (precision 0): 0 (default) chooses by size, 1 the
 * multi-kernel path (three launches per Arnoldi step, the host reads the Givens state once
 * per cycle), 2 and 3 the whole restarted solve in ONE launch whose CTAs own the rows in
 * blocks and meet at barriers instead of kernel boundaries: 2 on one thread-block cluster
 * (16 CTAs, or 8; hardware barriers, partial sums read from the other CTAs' shared memory),
 * 3 on one CTA per SM of the whole GPU (cooperative launch; partial sums through global
 * memory; a software barrier whose wait is bounded: KC_ERR_TIMEOUT if a CTA waits longer
 * than about a second).  0 takes 3 up to m = 393,216 rows (where it was measured faster
 * than 1), else 1.  All give the same iterates up to rounding. */
kc_status kc_set_gmres_path(kc_ctx* ctx, int path);
/* Test hook for the bounded grid barrier of gmres_path 3: when on, the next such solve
 * expects one arrival more than it has CTAs, so its first barrier cannot complete; every
 * CTA gives up after about a second and the solve returns KC_ERR_TIMEOUT (no fault, the
 * context stays usable).  The hook clears itself after that one solve. */
kc_status kc_set_barrier_test(kc_ctx* ctx, int on);
/* Number of SMs and the persistent grid size used for reductions. */
kc_status kc_device_info(const kc_ctx* ctx, int* num_sms, int* reduce_grid);
/* Number of kernels this context has launched since creation (host-side counter). */
int64_t kc_launch_count(const kc_ctx* ctx);
/* Per-kernel timing.  While enabled, CUDA events are recorded on the context's stream
 * around every kernel the library launches.  kc_timing_read synchronises the stream and
 * returns, per kernel kind, the summed elapsed milliseconds and launch counts, then
 * clears the records.  Kinds (index): 0 SpMV, 1 fused reduction, 2 DCGS2 update,
 * 3 projection update (x -= Q c), 4 norm / dot, 5 scaling, 6 MGS axpy, 7 small dense
 * kernels, 8 other, 9 the CGS2 finish's reductions, 10 the fused SpMV and reduction of
 * the first DCGS2 steps.  nkinds must be >= 11. */
kc_status kc_timing_enable(kc_ctx* ctx, int on);
kc_status kc_timing_read(kc_ctx* ctx, double* ms, int64_t* count, int nkinds);
/* Read (and synchronise on) the device status word written by the last reductions:
 * KC_OK, KC_ERR_BREAKDOWN, KC_ERR_NONFINITE or KC_ERR_PYTHAGORAS_NEG.  Clears it. */
kc_status kc_read_status(kc_ctx* ctx, int* device_status);
/* Copy the last step's scalars to host: alpha, beta (w^T w), s (w^T A w). */
kc_status kc_last_scalars(kc_ctx* ctx, double* alpha, double* beta, double* s);

/* ---- building blocks ---------------------------------------------------------------- */

/* y = A x (K4': CSR SpMV, or the matrix-free stencil).  x, y: m-vectors of the matrix
 * value type (FP64 or FP32); x and y must not overlap. */
kc_status kc_spmv(kc_ctx* ctx, const kc_csr* A, const void* x, void* y);

/* ---- DCGS2-Arnoldi (Algorithm 4) ----------------------------------------------------- */

/* Start the expansion: w = r0 (unnormalised; the factorised matrix is B = [r0, A Q],
 * Section 1), k = 0.  r0 has the vector type of the state. */
kc_status dcgs2_arnoldi_init(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st, const void* r0);

/* One DCGS2 step (Algorithm 4): v = A w; the single fused reduction
 * C = Q_k^T w, S = Q_k^T v, beta = w^T w, s = w^T v; in the same launch
 * alpha = sqrt(beta - C^T C), H(0:k, k-1) = K(0:k, k-1) + C and H(k, k-1) = alpha,
 * T = S/alpha, T_k = (s - C^T S)/alpha^2 (eq. 30), K(0:k+1, k) =
 * T - H(0:k+1, 0:k) C / alpha (after H(k, k-1), which it reads); then the fused update q_k = (w - Q_k C)/alpha -> Q(:,k) and
 * w <- v/alpha - Q_k T(0:k) - q_k T_k.  Requires k+1 < ncap.
 * Three kernel launches; no host synchronisation.  Numerical failures are reported
 * through kc_read_status (the step still completes with a guarded alpha). */
kc_status dcgs2_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st);

/* Finish (end of Section 3: the last column by CGS2, two more reductions): with the
 * pending w, C1 = Q^T w, u = w - Q C1, C2 = Q^T u, u -= Q C2, alpha = ||u||;
 * H(0:k, k-1) = K(0:k, k-1) + C1 + C2, H(k, k-1) = alpha, Q(:,k) = u/alpha.
 * Afterwards Q has k+1 columns and H is (k+1) x k. */
kc_status dcgs2_arnoldi_finish(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st);

/* Gram matrix of a basis, G = Q^T Q, for the loss of orthogonality ||I - Q^T Q||_F
 * (Section 6.1).  Q: device, column-major with leading dimension ldq >= m, ncols columns
 * (1 <= ncols <= 128) of type q_dtype (KC_F64, KC_F32 or KC_BF16); G: device FP64,
 * ncols x ncols column-major, overwritten, exactly symmetric.  Products and sums in FP64;
 * the per-block sums are combined with atomics, so the last bits of G may vary from call
 * to call.
 * Asynchronous on the context stream. */
kc_status kc_basis_gram(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int64_t m,
                        int ncols, double* G);

/* ---- row-partitioned DCGS2 (Section 5; Tables 1-2: rows split across processes) ---------
 * The distributed layout of the paper: rank p owns a contiguous block of m_p rows of A, Q,
 * w and v, and every step makes ONE global sum of its 2k + 2 partial dot products (the
 * MPI_Allreduce of Section 5); the small scalar step is replicated.  These calls are the
 * per-rank work of one GPU; the caller sums the partials over the ranks (NCCL or any other
 * collective: the library makes none) and supplies the halo of w for the matvec.
 *   A_local: the rank's m_p rows in CSR form (FP64 values), its column indices pointing
 *            into w_ext;
 *   st:      the rank's state: Q, w, v with m_p rows (ldq >= m_p), H and K replicated
 *            (identical on every rank), FP64 basis; start with dcgs2_arnoldi_init on the
 *            rank's rows of r0;
 *   partial, totals: device FP64 arrays.  All calls are asynchronous on the context stream.
 *
 * dcgs2_part_reduce: v = A_local w_ext (this rank's rows of A w; w_ext holds w's rows that
 * A_local's columns reach, i.e. the rank's own rows and the halo), then this rank's partial
 * sums of [Q_k, w]^T [w, v] into partial[0 : 2k+2] = [C_0, S_0, ..., C_{k-1}, S_{k-1},
 * beta, s] (the single reduction of Algorithm 4, over the local rows).
 * dcgs2_part_update: totals = the element-wise sum of every rank's partial; the scalar step
 * of Algorithm 4 (Pythagoras, eq. 30, the H and K columns) from it and the row-local update
 * of q_k and w; k += 1.  Numerical failures go to kc_read_status as for dcgs2_arnoldi_step.
 * dcgs2_part_finish: the CGS2 finish (end of Section 3) as four phases with three global
 * sums between them: phase 0 writes partial[0 : k+1] = [Q^T w, w^T w]; phase 1 takes their
 * sums, forms u = w - Q C1 and writes partial[0 : k+1] = [Q^T u, u^T u]; phase 2 takes those
 * sums, forms u -= Q C2 and writes partial[0] = u^T u; phase 3 takes that sum and writes
 * H(:, k-1), alpha and q_k = u / alpha (totals unused in phase 0, partial in phase 3).
 * FP64 modes 0 and 1 as for dcgs2_arnoldi_step (mode 2 takes mode 1's reduction here). */
kc_status dcgs2_part_reduce(kc_ctx* ctx, const kc_csr* A_local, kc_arnoldi* st,
                            const double* w_ext, double* partial);
kc_status dcgs2_part_update(kc_ctx* ctx, const kc_csr* A_local, kc_arnoldi* st,
                            const double* totals);
kc_status dcgs2_part_finish(kc_ctx* ctx, const kc_csr* A_local, kc_arnoldi* st, int phase,
                            const double* totals, double* partial);

/* One FP64 DCGS2 step, as dcgs2_arnoldi_step in its all-FP64 mode, that allocates
 * nothing and needs no context.  (The paper has no counterpart: this is a deployment
 * variant.)  It is meant for callers that cannot call cudaMalloc: code running inside
 * a stream-ordered allocator or graph callback, plugins whose host application owns the
 * device memory budget, or code that must not create a context.  The caller still passes
 * the matrix and every state buffer (Q, w, v, H, K), exactly as for
 * dcgs2_arnoldi_step; the reduction's scratch (per-CTA partial sums, the last-CTA ticket,
 * the step scalars) lives in a file-scope device array of about 325 KB that every GPU
 * loading the library keeps until the process exits.  Limits: FP64 basis and matrix
 * only, ncap <= 128 (the same limit as the other entry points), at most 152 reduction
 * CTAs; other sizes return KC_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current: make that
 * first call before any stream capture.  All calls share the one array and it keeps the
 * last call's contents; the call clears what must start at zero (ticket, flags), and two
 * calls that overlap on the GPU (different streams, concurrent graphs) race on it.
 * The looked-up address is kept for the rest of the process: a cudaDeviceReset, which
 * unloads the library from the device, leaves this entry point unusable on that device
 * until the process exits.
 * Enqueued on `cuda_stream` (a cudaStream_t, NULL for the legacy stream); returns
 * KC_ERR_CUDA if the set-up or a launch fails.  Numerical failures of the step (a
 * non-positive Pythagorean norm, a breakdown, a non-finite value) are kept in the shared
 * array's status word until the next call clears it: dcgs2_noalloc_read_status reads it. */
kc_status dcgs2_arnoldi_step_noalloc(const kc_csr* A, kc_arnoldi* st, void* cuda_stream);

/* The status word of the last dcgs2_arnoldi_step_noalloc call on the current device
 * (KC_OK or the first numerical failure of that step), copied to the host int *status
 * after waiting for `cuda_stream`.  Allocates nothing; the paper has no counterpart.
 * Returns KC_ERR_INVALID_ARG for a NULL status and KC_ERR_CUDA if the copy fails. */
kc_status dcgs2_noalloc_read_status(int* status, void* cuda_stream);

/* ---- baselines ---------------------------------------------------------------------- */

/* DCGS2 QR of a tall-skinny matrix (Algorithm 2, Section 3): A (m x n, column-major, leading
 * dimension lda) = Q R with Q (m x n, ldq) orthonormal and R (n x n, ldr, upper triangular;
 * the strictly lower part is set to zero).  One fused reduction per column, the delayed
 * reorthogonalisation of the previous column inside it, the last column by CGS2 with an
 * explicit norm; the same kernels and FP64 mode as the Arnoldi step.  Device pointers, FP64;
 * A and Q 16-byte aligned with even leading dimensions; 1 <= n <= 127.  A is not modified.
 * Asynchronous on the context stream; a rank-deficient A is reported by kc_read_status as
 * KC_ERR_BREAKDOWN (alpha_j <= 1e-13 ||R(:, j)||) or KC_ERR_PYTHAGORAS_NEG. */
kc_status dcgs2_qr(kc_ctx* ctx, const double* A, int64_t lda, int64_t m, int n, double* Q,
                   int64_t ldq, double* R, int ldr);

/* ICWY-MGS (Section 5): MGS with its rank-1 projections batched into the inverse compact
 * WY projector I - Q T Q^T, T = (I + L)^{-1} with L the strictly lower triangular part of
 * Q^T Q, one reduction per iteration (the fused reduction [Q_k, w]^T [w, A w] of the DCGS2
 * step: its C gives row k of L, beta the norm of the pending w, S and s the projections),
 * a triangular solve for the coefficients, and the update with C = 0.  Its loss of
 * orthogonality is MGS's, O(eps) kappa (Table 3).  FP64 basis, every product in FP64.
 *   icwy_arnoldi_step: start with dcgs2_arnoldi_init (w = r0); step k normalises w into q_k
 *     (H(k, k-1) = ||w||), stores row k of L in the K workspace and appends H(0:k+1, k) with
 *     the next pending w;  icwy_arnoldi_finish normalises the last pending w into q_k.
 *   icwy_qr: Q R of a tall-skinny matrix, the arguments and layout of dcgs2_qr. */
kc_status icwy_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st);
kc_status icwy_arnoldi_finish(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st);
kc_status icwy_qr(kc_ctx* ctx, const double* A, int64_t lda, int64_t m, int n, double* Q,
                  int64_t ldq, double* R, int ldr);

/* CGS2-Arnoldi (Algorithm 3) and MGS-Arnoldi (Section 2, "MGS Level 1"): init sets
 * q_0 = r0/||r0|| (k = 1); each step appends column k-1 of H and q_k.  CGS2 does three
 * reductions per step (two projections + norm), MGS one per inner product. */
kc_status cgs2_arnoldi_init(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st, const void* r0);
kc_status cgs2_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st);
kc_status mgs_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st);

/* ---- GMRES / iterative refinement / flexible GMRES ---------------------------------- */

typedef struct {
  int32_t restart;        /* basis size n of GMRES(n) */
  int32_t maxit;          /* matvec limit */
  int32_t precision;      /* 0 = FP64; 1 = FP32 inner solve in FP64 IR; 2 = BF16 basis IR */
  int32_t max_outer;      /* IR: outer refinement limit */
  double rtol;            /* relative residual target ||b - A x|| / ||b|| */
  double inner_rtol;      /* IR: inner solve tolerance (relative to its right-hand side) */
  int32_t inner_max_cycles; /* IR: cycles per inner solve */
  int32_t precond;        /* a kc_precond_kind.  gmres_solve: KC_PREC_AUTO = none,
                             KC_PREC_JACOBI = right Jacobi preconditioning (precision 0;
                             solved by fgmres_solve, A a CSR matrix); fgmres_solve: below */
  int32_t diag_loo;       /* gmres_solve diagnostics: 1 = after every (inner) cycle form the
                             Gram matrix of the n (or, at an early stop, ncols) columns that
                             formed its correction (kc_basis_gram) and report the largest
                             ||I - Q^T Q||_F in kc_gmres_info.max_loo (one extra pass of
                             O(m n^2) FP64 work per cycle, and the multi-kernel path) */
} kc_gmres_opts;

/* Right preconditioner of fgmres_solve. */
typedef enum {
  KC_PREC_AUTO = 0,       /* the network when weights are given, else the identity */
  KC_PREC_JACOBI = 1      /* the Jacobi step D^{-1} w alone (network weights ignored) */
} kc_precond_kind;

typedef struct {
  int32_t iters;          /* matvecs with A (inner iterations for IR) */
  int32_t restarts;       /* GMRES cycles (all inner cycles for IR) */
  int32_t outer;          /* IR refinement steps */
  int32_t status;         /* kc_status of the solve */
  double rel_resid_est;   /* last Givens estimate |g_k| / ||b|| */
  double rel_resid_true;  /* FP64 ||b - A x|| / ||b|| recomputed on the device */
  double max_loo;         /* largest ||I - Q^T Q||_F over the cycles' bases when
                             kc_gmres_opts.diag_loo is set, else -1 (Section 6.1 metric) */
} kc_gmres_info;

/* Restarted DCGS2-GMRES(n) (FP64), or FP32/BF16-basis DCGS2-GMRES inside FP64 iterative
 * refinement (precision 1/2; then A32 must be the FP32 copy of A, else it is ignored).
 * b, x: FP64 m-vectors; x holds x0 on entry and the solution on return.  Synchronises. */
kc_status gmres_solve(kc_ctx* ctx, const kc_csr* A, const kc_csr* A32, const double* b,
                      double* x, const kc_gmres_opts* opts, kc_gmres_info* info);

/* ---- Krylov-Schur ------------------------------------------------------------------- */

typedef struct {
  int32_t nev;            /* wanted eigenvalues (largest real part) */
  int32_t ncv;            /* basis size */
  int32_t nkeep;          /* columns kept at a restart (+1 to keep a conjugate pair) */
  int32_t maxrestarts;
  double tol;             /* ||(A - lambda I) z|| <= tol * |lambda| (eq. "ArnoldiRes") */
} kc_ks_opts;

/* Krylov-Schur on DCGS2-Arnoldi.  v0: FP64 start vector (device).  eig_re, eig_im,
 * resid: HOST arrays of length nev (largest real part first).  nconv, restarts,
 * matvecs: host outputs (may be NULL).  The small dense Schur step runs on the GPU in
 * FP64.  Synchronises. */
kc_status krylov_schur_eigs(kc_ctx* ctx, const kc_csr* A, const double* v0,
                            const kc_ks_opts* opts, double* eig_re, double* eig_im,
                            double* resid, int* nconv, int* restarts, int* matvecs);

/* ---- learned preconditioner and flexible GMRES (additions; not in the paper) ----------- */

/* The network: 6 layers of 3x3 convolutions, channels 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1,
 * zero padding, no bias, ReLU after layers 0..4; BF16 weights and activations, FP32
 * accumulation (tensor cores for the 32 -> 32 layers).  w32: FP32 master weights, layer by
 * layer, each [Cout][3][3][Cin]; kc_cnn_param_count() values (37,440). */
int64_t kc_cnn_param_count(void);

/* y = net(x) for B single-channel H x W images (FP32, row-major, device).  Uses context
 * workspace (grown on demand). */
kc_status kc_cnn_forward(kc_ctx* ctx, const float* w32, const float* x, float* y, int B,
                         int H, int W);

/* One training step on a batch: forward (y = net(x), written to y), loss
 * L = (1/B) sum_b ||y_b - e_b||^2 / ||e_b||^2 (host *loss, may be NULL; reading it
 * synchronises), backward (dL/dw into grad if non-NULL, FP32), and, when t > 0, the Adam
 * update of w32 with step number t, learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8
 * (adam_m, adam_v: FP32 moment buffers, kc_cnn_param_count() each, zero-initialised by
 * the caller). */
kc_status kc_cnn_train_step(kc_ctx* ctx, float* w32, float* adam_m, float* adam_v, int64_t t,
                            float lr, const float* x, const float* e, int B, int H, int W,
                            float* y, float* grad, double* loss);

/* The same training step with the residual loss of the preconditioner that fgmres_solve
 * applies: for network inputs x_b (the Jacobi-scaled residuals D^{-1} r_b divided by a
 * common factor s_b) and residuals r_b (divided by the same s_b),
 *   L = (1/B) sum_b ||A (x_b + net(x_b)) - r_b||^2 / ||r_b||^2,
 * i.e. ||A (M(r_b) - e_b)||^2 / ||r_b||^2 for the exact correction e_b = A^{-1} r_b.
 * A: FP64 CSR operator with m = H W (device), shared by the batch.  dL/dy is formed as
 * (2/B) A^T res_b / ||r_b||^2 by scattering along the rows of A (FP32 atomics: the
 * summation order, and so the last bits of grad, vary from run to run). */
kc_status kc_cnn_train_step_residual(kc_ctx* ctx, float* w32, float* adam_m, float* adam_v,
                                     int64_t t, float lr, const kc_csr* A, const float* x,
                                     const float* r, int B, int H, int W, float* y, float* grad,
                                     double* loss);

/* One training sample of the residual loss from the current iterate of a solve (the
 * (residual, correction) pairs, the correction left implicit):
 *   r = b - A x,  u = D^{-1} r,  s = rms(u) = sqrt(u^T u / m),
 *   xin = u / s,  res = r / s   (FP32, m each, device),
 * D = diag(A) as in fgmres_solve.  A: FP64 CSR (device); b, x: FP64 device vectors of
 * length m, 16-byte aligned; xin, res: caller-owned FP32 outputs.  *rnorm (host, required)
 * receives ||r||_2; reading it synchronises.  When r = 0 (s = 0) xin and res are zero.
 * Uses context workspace (4 m doubles, grown on demand). */
kc_status kc_cnn_residual_sample(kc_ctx* ctx, const kc_csr* A, const double* b,
                                 const double* x, float* xin, float* res, double* rnorm);

/* Restarted flexible GMRES(opts->restart) with flexible DCGS2 and a right preconditioner
 * chosen by opts->precond:
 *   KC_PREC_AUTO with w32 != NULL: the network on the H x W grid (m = H W, row-major),
 *     M(w) = u + s net(u / s), u = D^{-1} w, s = rms(u), D = diag(A) (rows with no or a
 *     zero diagonal entry are not scaled): the Jacobi step plus the learned correction;
 *   KC_PREC_AUTO with w32 == NULL: the identity (the flexible machinery alone);
 *   KC_PREC_JACOBI: M(w) = D^{-1} w.
 * The flexible step stores zhat_k = M(w_k), applies A to it, keeps the single reduction of
 * Algorithm 4, and finalises H(:, k) = T + C_{k+1} (no H C / alpha correction); the update
 * is x += sum_k zhat_k y_k / alpha_k.  FP64 vectors; b, x device, x = x0 on entry.
 * opts->precision must be 0.  Synchronises once per cycle. */
kc_status fgmres_solve(kc_ctx* ctx, const kc_csr* A, const float* w32, int H, int W,
                       const double* b, double* x, const kc_gmres_opts* opts,
                       kc_gmres_info* info);

#ifdef __cplusplus
}
#endif

#endif /* KRYLOV_H */
