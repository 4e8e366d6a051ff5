// Internal declarations shared by the libkrylov translation units (not part of the ABI).
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>
#include <string.h>
#include <math.h>

#include "../../include/krylov.h"

namespace kc {

constexpr int NMAX = 128;            // largest basis (ncap) any kernel supports
constexpr int RED_THREADS = 512;     // threads of a reduction CTA (16 warps)
constexpr int RED_WARPS = RED_THREADS / 32;
constexpr int RED_RSUB_TASKS = 8;    // FP32 / BF16 reductions of at most this many tasks: row sub-blocks
constexpr int RED_GROUP = 16;        // partials rows per group of a two-level reduction completion
constexpr int PARTIAL_CTAS_PER_SM = 16;  // reduction CTAs per SM the partials buffer holds
                                          // (16 two-warp CTAs stream w and v at k = 0: 90 us
                                          // instead of 121 with 8, at m = 16 M)
constexpr int UPD_THREADS = 256;

// Device-resident scalars of the current step, written by the last CTA of a reduction
// (the scalar step of Algorithm 4) and read by the update kernels.
struct Scalars {
  double C[NMAX];       // delayed reorthogonalisation coefficients C_{0:k-1}
  double S[NMAX];       // projections of v (S_{0:k-1}), or a second coefficient set
  double T[NMAX + 1];   // T_{0:k}: scaled projection (Algorithm 4, eq. 30)
  double C2[NMAX];      // second CGS2 pass coefficients (finish / CGS2 baseline)
  double alpha, inv_alpha, beta, s;
  double vscale;        // factor of v in the update: 1/alpha (Arnoldi), 1 (QR of given columns)
  double cs;            // C^T S (Stephen's trick)
  double h;             // last MGS inner product
  double norm_sq;       // last explicit squared norm
  int status;           // kc_status of the last numerical check (sticky until read)
  int stop;             // drivers: set when remaining work in a captured cycle is skipped
  int ncols;            // GMRES: columns finalised so far in the cycle
  int pyth_fallbacks;
  int fallback;         // set when the explicit-norm pass must supply alpha
  // GMRES Givens state (FP64, lagged one column behind the expansion)
  double gc[NMAX], gs[NMAX], g[NMAX + 1];
  double resid_est;     // |g_{j+1}| of the last rotated column
  double rtol_abs;      // stop threshold on |g| (absolute)
  double y[NMAX];
  double zscale[NMAX];  // flexible GMRES: 1/alpha_k, the scale of the stored M(w_k)
};

// GMRES: rotate the just-finalised Hessenberg column j (rows 0..j+1) with the previous
// Givens rotations (gc, gs), make a new one, update g; R (ld ldr) receives the rotated
// column.  Returns |g_{j+1}|, the residual estimate.  Serial (one thread), O(j).
__device__ inline double givens_rotate(double* gc, double* gs, double* g, const double* H,
                                       int ldh, int j, double* R, int ldr) {
  double h[NMAX + 1];
  for (int i = 0; i <= j + 1; i++) h[i] = H[i + (int64_t)j * ldh];
  for (int i = 0; i < j; i++) {
    double t = gc[i] * h[i] + gs[i] * h[i + 1];
    h[i + 1] = -gs[i] * h[i] + gc[i] * h[i + 1];
    h[i] = t;
  }
  double r = hypot(h[j], h[j + 1]);
  double c = h[j] / r, s = h[j + 1] / r;
  gc[j] = c;
  gs[j] = s;
  h[j] = r;
  for (int i = 0; i <= j; i++) R[i + (int64_t)j * ldr] = h[i];
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  return fabs(g[j + 1]);
}

// givens_rotate on the state in sc, raising `stop` when |g_{j+1}| <= rtol_abs
__device__ inline void givens_column(Scalars* sc, const double* H, int ldh, int j, double* R,
                                     int ldr) {
  sc->resid_est = givens_rotate(sc->gc, sc->gs, sc->g, H, ldh, j, R, ldr);
  sc->ncols = j + 1;
  if (!(sc->resid_est > sc->rtol_abs)) sc->stop = 1;
}

enum Epilogue : int {
  EPI_DCGS2 = 0,        // full DCGS2 scalar step (flexible variant: see flags)
  EPI_STORE_C = 1,      // store Q^T x into C (CGS2 second projection), every product FP64
  EPI_STORE_C2 = 2,     // store Q^T x into C2
  EPI_STORE_S = 3,      // store Q^T x into S (CGS2 first projection)
  EPI_PARTIAL = 4,      // row-partitioned step: store the (k + 1) x NRHS sums to sa.part
  EPI_ICWY = 5,         // ICWY-MGS step (Section 5): norm, row of L, triangular solve
  EPI_STORE_C1 = 6,     // store Q^T x into C as a first projection, whose error a second
                        // projection removes: the offload reduction may sum it in
                        // float-float (CGS2 finish first pass)
};

enum NormEpilogue : int {
  NEPI_INIT = 0,        // alpha = ||x||, inv_alpha (start of CGS2 / MGS)
  NEPI_FINISH = 1,      // DCGS2 finish: H(:,k-1) = K + C + C2, H(k,k-1) = alpha
  NEPI_CGS2 = 2,        // CGS2 step: H(:,j) = S + C, H(j+1,j) = alpha
  NEPI_MGS = 3,         // MGS step: H(j+1,j) = alpha
  NEPI_DOT = 4,         // store x.y into h and H(i,j) (MGS inner product)
  NEPI_SQ = 5,          // store x^T x into norm_sq only (a host-read norm, no state change)
};

struct StepArgs {
  double* H;
  int ldh;
  double* K;
  int ldk;
  double* R;            // GMRES: rotated Hessenberg columns (ld ldr)
  int ldr;
  int k;                // final basis columns before this step
  int row;              // MGS inner product: row index i of H(i, k-1)
  int flags;            // bit 0: flexible (no H C / alpha correction); bit 1: GMRES Givens
  double pyth_tol;      // relative threshold on (beta - C^T C)/beta
  double* part;         // EPI_PARTIAL: destination of this rank's sums (device)
};

// SF_QR: DCGS2 QR of given columns (Algorithm 2): v is the next column a_{k+1}, not A w,
// so T = S, T_k = (s - C^T S) / alpha, the update takes v unscaled, and the pending
// column is T (no representation correction, as SF_FLEXIBLE); H(k, k-1) is written for
// k = 0 too (H points one column before R).
enum StepFlags : int { SF_FLEXIBLE = 1, SF_GIVENS = 2, SF_FALLBACK = 4, SF_QR = 8 };

}  // namespace kc

namespace kc {
enum KernelId : int {
  KID_SPMV = 0, KID_REDUCE, KID_UPDATE, KID_GEMV_SUB, KID_NORM, KID_SCALE, KID_AXPY,
  KID_SMALL, KID_OTHER, KID_FIN_REDUCE, KID_SPMV_REDUCE, KID_COUNT
};
struct TimingRec { cudaEvent_t a, b; int kid; };
}  // namespace kc

struct kc_ctx {
  int device;
  cudaStream_t stream;
  int num_sms;
  int reduce_grid;
  int red_occ[4][33];      // resident CTAs per SM of the offload reduction, by (TPW, warps)
  int red_pick[2][2][kc::NMAX + 1][6]; // its task layout per kernel (one / two vectors), size
                                       // class (m >= 2^22) and task count: nsplit, tasks per
                                       // subset, TPW, warps, CTAs/SM, row sub-blocks
  double* partials;        // PARTIAL_CTAS_PER_SM * num_sms * (2*NMAX + 4) doubles
  double* dots;            // the DCGS2 step's SpMV: per-CTA (w^T w, w^T v), 8 * num_sms pairs
  int dots_pending;        // CTAs whose pairs the next reduction of (dots_x, dots_y) takes
  const void* dots_x;
  const void* dots_y;
  unsigned int* counters;  // ticket counters for last-CTA reductions (16), then the
                           // group counters of two-level completions (group_counters)
  kc::Scalars* scal;       // device scalars
  kc::Scalars* scal_host;  // pinned host mirror for reads
  double* dwork;           // general FP64 device workspace (small dense solves)
  size_t dwork_len;
  void* ws;                // solver workspace (basis, vectors), grown on demand
  size_t ws_len;
  void* cnn_ws;            // convolutional preconditioner workspace, grown on demand
  size_t cnn_ws_len;
  int64_t launches;
  int fp64_mode;           // 0: every product in FP64; 1: FP64 with float-float offload
  int staged;              // bit 0: staged FP64 update; bit 1: tensor-copy staged reduction
  int conv_tc;             // 32 -> 32 convolutions: 0 mma.sync, 1 tcgen05 (tensor memory)
  int gmres_path;          // FP64 gmres_solve: 0 auto, 1 multi-kernel, 2 cluster, 3 grid
  int gmres_cluster;       // its cluster size once probed (0: not yet, -1: none schedulable)
  int barrier_test;        // test hook: the next grid-form solve's first barrier times out
  // optional per-kernel timing: events recorded around every launch on ctx->stream
  int timing_on;
  int timing_phase;     // 1 inside dcgs2_arnoldi_finish: its reductions count as KID_FIN_REDUCE
  kc::TimingRec* trec;
  int trec_len, trec_cap;
  char err[512];
};

namespace kc {

inline kc_status fail(kc_ctx* ctx, kc_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define KC_CUDA(ctx, call)                                                             \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return kc::fail((ctx), KC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Timing bracket around one launch (no-op unless kc_timing_enable was called).
void timing_begin(kc_ctx* ctx, int kid);
void timing_end(kc_ctx* ctx);

// Raise a kernel's dynamic shared-memory limit on the context's device, once per device
// (the attribute is per device; `done` holds one bit per device id).
template <typename Kernel>
inline kc_status smem_attr_once(kc_ctx* ctx, std::atomic<unsigned long long>& done,
                                Kernel kernel, int bytes, const char* what) {
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (done.load(std::memory_order_acquire) & bit) return KC_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return fail(ctx, KC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  done.fetch_or(bit, std::memory_order_release);
  return KC_OK;
}

// return the status of a kc_status-valued call if it is not KC_OK
#define KC_TRY(x)                 \
  do {                            \
    kc_status s_ = (x);           \
    if (s_ != KC_OK) return s_;   \
  } while (0)

#define KC_LAUNCHED(ctx)                                                               \
  do {                                                                                 \
    (ctx)->launches++;                                                                 \
    kc::timing_end(ctx);                                                               \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess)                                                             \
      return kc::fail((ctx), KC_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
  } while (0)

// Launch helpers implemented in kc_ortho.cu, used by the drivers in kc_solvers.cu.
kc_status launch_spmv(kc_ctx* ctx, const kc_csr* A, const void* x, void* y, int vec_dtype);
// v = A w of a DCGS2 step (FP64) that also forms beta = w^T w and s = w^T v per CTA; the
// next launch_reduce of (w, v) with the DCGS2 epilogue in the offload mode takes them
// instead of computing them (any other launch_reduce drops them)
kc_status launch_spmv_dots(kc_ctx* ctx, const kc_csr* A, const void* x, void* y, int vec_dtype);
// v = A w and the fused DCGS2 reduction of step k with the scalar step (EPI_DCGS2):
// launch_spmv_dots (or launch_spmv for FP32) and launch_reduce, or with kc_set_staged flag
// 8 the first steps (k <= 4, FP64 offload mode) as one fused pass
kc_status launch_matvec_reduce(kc_ctx* ctx, const kc_csr* A, const void* Q, int64_t ldq,
                               int q_dtype, int k, const void* w, void* v, int64_t m, int vec,
                               const StepArgs& sa);
kc_status launch_reduce(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k,
                        const void* x, const void* y, int64_t m, int vec_dtype, int epilogue,
                        const StepArgs& sa);
kc_status launch_dcgs2_update(kc_ctx* ctx, void* Q, int64_t ldq, int q_dtype, int k, void* w,
                              const void* v, int64_t m, int vec_dtype);
kc_status launch_gemv_sub(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k, void* x,
                          int64_t m, int vec_dtype, int which);
// the CGS2 finish's u = w - Q C1 and the sums [Q^T u, u^T u] (EPI_STORE_C2) in one pass over
// Q where it can (FP64 offload modes, k <= 64), else the two launches apart
kc_status launch_proj_reduce(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k, void* w,
                             int64_t m, int vec_dtype, const StepArgs& sa);
kc_status launch_fallback_norm(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k,
                               const void* w, int64_t m, const StepArgs& sa);
kc_status launch_norm(kc_ctx* ctx, const void* x, const void* y, int64_t m, int vec_dtype,
                      int nepi, const StepArgs& sa);
kc_status launch_scale_to(kc_ctx* ctx, const void* x, void* qcol, int q_dtype, int64_t m,
                          int vec_dtype);
kc_status launch_axpy_h(kc_ctx* ctx, const void* q, int q_dtype, void* v, int64_t m,
                        int vec_dtype);
// row-partitioned DCGS2 (kc_ortho.cu): the scalar step of Algorithm 4 from all-reduced sums
// [C_0, S_0, ..., C_{k-1}, S_{k-1}, beta, s]; the coefficients of a finish projection
// (which 0: C, 1: C2) and the squared norm from all-reduced sums; the finish's last
// column from an all-reduced ||u||^2
kc_status launch_scalar_from_totals(kc_ctx* ctx, const double* totals, int k,
                                    const StepArgs& sa);
kc_status launch_store_totals(kc_ctx* ctx, const double* totals, int k, int which);
kc_status launch_finish_from_norm(kc_ctx* ctx, const double* totals, const StepArgs& sa);
kc_status ensure_workspace(kc_ctx* ctx, size_t bytes);
// Gram matrix G = Q^T Q (FP64, ncols x ncols, column-major) and ||I - G||_F (kc_gram.cu):
// out[0] = the value, out[1] = max(out[1], value)
kc_status launch_gram(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int64_t m,
                      int ncols, double* G);
kc_status launch_loo_from_gram(kc_ctx* ctx, const double* G, int ncols, double* out);
kc_status launch_update_staged(kc_ctx* ctx, double* Q, int64_t ldq, int k, double* w,
                               const double* v, int64_t m);
// convolutional preconditioner (kc_cnn.cu)
kc_status cnn_prep(kc_ctx* ctx, const float* w32, __nv_bfloat16* wf, __nv_bfloat16* wt);
kc_status cnn_forward(kc_ctx* ctx, const __nv_bfloat16* wf, const float* x, float* y,
                      __nv_bfloat16* const* acts, bool keep, int B, int H, int W);
kc_status cnn_backward(kc_ctx* ctx, const __nv_bfloat16* wf, const __nv_bfloat16* wt,
                       const float* x, const float* g, __nv_bfloat16* const* acts,
                       __nv_bfloat16* const* dz, float* dw, int B, int H, int W);
kc_status cnn_loss_grad(kc_ctx* ctx, const float* y, const float* e, double* sums, float* g,
                        int B, int64_t npix);
kc_status cnn_conv32_tc(kc_ctx* ctx, const __nv_bfloat16* in, __nv_bfloat16* out,
                        const __nv_bfloat16* w, int B, int H, int W, int epi,
                        const __nv_bfloat16* mask);
kc_status cnn_residual_loss_grad(kc_ctx* ctx, const kc_csr* A, const float* x, const float* y,
                                 const float* r, float* res, double* sums, float* g, int B,
                                 int64_t npix);
kc_status cnn_adam(kc_ctx* ctx, float* w, const float* g, float* m, float* v, int64_t t,
                   float lr, float b1, float b2, float eps);
int64_t cnn_nparam();
// the operator is the matrix-free 7-point stencil rather than a CSR matrix
inline bool is_stencil(const kc_csr* A) { return A->grid[0] > 0; }
// the group counters of the two-level reduction completion (tree_arrive)
inline unsigned int* group_counters(kc_ctx* ctx) { return ctx->counters + 16; }

// Programmatic dependent launch (griddepcontrol) for the kernels of the DCGS2 step, which
// follow one another on the stream without a host synchronisation.  A kernel launched with
// launch_pdl may be scheduled before its predecessor has finished; it calls pdl_wait()
// before it reads anything (device scalars included), which returns once the predecessor
// grid has completed and its writes are visible (at once when the launch was an ordinary
// one).  pdl_trigger() in the predecessor lets the successor's CTAs be scheduled as soon
// as every CTA of the predecessor has passed it (or exited), so that they are resident
// while the predecessor's last CTA runs its epilogue.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(cudaStream_t stream, void (*kern)(KArgs...), dim3 grid,
                              dim3 block, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
// restarted FP64 DCGS2-GMRES in one launch (kc_gmres_cluster.cu): one thread-block
// cluster (grid_form 0) or one CTA per SM with a bounded grid barrier (grid_form 1, needs
// gmres_grid_workspace bytes at grid_ws); writes out_host[0..6] = matvecs, cycles, |g|
// estimate, ||b - A x||, ||b||, result, last status
kc_status gmres_fused_solve(kc_ctx* ctx, int grid_form, const kc_csr* A, const double* b,
                            double* x, double* Q, int64_t ldq, double* w, double* v, double* H,
                            double* K, double* R, int n, int maxit, double rtol,
                            void* grid_ws, double* out_dev, double* out_host);
size_t gmres_grid_workspace(const kc_ctx* ctx);
// gmres_path 0 takes the one-launch grid kernel up to 393,216 rows (measured crossover with
// the multi-kernel path), the multi-kernel path beyond
bool gmres_grid_preferred(kc_ctx* ctx, int64_t m, int n);
kc_status validate_csr(kc_ctx* ctx, const kc_csr* A);
// validate_csr, and A must be a CSR matrix (for callers that read its entries)
kc_status validate_csr_entries(kc_ctx* ctx, const kc_csr* A);
kc_status validate_state(kc_ctx* ctx, const kc_csr* A, const kc_arnoldi* st);

}  // namespace kc
