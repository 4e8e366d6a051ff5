// C-ABI entry points: context, validation, and the Arnoldi steps (DCGS2, CGS2, MGS).
#include "kc_internal.cuh"

#include <new>
#include <string.h>

using namespace kc;

namespace kc {

kc_status validate_csr(kc_ctx* ctx, const kc_csr* A) {
  if (!A) return fail(ctx, KC_ERR_INVALID_ARG, "A is NULL");
  if (A->m <= 0 || A->m >= (int64_t)1 << 31)
    return fail(ctx, KC_ERR_INVALID_ARG, "matrix size m = %lld out of range", (long long)A->m);
  if (A->val_dtype != KC_F64 && A->val_dtype != KC_F32)
    return fail(ctx, KC_ERR_INVALID_ARG, "matrix values must be KC_F64 or KC_F32");
  if (A->grid[0] != 0) {
    if (A->grid[0] < 0 || A->grid[1] <= 0 || A->grid[2] <= 0 ||
        (int64_t)A->grid[0] * A->grid[1] * A->grid[2] != A->m)
      return fail(ctx, KC_ERR_INVALID_ARG, "stencil grid %d x %d x %d does not have m = %lld points",
                  A->grid[0], A->grid[1], A->grid[2], (long long)A->m);
    return KC_OK;
  }
  if (A->nnz < 0 || A->nnz >= (int64_t)1 << 31)
    return fail(ctx, KC_ERR_INVALID_ARG, "nnz = %lld does not fit int32 indices", (long long)A->nnz);
  if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val)))
    return fail(ctx, KC_ERR_INVALID_ARG, "CSR arrays must be non-NULL device pointers");
  return KC_OK;
}

kc_status validate_csr_entries(kc_ctx* ctx, const kc_csr* A) {
  KC_TRY(validate_csr(ctx, A));
  if (is_stencil(A))
    return fail(ctx, KC_ERR_INVALID_ARG, "this entry point reads matrix entries: A must be CSR");
  return KC_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

kc_status validate_state(kc_ctx* ctx, const kc_csr* A, const kc_arnoldi* st) {
  if (!st) return fail(ctx, KC_ERR_INVALID_ARG, "state is NULL");
  if (!st->Q || !st->w || !st->v || !st->H || !st->K)
    return fail(ctx, KC_ERR_INVALID_ARG, "state buffers must be non-NULL device pointers");
  if (!aligned16(st->Q) || !aligned16(st->w) || !aligned16(st->v))
    return fail(ctx, KC_ERR_INVALID_ARG, "Q, w and v must be 16-byte aligned");
  if (st->ncap < 2 || st->ncap > NMAX)
    return fail(ctx, KC_ERR_INVALID_ARG, "ncap = %d outside [2, %d]", st->ncap, NMAX);
  if (st->ldq < A->m || (st->ldq % 8) != 0)
    return fail(ctx, KC_ERR_INVALID_ARG, "ldq = %lld must be >= m and a multiple of 8",
                (long long)st->ldq);
  if (st->ldh < st->ncap) return fail(ctx, KC_ERR_INVALID_ARG, "ldh < ncap");
  if (st->q_dtype != KC_F64 && st->q_dtype != KC_F32 && st->q_dtype != KC_BF16)
    return fail(ctx, KC_ERR_INVALID_ARG, "q_dtype must be KC_F64, KC_F32 or KC_BF16");
  const int vec = st->q_dtype == KC_F64 ? KC_F64 : KC_F32;
  if (A->val_dtype != vec)
    return fail(ctx, KC_ERR_INVALID_ARG,
                "basis type %d needs %s matrix values", st->q_dtype, vec == KC_F64 ? "FP64" : "FP32");
  if (st->k < 0 || st->k >= st->ncap) return fail(ctx, KC_ERR_INVALID_ARG, "corrupt k = %d", st->k);
  return KC_OK;
}

void timing_begin(kc_ctx* ctx, int kid) {
  if (!ctx->timing_on) return;
  if (ctx->trec_len == ctx->trec_cap) {
    int ncap = ctx->trec_cap ? 2 * ctx->trec_cap : 1024;
    TimingRec* n = new (std::nothrow) TimingRec[ncap];
    if (!n) return;
    for (int i = 0; i < ctx->trec_cap; i++) n[i] = ctx->trec[i];
    for (int i = ctx->trec_cap; i < ncap; i++) {
      cudaEventCreate(&n[i].a);
      cudaEventCreate(&n[i].b);
    }
    delete[] ctx->trec;
    ctx->trec = n;
    ctx->trec_cap = ncap;
  }
  TimingRec& r = ctx->trec[ctx->trec_len];
  r.kid = (ctx->timing_phase == 1 && kid == KID_REDUCE) ? KID_FIN_REDUCE : kid;
  cudaEventRecord(r.a, ctx->stream);
}

void timing_end(kc_ctx* ctx) {
  if (!ctx->timing_on || ctx->trec_len >= ctx->trec_cap) return;
  cudaEventRecord(ctx->trec[ctx->trec_len].b, ctx->stream);
  ctx->trec_len++;
}

}  // namespace kc

static int vec_of(const kc_arnoldi* st) { return st->q_dtype == KC_F64 ? KC_F64 : KC_F32; }
static size_t qsize(int dt) { return dt == KC_F64 ? 8 : (dt == KC_F32 ? 4 : 2); }
static void* qcol(const kc_arnoldi* st, int j) {
  return (char*)st->Q + (size_t)j * st->ldq * qsize(st->q_dtype);
}

static StepArgs step_args(const kc_arnoldi* st, int k, int flags) {
  StepArgs sa;
  sa.H = st->H;
  sa.ldh = st->ldh;
  sa.K = st->K;
  sa.ldk = st->ncap;
  sa.R = nullptr;
  sa.ldr = 0;
  sa.k = k;
  sa.row = 0;
  sa.flags = flags;
  // FP64: flag only a non-positive Pythagorean norm; FP32/BF16: 64 unit roundoffs
  sa.pyth_tol = st->q_dtype == KC_F64 ? 0.0 : 64.0 * 5.9604644775390625e-08;
  return sa;
}

extern "C" {

kc_status kc_create(kc_ctx** out, int device, void* cuda_stream) {
  if (!out) return KC_ERR_INVALID_ARG;
  *out = nullptr;
  kc_ctx* ctx = new (std::nothrow) kc_ctx;
  if (!ctx) return KC_ERR_OOM;
  memset(ctx, 0, sizeof(*ctx));
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) { delete ctx; return KC_ERR_CUDA; }
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) { delete ctx; return KC_ERR_CUDA; }
  ctx->num_sms = p.multiProcessorCount;
  ctx->fp64_mode = 1;
  ctx->conv_tc = 1;
  ctx->reduce_grid = 2 * p.multiProcessorCount;
  const size_t plen =
      (size_t)PARTIAL_CTAS_PER_SM * p.multiProcessorCount * (2 * NMAX + 4) * sizeof(double);
  // 16 ticket counters, then one per group of RED_GROUP partials rows (group_counters)
  const size_t ncount = 16 + ((size_t)PARTIAL_CTAS_PER_SM * p.multiProcessorCount + RED_GROUP - 1) / RED_GROUP;
  bool ok = cudaMalloc(&ctx->partials, plen) == cudaSuccess &&
            cudaMalloc(&ctx->dots, (size_t)16 * p.multiProcessorCount * sizeof(double)) ==
                cudaSuccess &&
            cudaMalloc(&ctx->counters, ncount * sizeof(unsigned int)) == cudaSuccess &&
            cudaMalloc(&ctx->scal, sizeof(Scalars)) == cudaSuccess &&
            cudaMallocHost(&ctx->scal_host, sizeof(Scalars)) == cudaSuccess;
  ctx->dwork_len = 1 << 20;
  ok = ok && cudaMalloc(&ctx->dwork, ctx->dwork_len * sizeof(double)) == cudaSuccess;
  if (ok) ok = cudaMemset(ctx->counters, 0, ncount * sizeof(unsigned int)) == cudaSuccess &&
               cudaMemset(ctx->scal, 0, sizeof(Scalars)) == cudaSuccess &&
               cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    kc_destroy(ctx);
    return KC_ERR_OOM;
  }
  *out = ctx;
  return KC_OK;
}

kc_status kc_destroy(kc_ctx* ctx) {
  if (!ctx) return KC_OK;
  for (int i = 0; i < ctx->trec_cap; i++) {
    cudaEventDestroy(ctx->trec[i].a);
    cudaEventDestroy(ctx->trec[i].b);
  }
  delete[] ctx->trec;
  if (ctx->partials) cudaFree(ctx->partials);
  if (ctx->dots) cudaFree(ctx->dots);
  if (ctx->counters) cudaFree(ctx->counters);
  if (ctx->scal) cudaFree(ctx->scal);
  if (ctx->scal_host) cudaFreeHost(ctx->scal_host);
  if (ctx->dwork) cudaFree(ctx->dwork);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->cnn_ws) cudaFree(ctx->cnn_ws);
  delete ctx;
  return KC_OK;
}

kc_status kc_set_fp64_mode(kc_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return KC_ERR_INVALID_ARG;
  ctx->fp64_mode = mode;
  return KC_OK;
}

int kc_get_fp64_mode(const kc_ctx* ctx) { return ctx ? ctx->fp64_mode : -1; }

kc_status kc_set_conv_kernel(kc_ctx* ctx, int kind) {
  if (!ctx || kind < 0 || kind > 1) return KC_ERR_INVALID_ARG;
  ctx->conv_tc = kind;
  return KC_OK;
}

kc_status kc_set_gmres_path(kc_ctx* ctx, int path) {
  if (!ctx || path < 0 || path > 3) return KC_ERR_INVALID_ARG;
  ctx->gmres_path = path;
  return KC_OK;
}

kc_status kc_set_barrier_test(kc_ctx* ctx, int on) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  ctx->barrier_test = on ? 1 : 0;
  return KC_OK;
}

kc_status kc_set_staged(kc_ctx* ctx, int flags) {
  if (!ctx || flags < 0 || flags > 15) return KC_ERR_INVALID_ARG;
  ctx->staged = flags;
  return KC_OK;
}

kc_status kc_set_stream(kc_ctx* ctx, void* cuda_stream) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)cuda_stream;
  return KC_OK;
}

const char* kc_last_error(const kc_ctx* ctx) { return ctx ? ctx->err : "no context"; }

kc_status kc_device_info(const kc_ctx* ctx, int* num_sms, int* reduce_grid) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  if (num_sms) *num_sms = ctx->num_sms;
  if (reduce_grid) *reduce_grid = ctx->reduce_grid;
  return KC_OK;
}

int64_t kc_launch_count(const kc_ctx* ctx) { return ctx ? ctx->launches : -1; }

kc_status kc_timing_enable(kc_ctx* ctx, int on) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  ctx->timing_on = on;
  ctx->trec_len = 0;
  return KC_OK;
}

kc_status kc_timing_read(kc_ctx* ctx, double* ms, int64_t* count, int nkinds) {
  if (!ctx || !ms || !count || nkinds < KID_COUNT) return fail(ctx, KC_ERR_INVALID_ARG, "kc_timing_read: bad arguments");
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < nkinds; i++) { ms[i] = 0.0; count[i] = 0; }
  for (int i = 0; i < ctx->trec_len; i++) {
    float t = 0.f;
    KC_CUDA(ctx, cudaEventElapsedTime(&t, ctx->trec[i].a, ctx->trec[i].b));
    ms[ctx->trec[i].kid] += t;
    count[ctx->trec[i].kid] += 1;
  }
  ctx->trec_len = 0;
  return KC_OK;
}

kc_status kc_read_status(kc_ctx* ctx, int* device_status) {
  if (!ctx || !device_status) return KC_ERR_INVALID_ARG;
  KC_CUDA(ctx, cudaMemcpyAsync(&ctx->scal_host->status, &ctx->scal->status, sizeof(int),
                               cudaMemcpyDeviceToHost, ctx->stream));
  KC_CUDA(ctx, cudaMemsetAsync(&ctx->scal->status, 0, sizeof(int), ctx->stream));
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *device_status = ctx->scal_host->status;
  return KC_OK;
}

kc_status kc_last_scalars(kc_ctx* ctx, double* alpha, double* beta, double* s) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_CUDA(ctx, cudaMemcpyAsync(&ctx->scal_host->alpha, &ctx->scal->alpha, 4 * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (alpha) *alpha = ctx->scal_host->alpha;
  if (beta) *beta = ctx->scal_host->beta;
  if (s) *s = ctx->scal_host->s;
  return KC_OK;
}

kc_status kc_spmv(kc_ctx* ctx, const kc_csr* A, const void* x, void* y) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  if (!x || !y) return fail(ctx, KC_ERR_INVALID_ARG, "x and y must be non-NULL");
  return launch_spmv(ctx, A, x, y, A->val_dtype);
}

kc_status dcgs2_arnoldi_init(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st, const void* r0) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  st->k = 0;
  st->finished = 0;
  KC_TRY(validate_state(ctx, A, st));
  if (!r0) return fail(ctx, KC_ERR_INVALID_ARG, "r0 is NULL");
  const size_t vbytes = (size_t)A->m * (vec_of(st) == KC_F64 ? 8 : 4);
  if (r0 != st->w)
    KC_CUDA(ctx, cudaMemcpyAsync(st->w, r0, vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return KC_OK;
}

kc_status dcgs2_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  KC_TRY(validate_state(ctx, A, st));
  const int k = st->k;
  if (k + 2 > st->ncap)
    return fail(ctx, KC_ERR_INVALID_ARG, "basis full: k = %d, ncap = %d", k, st->ncap);
  if (st->finished) return fail(ctx, KC_ERR_INVALID_ARG, "expansion already finished");
  const int vec = vec_of(st);
  StepArgs sa = step_args(st, k, vec == KC_F32 ? SF_FALLBACK : 0);
  KC_TRY(launch_matvec_reduce(ctx, A, st->Q, st->ldq, st->q_dtype, k, st->w, st->v, A->m, vec,
                              sa));                      // v = A w and the one reduction
  if (vec == KC_F32)   // reduced precision: explicit norm when Pythagoras lost its digits
    KC_TRY(launch_fallback_norm(ctx, st->Q, st->ldq, st->q_dtype, k, st->w, A->m, sa));
  KC_TRY(launch_dcgs2_update(ctx, st->Q, st->ldq, st->q_dtype, k, st->w, st->v, A->m, vec));
  st->k = k + 1;
  return KC_OK;
}

kc_status dcgs2_arnoldi_finish(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  KC_TRY(validate_state(ctx, A, st));
  const int k = st->k;
  if (k < 1) return fail(ctx, KC_ERR_INVALID_ARG, "finish needs at least one step");
  if (st->finished) return fail(ctx, KC_ERR_INVALID_ARG, "expansion already finished");
  const int vec = vec_of(st);
  StepArgs sa = step_args(st, k, 0);
  struct Phase {                       // the finish's reductions are timed on their own
    kc_ctx* c;
    explicit Phase(kc_ctx* cc) : c(cc) { c->timing_phase = 1; }
    ~Phase() { c->timing_phase = 0; }
  } phase(ctx);
  KC_TRY(launch_reduce(ctx, st->Q, st->ldq, st->q_dtype, k, st->w, nullptr, A->m, vec,
                       EPI_STORE_C1, sa));                               // C1 = Q^T w
  KC_TRY(launch_proj_reduce(ctx, st->Q, st->ldq, st->q_dtype, k, st->w, A->m, vec,
                            sa));                  // u = w - Q C1, C2 = Q^T u in one pass
  KC_TRY(launch_gemv_sub(ctx, st->Q, st->ldq, st->q_dtype, k, st->w, A->m, vec, 1));
  KC_TRY(launch_norm(ctx, st->w, nullptr, A->m, vec, NEPI_FINISH, sa));  // alpha = ||u||
  KC_TRY(launch_scale_to(ctx, st->w, qcol(st, k), st->q_dtype, A->m, vec));
  st->finished = 1;
  return KC_OK;
}

// ---- row-partitioned DCGS2 (Section 5: rows of Q, w, v and A split across ranks) -----

static kc_status part_checks(kc_ctx* ctx, const kc_csr* A, const kc_arnoldi* st) {
  if (st->q_dtype != KC_F64)
    return fail(ctx, KC_ERR_INVALID_ARG, "row-partitioned step: FP64 basis only");
  if (A && (A->val_dtype != KC_F64 || is_stencil(A)))
    return fail(ctx, KC_ERR_INVALID_ARG, "row-partitioned step: FP64 CSR rows only");
  return KC_OK;
}

kc_status dcgs2_part_reduce(kc_ctx* ctx, const kc_csr* A_local, kc_arnoldi* st,
                            const double* w_ext, double* partial) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr_entries(ctx, A_local));
  KC_TRY(validate_state(ctx, A_local, st));
  KC_TRY(part_checks(ctx, A_local, st));
  if (!w_ext || !partial) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  const int k = st->k;
  if (k + 2 > st->ncap)
    return fail(ctx, KC_ERR_INVALID_ARG, "basis full: k = %d, ncap = %d", k, st->ncap);
  if (st->finished) return fail(ctx, KC_ERR_INVALID_ARG, "expansion already finished");
  KC_TRY(launch_spmv(ctx, A_local, w_ext, st->v, KC_F64));          // this rank's rows of A w
  StepArgs sa = step_args(st, k, 0);
  sa.part = partial;
  return launch_reduce(ctx, st->Q, st->ldq, KC_F64, k, st->w, st->v, A_local->m, KC_F64,
                       EPI_PARTIAL, sa);
}

kc_status dcgs2_part_update(kc_ctx* ctx, const kc_csr* A_local, kc_arnoldi* st,
                            const double* totals) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A_local));
  KC_TRY(validate_state(ctx, A_local, st));
  KC_TRY(part_checks(ctx, A_local, st));
  if (!totals) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  const int k = st->k;
  if (k + 2 > st->ncap || st->finished)
    return fail(ctx, KC_ERR_INVALID_ARG, "no step to complete at k = %d", k);
  StepArgs sa = step_args(st, k, 0);
  KC_TRY(launch_scalar_from_totals(ctx, totals, k, sa));
  KC_TRY(launch_dcgs2_update(ctx, st->Q, st->ldq, KC_F64, k, st->w, st->v, A_local->m, KC_F64));
  st->k = k + 1;
  return KC_OK;
}

kc_status dcgs2_part_finish(kc_ctx* ctx, const kc_csr* A_local, kc_arnoldi* st, int phase,
                            const double* totals, double* partial) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A_local));
  KC_TRY(validate_state(ctx, A_local, st));
  KC_TRY(part_checks(ctx, A_local, st));
  const int k = st->k;
  if (k < 1 || st->finished) return fail(ctx, KC_ERR_INVALID_ARG, "nothing to finish");
  if (phase < 0 || phase > 3) return fail(ctx, KC_ERR_INVALID_ARG, "phase must be 0..3");
  if ((phase > 0 && !totals) || (phase < 3 && !partial))
    return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  const int64_t m = A_local->m;
  StepArgs sa = step_args(st, k, 0);
  sa.part = partial;
  struct Phase {
    kc_ctx* c;
    explicit Phase(kc_ctx* cc) : c(cc) { c->timing_phase = 1; }
    ~Phase() { c->timing_phase = 0; }
  } timing(ctx);
  if (phase == 0)                  // partial = [Q^T w, w^T w]
    return launch_reduce(ctx, st->Q, st->ldq, KC_F64, k, st->w, nullptr, m, KC_F64,
                         EPI_PARTIAL, sa);
  if (phase == 1 || phase == 2) {  // u -= Q c with the summed c; partial of the next sums
    KC_TRY(launch_store_totals(ctx, totals, k, phase - 1));
    KC_TRY(launch_gemv_sub(ctx, st->Q, st->ldq, KC_F64, k, st->w, m, KC_F64, phase - 1));
    if (phase == 1)                // partial = [Q^T u, u^T u]
      return launch_reduce(ctx, st->Q, st->ldq, KC_F64, k, st->w, nullptr, m, KC_F64,
                           EPI_PARTIAL, sa);
    return launch_reduce(ctx, st->Q, st->ldq, KC_F64, 0, st->w, nullptr, m, KC_F64,
                         EPI_PARTIAL, sa);        // partial = [u^T u]
  }
  KC_TRY(launch_finish_from_norm(ctx, totals, sa));   // H column, alpha = ||u||
  KC_TRY(launch_scale_to(ctx, st->w, qcol(st, k), KC_F64, m, KC_F64));
  st->finished = 1;
  return KC_OK;
}

// DCGS2 QR of given columns (Algorithm 2): the Arnoldi step's kernels with v = a_{k+1}
// (SF_QR in the scalar step), H pointing one column before R so that H(:, k - 1) is
// R(:, k), and the CGS2 finish for the last column.
kc_status dcgs2_qr(kc_ctx* ctx, const double* A, int64_t lda, int64_t m, int n, double* Q,
                   int64_t ldq, double* R, int ldr) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  if (!A || !Q || !R) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  if (m < 1 || n < 1 || n + 1 > NMAX)
    return fail(ctx, KC_ERR_INVALID_ARG, "dcgs2_qr: need m >= 1 and 1 <= n <= %d", NMAX - 1);
  if (lda < m || ldq < m || ldr < n)
    return fail(ctx, KC_ERR_INVALID_ARG, "dcgs2_qr: leading dimensions too small");
  if ((lda & 1) || (ldq & 1) || ((uintptr_t)A & 15) || ((uintptr_t)Q & 15))
    return fail(ctx, KC_ERR_INVALID_ARG,
                "dcgs2_qr: A, Q must be 16-byte aligned with even leading dimensions");
  const int64_t ldw = (m + 31) / 32 * 32;
  const size_t kbytes = (size_t)(n + 1) * n * 8;
  KC_TRY(ensure_workspace(ctx, (size_t)ldw * 8 + kbytes));
  double* w = (double*)ctx->ws;
  double* K = w + ldw;
  KC_CUDA(ctx, cudaMemsetAsync(K, 0, kbytes, ctx->stream));
  KC_CUDA(ctx, cudaMemset2DAsync(R, (size_t)ldr * 8, 0, (size_t)n * 8, (size_t)n, ctx->stream));
  KC_CUDA(ctx, cudaMemcpyAsync(w, A, (size_t)m * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  StepArgs sa = {};
  sa.H = R + ldr;                      // H(i, j) = R(i, j + 1)
  sa.ldh = ldr;
  sa.K = K;
  sa.ldk = n + 1;
  sa.flags = SF_QR;
  if (n == 1) {                        // q_0 = a_0 / ||a_0||, R(0, 0) = ||a_0||
    KC_TRY(launch_norm(ctx, w, nullptr, m, KC_F64, NEPI_INIT, sa));
    KC_TRY(launch_scale_to(ctx, w, Q, KC_F64, m, KC_F64));
    KC_CUDA(ctx, cudaMemcpyAsync(R, &ctx->scal->alpha, 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return KC_OK;
  }
  for (int k = 0; k + 1 < n; k++) {    // step k: q_k and R(:, k); pending a_{k+1}
    const double* v = A + (int64_t)(k + 1) * lda;
    sa.k = k;
    KC_TRY(launch_reduce(ctx, Q, ldq, KC_F64, k, w, v, m, KC_F64, EPI_DCGS2, sa));
    KC_TRY(launch_dcgs2_update(ctx, Q, ldq, KC_F64, k, w, v, m, KC_F64));
  }
  const int k = n - 1;                 // last column: CGS2 with an explicit norm
  sa.k = k;
  KC_TRY(launch_reduce(ctx, Q, ldq, KC_F64, k, w, nullptr, m, KC_F64, EPI_STORE_C1, sa));
  KC_TRY(launch_gemv_sub(ctx, Q, ldq, KC_F64, k, w, m, KC_F64, 0));
  KC_TRY(launch_reduce(ctx, Q, ldq, KC_F64, k, w, nullptr, m, KC_F64, EPI_STORE_C2, sa));
  KC_TRY(launch_gemv_sub(ctx, Q, ldq, KC_F64, k, w, m, KC_F64, 1));
  KC_TRY(launch_norm(ctx, w, nullptr, m, KC_F64, NEPI_FINISH, sa));
  KC_TRY(launch_scale_to(ctx, w, Q + (int64_t)k * ldq, KC_F64, m, KC_F64));
  return KC_OK;
}

// ---- ICWY-MGS (Section 5): the fused reduction with the ICWY epilogue, then the DCGS2
// update with C = 0 (q_k = w / alpha, w <- v / alpha - Q_{k+1} y) -------------------------

kc_status icwy_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  KC_TRY(validate_state(ctx, A, st));
  if (st->q_dtype != KC_F64) return fail(ctx, KC_ERR_INVALID_ARG, "ICWY-MGS: FP64 basis only");
  const int k = st->k;
  if (k + 2 > st->ncap)
    return fail(ctx, KC_ERR_INVALID_ARG, "basis full: k = %d, ncap = %d", k, st->ncap);
  if (st->finished) return fail(ctx, KC_ERR_INVALID_ARG, "expansion already finished");
  KC_TRY(launch_spmv(ctx, A, st->w, st->v, KC_F64));                  // v = A w
  StepArgs sa = step_args(st, k, 0);
  KC_TRY(launch_reduce(ctx, st->Q, st->ldq, KC_F64, k, st->w, st->v, A->m, KC_F64, EPI_ICWY,
                       sa));                                          // the one reduction
  KC_TRY(launch_dcgs2_update(ctx, st->Q, st->ldq, KC_F64, k, st->w, st->v, A->m, KC_F64));
  st->k = k + 1;
  return KC_OK;
}

kc_status icwy_arnoldi_finish(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  KC_TRY(validate_state(ctx, A, st));
  const int k = st->k;
  if (k < 1) return fail(ctx, KC_ERR_INVALID_ARG, "finish needs at least one step");
  if (st->finished) return fail(ctx, KC_ERR_INVALID_ARG, "expansion already finished");
  StepArgs sa = step_args(st, k, 0);
  KC_TRY(launch_norm(ctx, st->w, nullptr, A->m, KC_F64, NEPI_MGS, sa));   // H(k, k-1) = ||w||
  KC_TRY(launch_scale_to(ctx, st->w, qcol(st, k), KC_F64, A->m, KC_F64));
  st->finished = 1;
  return KC_OK;
}

kc_status icwy_qr(kc_ctx* ctx, const double* A, int64_t lda, int64_t m, int n, double* Q,
                  int64_t ldq, double* R, int ldr) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  if (!A || !Q || !R) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  if (m < 1 || n < 1 || n + 1 > NMAX)
    return fail(ctx, KC_ERR_INVALID_ARG, "icwy_qr: need m >= 1 and 1 <= n <= %d", NMAX - 1);
  if (lda < m || ldq < m || ldr < n)
    return fail(ctx, KC_ERR_INVALID_ARG, "icwy_qr: leading dimensions too small");
  if ((lda & 1) || (ldq & 1) || ((uintptr_t)A & 15) || ((uintptr_t)Q & 15))
    return fail(ctx, KC_ERR_INVALID_ARG,
                "icwy_qr: A, Q must be 16-byte aligned with even leading dimensions");
  const int64_t ldw = (m + 31) / 32 * 32;
  const size_t lbytes = (size_t)(n + 1) * n * 8;
  KC_TRY(ensure_workspace(ctx, (size_t)ldw * 8 + lbytes));
  double* w = (double*)ctx->ws;
  double* L = w + ldw;                 // the strictly lower triangular L, ld n + 1
  KC_CUDA(ctx, cudaMemsetAsync(L, 0, lbytes, ctx->stream));
  KC_CUDA(ctx, cudaMemset2DAsync(R, (size_t)ldr * 8, 0, (size_t)n * 8, (size_t)n, ctx->stream));
  KC_CUDA(ctx, cudaMemcpyAsync(w, A, (size_t)m * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  StepArgs sa = {};
  sa.H = R + ldr;                      // H(i, j) = R(i, j + 1)
  sa.ldh = ldr;
  sa.K = L;
  sa.ldk = n + 1;
  sa.flags = SF_QR;
  for (int k = 0; k + 1 < n; k++) {    // step k: q_k, R(k, k) and R(0:k+1, k+1); pending a_{k+1}
    const double* v = A + (int64_t)(k + 1) * lda;
    sa.k = k;
    KC_TRY(launch_reduce(ctx, Q, ldq, KC_F64, k, w, v, m, KC_F64, EPI_ICWY, sa));
    KC_TRY(launch_dcgs2_update(ctx, Q, ldq, KC_F64, k, w, v, m, KC_F64));
  }
  sa.k = n - 1;                        // the last column: its norm (R(n-1, n-1)) and q_{n-1}
  KC_TRY(launch_norm(ctx, w, nullptr, m, KC_F64, NEPI_MGS, sa));
  KC_TRY(launch_scale_to(ctx, w, Q + (int64_t)(n - 1) * ldq, KC_F64, m, KC_F64));
  return KC_OK;
}

kc_status cgs2_arnoldi_init(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st, const void* r0) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  st->k = 0;
  st->finished = 0;
  KC_TRY(validate_state(ctx, A, st));
  if (st->q_dtype != KC_F64)
    return fail(ctx, KC_ERR_INVALID_ARG, "the CGS2 / MGS baselines are FP64 only");
  if (!r0) return fail(ctx, KC_ERR_INVALID_ARG, "r0 is NULL");
  StepArgs sa = step_args(st, 0, 0);
  KC_TRY(launch_norm(ctx, r0, nullptr, A->m, KC_F64, NEPI_INIT, sa));
  KC_TRY(launch_scale_to(ctx, r0, st->Q, KC_F64, A->m, KC_F64));      // q_0 = r0/||r0||
  st->k = 1;
  return KC_OK;
}

kc_status cgs2_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  KC_TRY(validate_state(ctx, A, st));
  if (st->q_dtype != KC_F64)
    return fail(ctx, KC_ERR_INVALID_ARG, "the CGS2 / MGS baselines are FP64 only");
  const int k = st->k;
  if (k < 1 || k + 1 > st->ncap)
    return fail(ctx, KC_ERR_INVALID_ARG, "CGS2 step needs 1 <= k < ncap (k = %d)", k);
  StepArgs sa = step_args(st, k, 0);
  KC_TRY(launch_spmv(ctx, A, qcol(st, k - 1), st->v, KC_F64));          // v = A q_{k-1}
  KC_TRY(launch_reduce(ctx, st->Q, st->ldq, KC_F64, k, st->v, nullptr, A->m, KC_F64,
                       EPI_STORE_S, sa));                                // S = Q^T v
  KC_TRY(launch_gemv_sub(ctx, st->Q, st->ldq, KC_F64, k, st->v, A->m, KC_F64, 2));
  KC_TRY(launch_reduce(ctx, st->Q, st->ldq, KC_F64, k, st->v, nullptr, A->m, KC_F64,
                       EPI_STORE_C, sa));                                // C = Q^T w
  KC_TRY(launch_gemv_sub(ctx, st->Q, st->ldq, KC_F64, k, st->v, A->m, KC_F64, 0));
  KC_TRY(launch_norm(ctx, st->v, nullptr, A->m, KC_F64, NEPI_CGS2, sa)); // alpha = ||u||
  KC_TRY(launch_scale_to(ctx, st->v, qcol(st, k), KC_F64, A->m, KC_F64));
  st->k = k + 1;
  return KC_OK;
}

kc_status mgs_arnoldi_step(kc_ctx* ctx, const kc_csr* A, kc_arnoldi* st) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  KC_TRY(validate_csr(ctx, A));
  KC_TRY(validate_state(ctx, A, st));
  if (st->q_dtype != KC_F64)
    return fail(ctx, KC_ERR_INVALID_ARG, "the CGS2 / MGS baselines are FP64 only");
  const int k = st->k;
  if (k < 1 || k + 1 > st->ncap)
    return fail(ctx, KC_ERR_INVALID_ARG, "MGS step needs 1 <= k < ncap (k = %d)", k);
  StepArgs sa = step_args(st, k, 0);
  KC_TRY(launch_spmv(ctx, A, qcol(st, k - 1), st->v, KC_F64));
  for (int i = 0; i < k; i++) {
    sa.row = i;
    KC_TRY(launch_norm(ctx, qcol(st, i), st->v, A->m, KC_F64, NEPI_DOT, sa));  // h = q_i^T v
    KC_TRY(launch_axpy_h(ctx, qcol(st, i), KC_F64, st->v, A->m, KC_F64));      // v -= h q_i
  }
  KC_TRY(launch_norm(ctx, st->v, nullptr, A->m, KC_F64, NEPI_MGS, sa));
  KC_TRY(launch_scale_to(ctx, st->v, qcol(st, k), KC_F64, A->m, KC_F64));
  st->k = k + 1;
  return KC_OK;
}

}  // extern "C"
