// Drivers on top of the Arnoldi kernels:
//   gmres_solve: restarted DCGS2-GMRES(n) in FP64, or FP32 / BF16-basis inner solves in
//                FP64 iterative refinement (Givens rotations and the small triangular
//                solve stay in FP64 on the GPU);
//   krylov_schur_eigs: see kc_schur.cu.
// The expansion of a cycle is enqueued without host synchronisation; the Givens rotation
// of each finalised Hessenberg column runs in the last CTA of the next step's reduction and
// raises a device `stop` flag at convergence, after which every remaining kernel of the
// cycle returns at once.  The host reads the scalars once per cycle.
#include "kc_internal.cuh"

namespace kc {

kc_status ensure_workspace(kc_ctx* ctx, size_t bytes) {
  if (ctx->ws_len >= bytes) return KC_OK;
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_len = 0;
  if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess)
    return fail(ctx, KC_ERR_OOM, "could not allocate %zu bytes of solver workspace", bytes);
  ctx->ws_len = bytes;
  return KC_OK;
}

// ---- small kernels ----------------------------------------------------------------------

__global__ void k_cycle_begin(Scalars* sc, double rtol_abs) {
  sc->stop = 0;
  sc->ncols = 0;
  sc->fallback = 0;
  sc->rtol_abs = rtol_abs;
  sc->resid_est = 0.0;
}

// y = R^{-1} g (back substitution, FP64), R upper triangular ncols x ncols, ld ldr.
__global__ void k_tri_solve(const double* __restrict__ R, int ldr, Scalars* sc) {
  if (threadIdx.x != 0) return;
  const int n = sc->ncols;
  for (int i = n - 1; i >= 0; i--) {
    double t = sc->g[i];
    for (int j = i + 1; j < n; j++) t -= R[i + (int64_t)j * ldr] * sc->y[j];
    sc->y[i] = t / R[i + (int64_t)i * ldr];
  }
}

template <typename T> __device__ __forceinline__ double qval(const T* p, int64_t i);
template <> __device__ __forceinline__ double qval(const double* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ double qval(const float* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ double qval(const __nv_bfloat16* p, int64_t i) {
  return __uint_as_float(((unsigned int)reinterpret_cast<const unsigned short*>(p)[i]) << 16);
}

// x += Q(:, 0:ncols) y  (K9: basis update of the solution)
template <typename TQ, typename TX>
__global__ void __launch_bounds__(256) k_x_update(const TQ* __restrict__ Q, int64_t ldq,
                                                  TX* __restrict__ x, int64_t m,
                                                  const Scalars* __restrict__ sc) {
  __shared__ double y[NMAX];
  const int n = sc->ncols;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = sc->y[i];
  __syncthreads();
  // an FP32 solution (the inner solve of iterative refinement, tolerance 1e-4) is
  // accumulated in FP32: the FP64 pipe would bound this HBM pass at n FMAs per row
  using TS = typename std::conditional<sizeof(TX) == 4, float, double>::type;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    TS s = 0;
    for (int j = 0; j < n; j++) s += (TS)qval(Q + (int64_t)j * ldq, r) * (TS)y[j];
    x[r] = (TX)((TS)x[r] + s);
  }
}

// r = b - Av
template <typename T>
__global__ void __launch_bounds__(256) k_sub(const T* __restrict__ b, const T* __restrict__ Av,
                                             T* __restrict__ r, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - Av[i];
}

// w32 = (float)(r * s)
__global__ void __launch_bounds__(256) k_cast_scale(const double* __restrict__ r, double s,
                                                    float* __restrict__ w, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (float)(r[i] * s);
}

// x += s * d
__global__ void __launch_bounds__(256) k_add_scaled(double* __restrict__ x, double s,
                                                    const float* __restrict__ d, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += s * (double)d[i];
}

static int grid1d(const kc_ctx* ctx, int64_t m) {
  int64_t b = (m + 255) / 256;
  int64_t cap = (int64_t)ctx->num_sms * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

static kc_status read_scalars(kc_ctx* ctx) {
  KC_CUDA(ctx, cudaMemcpyAsync(ctx->scal_host, ctx->scal, sizeof(Scalars),
                               cudaMemcpyDeviceToHost, ctx->stream));
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return KC_OK;
}

// ||x||^2 of an m-vector (FP64 or FP32) -> host
static kc_status host_norm(kc_ctx* ctx, const void* x, int64_t m, int vec, double* out) {
  StepArgs sa = {};
  sa.k = 0;
  kc_status s = launch_norm(ctx, x, nullptr, m, vec, NEPI_INIT, sa);
  if (s != KC_OK) return s;
  KC_CUDA(ctx, cudaMemcpyAsync(&ctx->scal_host->norm_sq, &ctx->scal->norm_sq, sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *out = sqrt(ctx->scal_host->norm_sq);
  return KC_OK;
}

struct Cycle {
  void* Q;
  int64_t ldq;
  int qdt;          // basis type
  int vec;          // vector type (F64 / F32)
  void* w;          // holds the cycle's residual on entry
  void* v;
  double* H;
  double* K;
  double* R;
  int n;
  double* gram;     // diagnostics: (n+1)^2 Gram matrix and loo[2] (NULL: off)
  double* loo;
};

// One GMRES(n) cycle: expansion with lagged Givens rotations, then x += Q y.
static kc_status gmres_cycle(kc_ctx* ctx, const kc_csr* A, const Cycle& c, void* x,
                             double rtol_abs, int* ncols_out, double* est_out, int* matvecs,
                             int* status) {
  const int64_t m = A->m;
  timing_begin(ctx, KID_SMALL);
  k_cycle_begin<<<1, 1, 0, ctx->stream>>>(ctx->scal, rtol_abs);
  KC_LAUNCHED(ctx);
  StepArgs sa = {};
  sa.H = c.H;
  sa.ldh = c.n + 1;
  sa.K = c.K;
  sa.ldk = c.n + 1;
  sa.R = c.R;
  sa.ldr = c.n;
  sa.flags = SF_GIVENS | (c.vec == KC_F32 ? SF_FALLBACK : 0);
  sa.pyth_tol = c.vec == KC_F64 ? 0.0 : 64.0 * 5.9604644775390625e-08;
  kc_status s;
  for (int k = 0; k < c.n; k++) {
    sa.k = k;
    if ((s = launch_matvec_reduce(ctx, A, c.Q, c.ldq, c.qdt, k, c.w, c.v, m, c.vec, sa)) != KC_OK)
      return s;
    if (c.vec == KC_F32 &&
        (s = launch_fallback_norm(ctx, c.Q, c.ldq, c.qdt, k, c.w, m, sa)) != KC_OK) return s;
    if ((s = launch_dcgs2_update(ctx, c.Q, c.ldq, c.qdt, k, c.w, c.v, m, c.vec)) != KC_OK) return s;
  }
  sa.k = c.n;
  if ((s = launch_reduce(ctx, c.Q, c.ldq, c.qdt, c.n, c.w, nullptr, m, c.vec, EPI_STORE_C1, sa)) != KC_OK) return s;
  if ((s = launch_proj_reduce(ctx, c.Q, c.ldq, c.qdt, c.n, c.w, m, c.vec, sa)) != KC_OK) return s;
  if ((s = launch_gemv_sub(ctx, c.Q, c.ldq, c.qdt, c.n, c.w, m, c.vec, 1)) != KC_OK) return s;
  if ((s = launch_norm(ctx, c.w, nullptr, m, c.vec, NEPI_FINISH, sa)) != KC_OK) return s;
  // y = R^{-1} g and x += Q y
  timing_begin(ctx, KID_SMALL);
  k_tri_solve<<<1, 32, 0, ctx->stream>>>(c.R, c.n, ctx->scal);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_OTHER);
  if (c.qdt == KC_F64)
    k_x_update<double, double><<<grid1d(ctx, m), 256, 0, ctx->stream>>>((const double*)c.Q, c.ldq, (double*)x, m, ctx->scal);
  else if (c.qdt == KC_F32)
    k_x_update<float, float><<<grid1d(ctx, m), 256, 0, ctx->stream>>>((const float*)c.Q, c.ldq, (float*)x, m, ctx->scal);
  else
    k_x_update<__nv_bfloat16, float><<<grid1d(ctx, m), 256, 0, ctx->stream>>>((const __nv_bfloat16*)c.Q, c.ldq, (float*)x, m, ctx->scal);
  KC_LAUNCHED(ctx);
  if ((s = read_scalars(ctx)) != KC_OK) return s;
  const Scalars* h = ctx->scal_host;
  if (c.gram) {
    // loss of orthogonality of the basis that formed this cycle's correction: its n
    // columns (the cycle's finish normalises no column n), or the ncols built before an
    // early stop
    const int cols = h->stop ? h->ncols : c.n;
    if (cols >= 1) {
      if ((s = launch_gram(ctx, c.Q, c.ldq, c.qdt, m, cols, c.gram)) != KC_OK) return s;
      if ((s = launch_loo_from_gram(ctx, c.gram, cols, c.loo)) != KC_OK) return s;
    }
  }
  *ncols_out = h->ncols;
  *est_out = h->resid_est;
  *matvecs += (h->stop && h->ncols < c.n) ? h->ncols + 1 : c.n;
  *status = h->status;
  KC_CUDA(ctx, cudaMemsetAsync(&ctx->scal->status, 0, sizeof(int), ctx->stream));
  // the cycle is over: later kernels (the FP64 residual, the next cycle) must run
  KC_CUDA(ctx, cudaMemsetAsync(&ctx->scal->stop, 0, sizeof(int), ctx->stream));
  return KC_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace kc

using namespace kc;

extern "C" {

kc_status gmres_solve(kc_ctx* ctx, const kc_csr* A, const kc_csr* A32, const double* b,
                      double* x, const kc_gmres_opts* opts, kc_gmres_info* info) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  kc_status s = validate_csr(ctx, A);
  if (s != KC_OK) return s;
  if (!b || !x || !opts || !info) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  if (A->val_dtype != KC_F64) return fail(ctx, KC_ERR_INVALID_ARG, "A must have FP64 values");
  const int n = opts->restart;
  if (n < 1 || n + 1 > NMAX) return fail(ctx, KC_ERR_INVALID_ARG, "restart must be in [1, %d]", NMAX - 1);
  const int prec = opts->precision;
  if (prec < 0 || prec > 2) return fail(ctx, KC_ERR_INVALID_ARG, "precision must be 0, 1 or 2");
  if (opts->precond == KC_PREC_JACOBI) {
    // right Jacobi preconditioning: M = D^{-1} is linear, so flexible GMRES with it is
    // GMRES on A D^{-1}; the flexible solver stores the preconditioned basis it needs
    if (prec != 0)
      return fail(ctx, KC_ERR_INVALID_ARG, "the Jacobi preconditioner needs precision 0");
    return fgmres_solve(ctx, A, nullptr, 0, 0, b, x, opts, info);
  }
  if (opts->precond != KC_PREC_AUTO)
    return fail(ctx, KC_ERR_INVALID_ARG, "unknown preconditioner kind %d", opts->precond);
  if (prec > 0) {
    if ((s = validate_csr(ctx, A32)) != KC_OK) return s;
    if (A32->val_dtype != KC_F32 || A32->m != A->m)
      return fail(ctx, KC_ERR_INVALID_ARG, "A32 must be the FP32 copy of A");
  }
  if (((uintptr_t)b & 15) || ((uintptr_t)x & 15))
    return fail(ctx, KC_ERR_INVALID_ARG, "b and x must be 16-byte aligned");
  memset(info, 0, sizeof(*info));
  info->max_loo = -1.0;
  const int64_t m = A->m;
  const int64_t ldq = (m + 31) / 32 * 32;
  const int qdt = prec == 0 ? KC_F64 : (prec == 1 ? KC_F32 : KC_BF16);
  const size_t qel = qdt == KC_F64 ? 8 : (qdt == KC_F32 ? 4 : 2);
  const size_t vel = prec == 0 ? 8 : 4;
  // workspace layout
  size_t off = 0;
  const size_t oQ = off; off = align256(off + (size_t)(n + 1) * ldq * qel);
  const size_t ow = off; off = align256(off + (size_t)ldq * vel);
  const size_t ov = off; off = align256(off + (size_t)ldq * vel);
  const size_t oH = off; off = align256(off + (size_t)(n + 1) * n * 8);
  const size_t oK = off; off = align256(off + (size_t)(n + 1) * n * 8);
  const size_t oR = off; off = align256(off + (size_t)n * n * 8);
  const size_t or64 = off; off = align256(off + (size_t)ldq * 8);
  const size_t ov64 = off; off = align256(off + (size_t)ldq * 8);
  const size_t od = off; off = align256(off + (size_t)ldq * 4);
  const size_t orhs = off; off = align256(off + (size_t)ldq * 4);
  const size_t oout = off; off = align256(off + 8 * sizeof(double));
  const size_t ogram = off; off = align256(off + (size_t)(n + 1) * (n + 1) * 8 + 2 * 8);
  const size_t ogrid = off; off = align256(off + gmres_grid_workspace(ctx));
  if ((s = ensure_workspace(ctx, off)) != KC_OK) return s;
  char* ws = (char*)ctx->ws;
  Cycle c;
  c.Q = ws + oQ; c.ldq = ldq; c.qdt = qdt; c.vec = prec == 0 ? KC_F64 : KC_F32;
  c.w = ws + ow; c.v = ws + ov; c.H = (double*)(ws + oH); c.K = (double*)(ws + oK);
  c.R = (double*)(ws + oR); c.n = n;
  c.gram = opts->diag_loo ? (double*)(ws + ogram) : nullptr;
  c.loo = opts->diag_loo ? (double*)(ws + ogram) + (size_t)(n + 1) * (n + 1) : nullptr;
  if (c.loo) KC_CUDA(ctx, cudaMemsetAsync(c.loo, 0, 2 * sizeof(double), ctx->stream));
  double* r64 = (double*)(ws + or64);
  double* v64 = (double*)(ws + ov64);
  float* d32 = (float*)(ws + od);
  float* rhs32 = (float*)(ws + orhs);
  KC_CUDA(ctx, cudaMemsetAsync(c.H, 0, (size_t)(n + 1) * n * 8, ctx->stream));
  KC_CUDA(ctx, cudaMemsetAsync(c.K, 0, (size_t)(n + 1) * n * 8, ctx->stream));

  // small FP64 problems: the whole solve in one launch (one cluster, or the whole grid)
  const int path = (prec != 0 || opts->diag_loo) ? 1 : (ctx->gmres_path != 0 ? ctx->gmres_path
                                    : (gmres_grid_preferred(ctx, m, n) ? 3 : 1));
  if (path >= 2) {
    double out[7];
    if ((s = gmres_fused_solve(ctx, path == 3, A, b, x, (double*)c.Q, ldq, (double*)c.w,
                               (double*)c.v, c.H, c.K, c.R, n, opts->maxit, opts->rtol,
                               ws + ogrid, (double*)(ws + oout), out)) != KC_OK)
      return s;
    const double bn = out[4];
    info->iters = (int)out[0];
    info->restarts = (int)out[1];
    info->outer = 0;
    info->rel_resid_est = bn > 0.0 ? out[2] / bn : 0.0;
    info->rel_resid_true = bn > 0.0 ? out[3] / bn : 0.0;
    const kc_status result = (kc_status)(int)out[5], last = (kc_status)(int)out[6];
    info->status = result == KC_OK ? last : result;
    if (result != KC_OK)
      fail(ctx, result, "gmres_solve: %d matvecs, relative residual %.3e", info->iters,
           info->rel_resid_true);
    return result;
  }

  double bnorm;
  if ((s = host_norm(ctx, b, m, KC_F64, &bnorm)) != KC_OK) return s;
  if (!(bnorm > 0.0)) {
    KC_CUDA(ctx, cudaMemsetAsync(x, 0, m * 8, ctx->stream));
    info->rel_resid_true = 0.0;
    return KC_OK;
  }
  const double target = opts->rtol * bnorm;
  int matvecs = 0, cycles = 0, outer = 0, st = 0, last_status = KC_OK;
  double est = 0.0, rn = 0.0;
  const int g = grid1d(ctx, m);
  kc_status result = KC_ERR_NOT_CONVERGED;
  for (;;) {
    // FP64 residual r = b - A x
    if ((s = launch_spmv(ctx, A, x, v64, KC_F64)) != KC_OK) return s;
    timing_begin(ctx, KID_OTHER);
    k_sub<double><<<g, 256, 0, ctx->stream>>>(b, v64, r64, m);
    KC_LAUNCHED(ctx);
    if ((s = host_norm(ctx, r64, m, KC_F64, &rn)) != KC_OK) return s;
    if (rn <= target) { result = KC_OK; break; }
    if (matvecs >= opts->maxit) break;
    if (prec == 0) {
      KC_CUDA(ctx, cudaMemcpyAsync(c.w, r64, m * 8, cudaMemcpyDeviceToDevice, ctx->stream));
      int ncols;
      if ((s = gmres_cycle(ctx, A, c, x, target, &ncols, &est, &matvecs, &st)) != KC_OK) return s;
      cycles++;
      if (st != KC_OK && st != KC_ERR_BREAKDOWN) last_status = st;
    } else {
      if (outer >= opts->max_outer) break;
      // inner FP32 solve of A32 d = r / ||r|| from d = 0
      timing_begin(ctx, KID_OTHER);
      k_cast_scale<<<g, 256, 0, ctx->stream>>>(r64, 1.0 / rn, rhs32, m);
      KC_LAUNCHED(ctx);
      KC_CUDA(ctx, cudaMemsetAsync(d32, 0, m * 4, ctx->stream));
      KC_CUDA(ctx, cudaMemcpyAsync(c.w, rhs32, m * 4, cudaMemcpyDeviceToDevice, ctx->stream));
      for (int ic = 0; ic < opts->inner_max_cycles; ic++) {
        if (ic > 0) {   // inner residual rhs - A32 d
          if ((s = launch_spmv(ctx, A32, d32, c.v, KC_F32)) != KC_OK) return s;
          timing_begin(ctx, KID_OTHER);
          k_sub<float><<<g, 256, 0, ctx->stream>>>(rhs32, (const float*)c.v, (float*)c.w, m);
          KC_LAUNCHED(ctx);
        }
        int ncols;
        if ((s = gmres_cycle(ctx, A32, c, d32, opts->inner_rtol, &ncols, &est, &matvecs, &st)) != KC_OK)
          return s;
        cycles++;
        if (st != KC_OK && st != KC_ERR_BREAKDOWN) last_status = st;
        if (est <= opts->inner_rtol || matvecs >= opts->maxit) break;
      }
      timing_begin(ctx, KID_OTHER);
      k_add_scaled<<<g, 256, 0, ctx->stream>>>(x, rn, d32, m);
      KC_LAUNCHED(ctx);
      outer++;
    }
  }
  if (c.loo) {
    double lv[2];
    KC_CUDA(ctx, cudaMemcpyAsync(lv, c.loo, sizeof(lv), cudaMemcpyDeviceToHost, ctx->stream));
    KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    info->max_loo = lv[1];
  }
  info->iters = matvecs;
  info->restarts = cycles;
  info->outer = outer;
  info->rel_resid_est = prec == 0 ? est / bnorm : est;
  info->rel_resid_true = rn / bnorm;
  info->status = result == KC_OK ? (last_status == KC_OK ? KC_OK : last_status) : result;
  if (result != KC_OK) fail(ctx, result, "gmres_solve: %d matvecs, relative residual %.3e",
                            matvecs, rn / bnorm);
  return result;
}

}  // extern "C"
