// C-ABI entry points of the convolutional preconditioner (forward, one training step) and
// flexible GMRES with it as the right preconditioner.
//
// Flexible DCGS2 (an addition: the paper's DCGS2 applies the matvec to the unnormalised
// pending vector w, which needs a linear operator).  With a preconditioner M the step
// works on zhat_k = M(w_k): v = A zhat_k, the same single reduction, alpha, T and q as
// Algorithm 4, and z_k = zhat_k / alpha_k.  Then A z_k = v / alpha_k = w_{k+1} + Q_{k+1} T,
// so column k of H is T + C_{k+1}, with no H C / alpha correction (the flexible flag of
// the scalar step), and the solution update is x += Z y.
#include "kc_internal.cuh"

#include <vector>

namespace kc {

typedef __nv_bfloat16 bf16;

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

static kc_status ensure_cnn_workspace(kc_ctx* ctx, size_t bytes) {
  if (ctx->cnn_ws_len >= bytes) return KC_OK;
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->cnn_ws) cudaFree(ctx->cnn_ws);
  ctx->cnn_ws = nullptr;
  ctx->cnn_ws_len = 0;
  if (cudaMalloc(&ctx->cnn_ws, bytes) != cudaSuccess)
    return fail(ctx, KC_ERR_OOM, "could not allocate %zu bytes of network workspace", bytes);
  ctx->cnn_ws_len = bytes;
  return KC_OK;
}

struct CnnBufs {
  bf16* wf;
  bf16* wt;
  bf16* acts[5];
  bf16* dz[2];
  float* g;
  float* dw;
  double* sums;
  float* res;
};

// Carve the network workspace for B images of H x W (`train`: keep all activations).
static kc_status cnn_bufs(kc_ctx* ctx, int B, int H, int W, bool train, CnnBufs* cb) {
  const size_t n = (size_t)B * H * W;
  size_t off = 0;
  const size_t o_wf = off; off = al256(off + cnn_nparam() * 2);
  const size_t o_wt = off; off = al256(off + 4 * 9216 * 2);
  size_t o_act[5];
  const int nact = train ? 5 : 2;
  for (int i = 0; i < nact; i++) { o_act[i] = off; off = al256(off + n * 32 * 2); }
  size_t o_dz[2] = {0, 0}, o_g = 0, o_dw = 0, o_s = 0, o_res = 0;
  if (train) {
    for (int i = 0; i < 2; i++) { o_dz[i] = off; off = al256(off + n * 32 * 2); }
    o_g = off; off = al256(off + n * 4);
    o_dw = off; off = al256(off + cnn_nparam() * 4);
    o_s = off; off = al256(off + 2 * (size_t)B * 8);
    o_res = off; off = al256(off + n * 4);
  }
  kc_status s = ensure_cnn_workspace(ctx, off);
  if (s != KC_OK) return s;
  char* p = (char*)ctx->cnn_ws;
  cb->wf = (bf16*)(p + o_wf);
  cb->wt = (bf16*)(p + o_wt);
  for (int i = 0; i < 5; i++) cb->acts[i] = i < nact ? (bf16*)(p + o_act[i]) : nullptr;
  cb->dz[0] = train ? (bf16*)(p + o_dz[0]) : nullptr;
  cb->dz[1] = train ? (bf16*)(p + o_dz[1]) : nullptr;
  cb->g = train ? (float*)(p + o_g) : nullptr;
  cb->dw = train ? (float*)(p + o_dw) : nullptr;
  cb->sums = train ? (double*)(p + o_s) : nullptr;
  cb->res = train ? (float*)(p + o_res) : nullptr;
  return KC_OK;
}

static kc_status check_grid(kc_ctx* ctx, int B, int H, int W) {
  if (B < 1 || H < 1 || W < 1 || (int64_t)B * H * W >= ((int64_t)1 << 31))
    return fail(ctx, KC_ERR_INVALID_ARG, "bad network input shape %d x %d x %d", B, H, W);
  return KC_OK;
}

// ---- FGMRES helpers ------------------------------------------------------------------------

// dinv_i = 1 / a_ii (1 where row i stores no diagonal entry or a zero one)
__global__ void __launch_bounds__(256)
k_fgm_dinv(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
           const double* __restrict__ av, double* __restrict__ dinv, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; p++)
      if (ci[p] == i) d = av[p];
    dinv[i] = d != 0.0 ? 1.0 / d : 1.0;
  }
}

// u = D^{-1} w
__global__ void __launch_bounds__(256)
k_fgm_jacobi(const double* __restrict__ w, const double* __restrict__ dinv,
             double* __restrict__ u, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] = w[i] * dinv[i];
}

// u = D^{-1} w and sc->norm_sq = u^T u in one pass (the input scale of the network): CTA
// sums written in CTA order, added by the last CTA in a fixed order (lane-strided, then a
// warp tree), so the result is deterministic; the ticket counter is reset for the next call
__global__ void __launch_bounds__(256)
k_fgm_jacobi_sq(const double* __restrict__ w, const double* __restrict__ dinv,
                double* __restrict__ u, int64_t m, double* __restrict__ partials,
                unsigned int* __restrict__ counter, Scalars* __restrict__ sc) {
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[i] * dinv[i];
    u[i] = v;
    a = fma(v, v, a);
  }
  __shared__ double red[8];
  __shared__ unsigned int ticket;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if (lane == 0) red[warp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    partials[blockIdx.x] = t;
    __threadfence();
    ticket = atomicAdd(counter, 1u);
  }
  __syncthreads();
  if (ticket != gridDim.x - 1 || warp != 0) return;
  __threadfence();
  double t = 0.0;
  for (int i = lane; i < (int)gridDim.x; i += 32) t += __ldcg(partials + i);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) {
    sc->norm_sq = t;
    *counter = 0u;
  }
}

// network input: w / rms(w) in FP32 (rms from the norm kernel's sum of squares; the square
// root and reciprocal once per CTA: per thread they cost more FP64 work than the pass)
__global__ void k_fgm_prep(const double* __restrict__ w, float* __restrict__ x, int64_t m,
                           const Scalars* __restrict__ sc) {
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    const double rms = sqrt(sc->norm_sq / (double)m);
    s_inv = rms > 0.0 ? 1.0 / rms : 0.0;
  }
  __syncthreads();
  const double inv = s_inv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (float)(w[i] * inv);
}

// zhat = w + rms(w) * net(w / rms(w)), called with w = u = D^{-1} w: the Jacobi step plus
// the learned correction
__global__ void k_fgm_post(const float* __restrict__ y, const double* __restrict__ w,
                           double* __restrict__ z, int64_t m, const Scalars* __restrict__ sc) {
  __shared__ double s_rms;
  if (threadIdx.x == 0) s_rms = sqrt(sc->norm_sq / (double)m);
  __syncthreads();
  const double rms = s_rms;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = w[i] + (double)y[i] * rms;
}

// y <- R^{-1} g, then y_j <- y_j / alpha_j (so that x += Zhat y)
__global__ void k_fgm_solve(const double* __restrict__ R, int ldr, Scalars* sc) {
  if (threadIdx.x != 0) return;
  const int n = sc->ncols;
  for (int i = n - 1; i >= 0; i--) {
    double t = sc->g[i];
    for (int j = i + 1; j < n; j++) t -= R[i + (int64_t)j * ldr] * sc->y[j];
    sc->y[i] = t / R[i + (int64_t)i * ldr];
  }
  for (int i = 0; i < n; i++) sc->y[i] *= sc->zscale[i];
}

__global__ void __launch_bounds__(256)
k_fgm_xupdate(const double* __restrict__ Z, int64_t ldz, double* __restrict__ x, int64_t m,
              const Scalars* __restrict__ sc) {
  __shared__ double y[NMAX];
  const int n = sc->ncols;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = sc->y[i];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; j++) s += Z[r + (int64_t)j * ldz] * y[j];
    x[r] += s;
  }
}

__global__ void k_fgm_begin(Scalars* sc, double rtol_abs) {
  sc->stop = 0;
  sc->ncols = 0;
  sc->fallback = 0;
  sc->rtol_abs = rtol_abs;
  sc->resid_est = 0.0;
}

__global__ void __launch_bounds__(256) k_fgm_sub(const double* __restrict__ b,
                                                 const double* __restrict__ Av,
                                                 double* __restrict__ r, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - Av[i];
}

static int g1d(const kc_ctx* ctx, int64_t m) {
  int64_t b = (m + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

static kc_status host_norm64(kc_ctx* ctx, const double* x, int64_t m, double* out,
                             int nepi = NEPI_INIT) {
  StepArgs sa = {};
  kc_status s = launch_norm(ctx, x, nullptr, m, KC_F64, nepi, sa);
  if (s != KC_OK) return s;
  KC_CUDA(ctx, cudaMemcpyAsync(&ctx->scal_host->norm_sq, &ctx->scal->norm_sq, sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *out = sqrt(ctx->scal_host->norm_sq);
  return KC_OK;
}

}  // namespace kc

using namespace kc;

extern "C" {

int64_t kc_cnn_param_count(void) { return cnn_nparam(); }

kc_status kc_cnn_forward(kc_ctx* ctx, const float* w32, const float* x, float* y, int B, int H,
                         int W) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  if (!w32 || !x || !y) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  kc_status s = check_grid(ctx, B, H, W);
  if (s != KC_OK) return s;
  CnnBufs cb;
  if ((s = cnn_bufs(ctx, B, H, W, false, &cb)) != KC_OK) return s;
  if ((s = cnn_prep(ctx, w32, cb.wf, cb.wt)) != KC_OK) return s;
  return cnn_forward(ctx, cb.wf, x, y, cb.acts, false, B, H, W);
}

}  // extern "C"

// One training step: forward, loss and dL/dy, backward, Adam (t > 0).  A == nullptr:
// regression loss against the targets e; otherwise the residual loss with r = e.
static kc_status train_step(kc_ctx* ctx, float* w32, float* adam_m, float* adam_v, int64_t t,
                            float lr, const kc_csr* A, const float* x, const float* e, int B,
                            int H, int W, float* y, float* grad, double* loss) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  if (!w32 || !x || !e || !y || (t > 0 && (!adam_m || !adam_v)))
    return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  kc_status s = check_grid(ctx, B, H, W);
  if (s != KC_OK) return s;
  const int64_t npix = (int64_t)H * W;
  if (A) {
    if ((s = validate_csr_entries(ctx, A)) != KC_OK) return s;
    if (A->val_dtype != KC_F64) return fail(ctx, KC_ERR_INVALID_ARG, "A must have FP64 values");
    if (A->m != npix)
      return fail(ctx, KC_ERR_INVALID_ARG, "grid %d x %d does not match m = %lld", H, W,
                  (long long)A->m);
  }
  CnnBufs cb;
  if ((s = cnn_bufs(ctx, B, H, W, true, &cb)) != KC_OK) return s;
  if ((s = cnn_prep(ctx, w32, cb.wf, cb.wt)) != KC_OK) return s;
  if ((s = cnn_forward(ctx, cb.wf, x, y, cb.acts, true, B, H, W)) != KC_OK) return s;
  if (A)
    s = cnn_residual_loss_grad(ctx, A, x, y, e, cb.res, cb.sums, cb.g, B, npix);
  else
    s = cnn_loss_grad(ctx, y, e, cb.sums, cb.g, B, npix);
  if (s != KC_OK) return s;
  KC_CUDA(ctx, cudaMemsetAsync(cb.dw, 0, cnn_nparam() * sizeof(float), ctx->stream));
  if ((s = cnn_backward(ctx, cb.wf, cb.wt, x, cb.g, cb.acts, cb.dz, cb.dw, B, H, W)) != KC_OK)
    return s;
  if (grad)
    KC_CUDA(ctx, cudaMemcpyAsync(grad, cb.dw, cnn_nparam() * sizeof(float),
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  if (t > 0 && (s = cnn_adam(ctx, w32, cb.dw, adam_m, adam_v, t, lr, 0.9f, 0.999f, 1e-8f)) != KC_OK)
    return s;
  if (loss) {
    std::vector<double> hs(2 * (size_t)B);
    KC_CUDA(ctx, cudaMemcpyAsync(hs.data(), cb.sums, 2 * (size_t)B * sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double L = 0.0;
    for (int b = 0; b < B; b++) L += hs[2 * b] / hs[2 * b + 1];
    *loss = L / B;
  }
  return KC_OK;
}

extern "C" {

kc_status kc_cnn_train_step(kc_ctx* ctx, float* w32, float* adam_m, float* adam_v, int64_t t,
                            float lr, const float* x, const float* e, int B, int H, int W,
                            float* y, float* grad, double* loss) {
  return train_step(ctx, w32, adam_m, adam_v, t, lr, nullptr, x, e, B, H, W, y, grad, loss);
}

kc_status kc_cnn_train_step_residual(kc_ctx* ctx, float* w32, float* adam_m, float* adam_v,
                                     int64_t t, float lr, const kc_csr* A, const float* x,
                                     const float* r, int B, int H, int W, float* y, float* grad,
                                     double* loss) {
  if (ctx && !A) return fail(ctx, KC_ERR_INVALID_ARG, "NULL operator");
  return train_step(ctx, w32, adam_m, adam_v, t, lr, A, x, r, B, H, W, y, grad, loss);
}

kc_status kc_cnn_residual_sample(kc_ctx* ctx, const kc_csr* A, const double* b,
                                 const double* x, float* xin, float* res, double* rnorm) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  kc_status s = validate_csr_entries(ctx, A);
  if (s != KC_OK) return s;
  if (!b || !x || !xin || !res || !rnorm) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  if (A->val_dtype != KC_F64) return fail(ctx, KC_ERR_INVALID_ARG, "A must have FP64 values");
  if (((uintptr_t)b & 15) || ((uintptr_t)x & 15))
    return fail(ctx, KC_ERR_INVALID_ARG, "b and x must be 16-byte aligned");
  const int64_t m = A->m;
  const int64_t ld = (m + 31) / 32 * 32;
  if ((s = ensure_workspace(ctx, 4 * (size_t)ld * 8)) != KC_OK) return s;
  double* v = (double*)ctx->ws;
  double* r = v + ld;
  double* dinv = r + ld;
  double* u = dinv + ld;
  const int g = g1d(ctx, m);
  if ((s = launch_spmv(ctx, A, x, v, KC_F64)) != KC_OK) return s;
  timing_begin(ctx, KID_OTHER);
  k_fgm_sub<<<g, 256, 0, ctx->stream>>>(b, v, r, m);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_OTHER);
  k_fgm_dinv<<<g, 256, 0, ctx->stream>>>(A->row_ptr, A->col_idx, (const double*)A->val, dinv, m);
  KC_LAUNCHED(ctx);
  if ((s = host_norm64(ctx, r, m, rnorm, NEPI_SQ)) != KC_OK) return s;   // r = 0 is no error
  // norm_sq = u^T u, then both outputs are divided by s = sqrt(norm_sq / m)
  timing_begin(ctx, KID_OTHER);
  k_fgm_jacobi_sq<<<g, 256, 0, ctx->stream>>>(r, dinv, u, m, ctx->partials, ctx->counters + 3,
                                               ctx->scal);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_OTHER);
  k_fgm_prep<<<g, 256, 0, ctx->stream>>>(u, xin, m, ctx->scal);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_OTHER);
  k_fgm_prep<<<g, 256, 0, ctx->stream>>>(r, res, m, ctx->scal);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status fgmres_solve(kc_ctx* ctx, const kc_csr* A, const float* w32, int H, int W,
                       const double* b, double* x, const kc_gmres_opts* opts,
                       kc_gmres_info* info) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  kc_status s = validate_csr_entries(ctx, A);
  if (s != KC_OK) return s;
  if (!b || !x || !opts || !info) return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  if (A->val_dtype != KC_F64) return fail(ctx, KC_ERR_INVALID_ARG, "A must have FP64 values");
  if (opts->precond != KC_PREC_AUTO && opts->precond != KC_PREC_JACOBI)
    return fail(ctx, KC_ERR_INVALID_ARG, "unknown preconditioner kind %d", opts->precond);
  const bool use_net = w32 && opts->precond == KC_PREC_AUTO;
  const bool use_jacobi = use_net || opts->precond == KC_PREC_JACOBI;
  if (use_net && (int64_t)H * W != A->m)
    return fail(ctx, KC_ERR_INVALID_ARG, "grid %d x %d does not match m = %lld", H, W,
                (long long)A->m);
  const int n = opts->restart;
  if (n < 1 || n + 1 > NMAX) return fail(ctx, KC_ERR_INVALID_ARG, "restart must be in [1, %d]", NMAX - 1);
  if (((uintptr_t)b & 15) || ((uintptr_t)x & 15))
    return fail(ctx, KC_ERR_INVALID_ARG, "b and x must be 16-byte aligned");
  memset(info, 0, sizeof(*info));
  info->max_loo = -1.0;
  const int64_t m = A->m;
  const int64_t ld = (m + 31) / 32 * 32;
  size_t off = 0;
  const size_t oQ = off; off = al256(off + (size_t)(n + 1) * ld * 8);
  const size_t oZ = off; off = al256(off + (size_t)n * ld * 8);
  const size_t ow = off; off = al256(off + (size_t)ld * 8);
  const size_t ov = off; off = al256(off + (size_t)ld * 8);
  const size_t oH = off; off = al256(off + (size_t)(n + 1) * n * 8);
  const size_t oK = off; off = al256(off + (size_t)(n + 1) * n * 8);
  const size_t oR = off; off = al256(off + (size_t)n * n * 8);
  const size_t oi = off; off = al256(off + (size_t)ld * 4);
  const size_t oo = off; off = al256(off + (size_t)ld * 4);
  const size_t od = off; off = al256(off + (size_t)ld * 8);
  const size_t ou = off; off = al256(off + (size_t)ld * 8);
  if ((s = ensure_workspace(ctx, off)) != KC_OK) return s;
  char* ws = (char*)ctx->ws;
  double* Q = (double*)(ws + oQ);
  double* Z = (double*)(ws + oZ);
  double* w = (double*)(ws + ow);
  double* v = (double*)(ws + ov);
  double* Hm = (double*)(ws + oH);
  double* Km = (double*)(ws + oK);
  double* R = (double*)(ws + oR);
  float* xin = (float*)(ws + oi);
  float* yout = (float*)(ws + oo);
  double* dinv = (double*)(ws + od);
  double* u = (double*)(ws + ou);
  CnnBufs cb = {};
  if (use_net) {
    if ((s = cnn_bufs(ctx, 1, H, W, false, &cb)) != KC_OK) return s;
    if ((s = cnn_prep(ctx, w32, cb.wf, cb.wt)) != KC_OK) return s;
  }
  KC_CUDA(ctx, cudaMemsetAsync(Hm, 0, (size_t)(n + 1) * n * 8, ctx->stream));
  KC_CUDA(ctx, cudaMemsetAsync(Km, 0, (size_t)(n + 1) * n * 8, ctx->stream));
  double bnorm;
  if ((s = host_norm64(ctx, b, m, &bnorm)) != KC_OK) return s;
  if (!(bnorm > 0.0)) {
    KC_CUDA(ctx, cudaMemsetAsync(x, 0, m * 8, ctx->stream));
    return KC_OK;
  }
  const double target = opts->rtol * bnorm;
  StepArgs sa = {};
  sa.H = Hm;
  sa.ldh = n + 1;
  sa.K = Km;
  sa.ldk = n + 1;
  sa.R = R;
  sa.ldr = n;
  sa.flags = SF_GIVENS | SF_FLEXIBLE;
  sa.pyth_tol = 0.0;
  const int g = g1d(ctx, m);
  if (use_jacobi) {
    timing_begin(ctx, KID_OTHER);
    k_fgm_dinv<<<g, 256, 0, ctx->stream>>>(A->row_ptr, A->col_idx, (const double*)A->val, dinv, m);
    KC_LAUNCHED(ctx);
  }
  int matvecs = 0, cycles = 0, last_status = KC_OK;
  double rn = 0.0, est = 0.0;
  kc_status result = KC_ERR_NOT_CONVERGED;
  for (;;) {
    if ((s = launch_spmv(ctx, A, x, v, KC_F64)) != KC_OK) return s;
    timing_begin(ctx, KID_OTHER);
    k_fgm_sub<<<g, 256, 0, ctx->stream>>>(b, v, w, m);
    KC_LAUNCHED(ctx);
    if ((s = host_norm64(ctx, w, m, &rn)) != KC_OK) return s;
    if (rn <= target) { result = KC_OK; break; }
    if (matvecs >= opts->maxit) break;
    timing_begin(ctx, KID_SMALL);
    k_fgm_begin<<<1, 1, 0, ctx->stream>>>(ctx->scal, target);
    KC_LAUNCHED(ctx);
    for (int k = 0; k < n; k++) {
      double* zk = Z + (size_t)k * ld;
      sa.k = k;
      if (use_net) {   // zhat = u + rms(u) net(u / rms(u)), u = D^{-1} w
        timing_begin(ctx, KID_OTHER);
        k_fgm_jacobi_sq<<<g, 256, 0, ctx->stream>>>(w, dinv, u, m, ctx->partials,
                                                     ctx->counters + 3, ctx->scal);
        KC_LAUNCHED(ctx);
        timing_begin(ctx, KID_OTHER);
        k_fgm_prep<<<g, 256, 0, ctx->stream>>>(u, xin, m, ctx->scal);
        KC_LAUNCHED(ctx);
        if ((s = cnn_forward(ctx, cb.wf, xin, yout, cb.acts, false, 1, H, W)) != KC_OK) return s;
        timing_begin(ctx, KID_OTHER);
        k_fgm_post<<<g, 256, 0, ctx->stream>>>(yout, u, zk, m, ctx->scal);
        KC_LAUNCHED(ctx);
      } else if (use_jacobi) {   // zhat = D^{-1} w
        timing_begin(ctx, KID_OTHER);
        k_fgm_jacobi<<<g, 256, 0, ctx->stream>>>(w, dinv, zk, m);
        KC_LAUNCHED(ctx);
      } else {         // identity: zhat = w
        KC_CUDA(ctx, cudaMemcpyAsync(zk, w, m * 8, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      if ((s = launch_spmv(ctx, A, zk, v, KC_F64)) != KC_OK) return s;
      if ((s = launch_reduce(ctx, Q, ld, KC_F64, k, w, v, m, KC_F64, EPI_DCGS2, sa)) != KC_OK) return s;
      if ((s = launch_dcgs2_update(ctx, Q, ld, KC_F64, k, w, v, m, KC_F64)) != KC_OK) return s;
    }
    sa.k = n;
    if ((s = launch_reduce(ctx, Q, ld, KC_F64, n, w, nullptr, m, KC_F64, EPI_STORE_C1, sa)) != KC_OK) return s;
    if ((s = launch_proj_reduce(ctx, Q, ld, KC_F64, n, w, m, KC_F64, sa)) != KC_OK) return s;
    if ((s = launch_gemv_sub(ctx, Q, ld, KC_F64, n, w, m, KC_F64, 1)) != KC_OK) return s;
    if ((s = launch_norm(ctx, w, nullptr, m, KC_F64, NEPI_FINISH, sa)) != KC_OK) return s;
    timing_begin(ctx, KID_SMALL);
    k_fgm_solve<<<1, 32, 0, ctx->stream>>>(R, n, ctx->scal);
    KC_LAUNCHED(ctx);
    timing_begin(ctx, KID_OTHER);
    k_fgm_xupdate<<<g, 256, 0, ctx->stream>>>(Z, ld, x, m, ctx->scal);
    KC_LAUNCHED(ctx);
    KC_CUDA(ctx, cudaMemcpyAsync(ctx->scal_host, ctx->scal, sizeof(Scalars),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const Scalars* h = ctx->scal_host;
    matvecs += (h->stop && h->ncols < n) ? h->ncols + 1 : n;
    est = h->resid_est;
    if (h->status != KC_OK && h->status != KC_ERR_BREAKDOWN) last_status = h->status;
    KC_CUDA(ctx, cudaMemsetAsync(&ctx->scal->status, 0, sizeof(int), ctx->stream));
    KC_CUDA(ctx, cudaMemsetAsync(&ctx->scal->stop, 0, sizeof(int), ctx->stream));
    cycles++;
  }
  info->iters = matvecs;
  info->restarts = cycles;
  info->rel_resid_est = est / bnorm;
  info->rel_resid_true = rn / bnorm;
  info->status = result == KC_OK ? last_status : result;
  if (result != KC_OK)
    fail(ctx, result, "fgmres_solve: %d matvecs, relative residual %.3e", matvecs, rn / bnorm);
  return result;
}

}  // extern "C"
