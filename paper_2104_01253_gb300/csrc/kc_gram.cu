// Gram matrix of a tall-skinny basis, G = Q^T Q in FP64, and the loss of orthogonality
// ||I - Q^T Q||_F derived from it (the stability metric of Section 6.1).  A diagnostic:
// gmres_solve uses it to report the worst loss of orthogonality over its (inner) cycles
// when kc_gmres_opts.diag_loo is set, and kc_basis_gram exposes it to callers.
//
// One CTA per row tile group: a tile of GRAM_ROWS rows of every column is staged in shared
// memory as FP64 (FP32 and BF16 entries convert exactly), then each thread accumulates up
// to GRAM_PPT of the ncols (ncols + 1) / 2 column pairs over the tile; blockIdx.y picks
// the chunk of pairs.  The per-CTA sums are added into the upper triangle of G with FP64
// atomics (the order of those additions is not fixed: G is a measurement, not part of
// the method), and a second launch mirrors it into the lower triangle.
#include "kc_internal.cuh"

namespace kc {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_ROWS = 32;
constexpr int GRAM_PPT = 8;                        // pairs per thread
constexpr int GRAM_PAIRS = GRAM_THREADS * GRAM_PPT;

template <typename T> __device__ __forceinline__ double gval(const T* p, int64_t i);
template <> __device__ __forceinline__ double gval(const double* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ double gval(const float* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ double gval(const __nv_bfloat16* p, int64_t i) {
  return __uint_as_float(((unsigned int)reinterpret_cast<const unsigned short*>(p)[i]) << 16);
}

// pair index p -> (i, j), i <= j, row-major over the upper triangle
__device__ __forceinline__ void pair_of(int p, int n, int& i, int& j) {
  int r = 0, base = 0;
  while (base + (n - r) <= p) { base += n - r; r++; }
  i = r;
  j = r + (p - base);
}

template <typename TQ>
__global__ void __launch_bounds__(GRAM_THREADS)
k_gram(const TQ* __restrict__ Q, int64_t ldq, int64_t m, int ncols, double* __restrict__ G) {
  extern __shared__ double tile[];                 // ncols x (GRAM_ROWS + 1)
  const int npairs = ncols * (ncols + 1) / 2;
  int pi[GRAM_PPT], pj[GRAM_PPT];
  double acc[GRAM_PPT];
#pragma unroll
  for (int s = 0; s < GRAM_PPT; s++) {
    const int p = blockIdx.y * GRAM_PAIRS + s * GRAM_THREADS + threadIdx.x;
    if (p < npairs) pair_of(p, ncols, pi[s], pj[s]);
    else { pi[s] = -1; pj[s] = -1; }
    acc[s] = 0.0;
  }
  constexpr int LD = GRAM_ROWS + 1;
  const int64_t ntiles = (m + GRAM_ROWS - 1) / GRAM_ROWS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * GRAM_ROWS;
    __syncthreads();
    for (int e = threadIdx.x; e < ncols * GRAM_ROWS; e += GRAM_THREADS) {
      const int c = e / GRAM_ROWS, r = e % GRAM_ROWS;
      const int64_t row = r0 + r;
      tile[c * LD + r] = row < m ? gval(Q + (int64_t)c * ldq, row) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < GRAM_PPT; s++) {
      if (pi[s] < 0) continue;
      const double* a = tile + pi[s] * LD;
      const double* b = tile + pj[s] * LD;
      double sum = acc[s];
#pragma unroll 8
      for (int r = 0; r < GRAM_ROWS; r++) sum = fma(a[r], b[r], sum);
      acc[s] = sum;
    }
  }
#pragma unroll
  for (int s = 0; s < GRAM_PPT; s++)
    if (pi[s] >= 0) atomicAdd(G + pi[s] + (int64_t)pj[s] * ncols, acc[s]);   // upper triangle
}

// G(j, i) = G(i, j) for i < j: the lower triangle mirrors the accumulated upper one
__global__ void k_gram_mirror(double* __restrict__ G, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e % n, j = e / n;
    if (i > j) G[e] = G[j + (int64_t)i * n];
  }
}

// out[0] = ||I - G||_F; out[1] = max(out[1], out[0]) (NaN if either is NaN)
__global__ void k_loo_from_gram(const double* __restrict__ G, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const double d = (i == j ? 1.0 : 0.0) - G[e];
    s += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    out[0] = sqrt(t);
    if (!isnan(out[1]) && !(out[0] <= out[1])) out[1] = out[0];   // a NaN stays
  }
}

kc_status launch_gram(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int64_t m,
                      int ncols, double* G) {
  if (ncols < 1 || ncols > NMAX || m < 1 || ldq < m)
    return fail(ctx, KC_ERR_INVALID_ARG, "gram: need 1 <= ncols <= %d, m >= 1, ldq >= m", NMAX);
  KC_CUDA(ctx, cudaMemsetAsync(G, 0, (size_t)ncols * ncols * sizeof(double), ctx->stream));
  // at most 128 x 33 doubles (33 KB): within the default dynamic shared-memory limit
  const size_t smem = (size_t)ncols * (GRAM_ROWS + 1) * sizeof(double);
  const int npairs = ncols * (ncols + 1) / 2;
  const int64_t ntiles = (m + GRAM_ROWS - 1) / GRAM_ROWS;
  int64_t gx = (int64_t)ctx->num_sms * 4;
  if (gx > ntiles) gx = ntiles;
  const dim3 grid((unsigned int)gx, (unsigned int)((npairs + GRAM_PAIRS - 1) / GRAM_PAIRS));
  timing_begin(ctx, KID_OTHER);
  if (q_dtype == KC_F64) {
    k_gram<double><<<grid, GRAM_THREADS, smem, ctx->stream>>>((const double*)Q, ldq, m, ncols, G);
  } else if (q_dtype == KC_F32) {
    k_gram<float><<<grid, GRAM_THREADS, smem, ctx->stream>>>((const float*)Q, ldq, m, ncols, G);
  } else if (q_dtype == KC_BF16) {
    k_gram<__nv_bfloat16><<<grid, GRAM_THREADS, smem, ctx->stream>>>(
        (const __nv_bfloat16*)Q, ldq, m, ncols, G);
  } else {
    return fail(ctx, KC_ERR_INVALID_ARG, "gram: unknown basis type %d", q_dtype);
  }
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_SMALL);
  k_gram_mirror<<<(ncols * ncols + 255) / 256, 256, 0, ctx->stream>>>(G, ncols);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_loo_from_gram(kc_ctx* ctx, const double* G, int ncols, double* out) {
  timing_begin(ctx, KID_SMALL);
  k_loo_from_gram<<<1, 256, 0, ctx->stream>>>(G, ncols, out);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

}  // namespace kc

extern "C" kc_status kc_basis_gram(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype,
                                   int64_t m, int ncols, double* G) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  if (!Q || !G) return kc::fail(ctx, KC_ERR_INVALID_ARG, "kc_basis_gram: NULL argument");
  return kc::launch_gram(ctx, Q, ldq, q_dtype, m, ncols, G);
}
