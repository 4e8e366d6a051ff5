// Staged FP64 basis passes: one producer thread streams Q tiles (and the w, v tiles) from
// HBM into a ring of shared-memory stages with bulk asynchronous copies completed on
// mbarriers; eight consumer warps compute from shared memory.  This keeps up to
// NST x 40 KB per SM in flight independently of the consumers' registers, which the
// register-streaming kernels could not do once their FP64 work was offloaded.
//
// Work unit: a tile of TR = 512 rows; within a tile the basis columns come in chunks of
// CH = 8 (8 x 4 KB), the first chunk of a tile also carries w and v (2 x 4 KB).  Consumer
// thread t owns rows 2t, 2t+1 of the tile and keeps its partial sums in registers across
// the chunks; the last chunk writes q_k and the new w.  Every wait is bounded: on a timeout
// the kernel records KC_ERR_TIMEOUT, stops issuing copies and drains the ones in flight.
#include "kc_internal.cuh"
#include "kc_dfloat.cuh"
#include "kc_tma.cuh"

namespace kc {

constexpr int ST_TR = 512;                 // rows per tile
constexpr int ST_CH = 8;                   // basis columns per chunk
constexpr int ST_NST = 4;                  // stages in the ring
constexpr int ST_CONSUMERS = 256;          // 8 warps
constexpr int ST_THREADS = ST_CONSUMERS + 32;
constexpr int ST_STAGE_DOUBLES = (ST_CH + 2) * ST_TR;
constexpr size_t ST_SMEM = (size_t)ST_NST * ST_STAGE_DOUBLES * 8 + 2 * ST_NST * 8 + 16;

struct StagedCtl {
  int abort;
};

// DCGS2 update (Algorithm 4: normalisation and projection), FP64; OFF: Q C in float-float (offload mode).
template <bool OFF>
__global__ void __launch_bounds__(ST_THREADS, 1)
k_update_staged(double* __restrict__ Q, int64_t ldq, int k, double* __restrict__ w,
                const double* __restrict__ v, int64_t m, Scalars* __restrict__ sc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* stage = reinterpret_cast<double*>(smem_raw);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(
      smem_raw + (size_t)ST_NST * ST_STAGE_DOUBLES * 8);
  unsigned long long* empty = full + ST_NST;
  __shared__ double sC[NMAX], sT[NMAX + 1];
  __shared__ float cH[NMAX], cL[NMAX];
  __shared__ double s_scale;
  __shared__ int s_cok, s_abort;
  if (sc->stop) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < ST_NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], ST_CONSUMERS / 32);
    }
    fence_barrier_init();
    s_abort = 0;
  }
  for (int i = tid; i <= k; i += blockDim.x) {
    if (i < k) sC[i] = sc->C[i];
    sT[i] = sc->T[i];
  }
  __syncthreads();
  if (OFF) {
    if (tid == 0) {
      double cmax = 0.0;
      for (int i = 0; i < k; i++) cmax = fmax(cmax, fabs(sC[i]));
      int ex = 0;
      if (cmax > 0.0) frexp(cmax, &ex);
      s_scale = ldexp(1.0, ex);
      s_cok = 1;
    }
    __syncthreads();
    const double inv_scale = 1.0 / s_scale;
    for (int i = tid; i < k; i += blockDim.x) {
      float h, l;
      if (!split_df(sC[i] * inv_scale, h, l)) { h = 0.0f; l = 0.0f; if (sC[i] != 0.0) s_cok = 0; }
      cH[i] = h;
      cL[i] = l;
    }
    __syncthreads();
  }
  const int64_t ntiles = (m + ST_TR - 1) / ST_TR;
  const int nch = k > 0 ? (k + ST_CH - 1) / ST_CH : 1;
  if (tid >= ST_CONSUMERS) {
    // ---- producer (one thread) ----
    if (tid != ST_CONSUMERS) return;
    int s = 0;
    unsigned int pass = 0;
    int last_par[ST_NST];                      // parity of each stage's latest fill, -1: none
    for (int i = 0; i < ST_NST; i++) last_par[i] = -1;
    for (int64_t tile = blockIdx.x; tile < ntiles && !s_abort; tile += gridDim.x) {
      const int64_t r0 = tile * ST_TR;
      const int rows = (int)(m - r0 < ST_TR ? m - r0 : ST_TR);
      const unsigned int rbytes = (unsigned int)(rows & ~1) * 8u;   // even rows by bulk copy
      for (int c = 0; c < nch; c++) {
        if (!mbar_wait(&empty[s], pass ^ 1u, WAIT_LIMIT)) {
          s_abort = 1;
          atomicExch(&sc->status, (int)KC_ERR_TIMEOUT);
          break;
        }
        const int c0 = c * ST_CH;
        const int ncol = k - c0 < ST_CH ? (k - c0 > 0 ? k - c0 : 0) : ST_CH;
        double* st = stage + (size_t)s * ST_STAGE_DOUBLES;
        const unsigned int bytes = (unsigned int)ncol * rbytes + (c == 0 ? 2u * rbytes : 0u);
        if (bytes == 0) {
          mbar_arrive(&full[s]);                  // nothing to copy (tiny tail)
        } else {
          mbar_arrive_expect_tx(&full[s], bytes);
          for (int j = 0; j < ncol; j++)
            bulk_g2s(st + j * ST_TR, Q + (int64_t)(c0 + j) * ldq + r0, rbytes, &full[s]);
          if (c == 0) {
            bulk_g2s(st + ST_CH * ST_TR, w + r0, rbytes, &full[s]);
            bulk_g2s(st + (ST_CH + 1) * ST_TR, v + r0, rbytes, &full[s]);
          }
        }
        last_par[s] = (int)pass;
        if (++s == ST_NST) { s = 0; pass ^= 1u; }
      }
    }
    // drain: the latest fill of every stage has landed before this thread (and so the
    // CTA and its shared memory) goes away, even if the consumers gave up
    for (int i = 0; i < ST_NST; i++)
      if (last_par[i] >= 0) (void)mbar_wait(&full[i], (unsigned int)last_par[i], WAIT_LIMIT);
    return;
  }
  // ---- consumers ----
  const double inva = sc->inv_alpha, vsc = sc->vscale;
  const double scale = OFF ? s_scale : 1.0;
  const bool cok = OFF ? (s_cok != 0) : false;
  const int warp = tid >> 5, lane = tid & 31;
  int s = 0;
  unsigned int pass = 0;
  double* qk = Q + (int64_t)k * ldq;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * ST_TR;
    const int rows = (int)(m - r0 < ST_TR ? m - r0 : ST_TR);
    const int lr = 2 * tid;                    // local rows lr, lr+1
    double u64[2] = {0.0, 0.0}, wn[2] = {0.0, 0.0};
    float zh[2] = {0.f, 0.f}, zl[2] = {0.f, 0.f};
    bool ok = true;
    for (int c = 0; c < nch; c++) {
      if (!mbar_wait(&full[s], pass, WAIT_LIMIT)) {
        atomicExch(&sc->status, (int)KC_ERR_TIMEOUT);
        s_abort = 1;
        ok = false;
        break;
      }
      const double* st = stage + (size_t)s * ST_STAGE_DOUBLES;
      if (lr < (rows & ~1)) {
        if (c == 0) {
          const double2 wv = *reinterpret_cast<const double2*>(st + ST_CH * ST_TR + lr);
          const double2 vv = *reinterpret_cast<const double2*>(st + (ST_CH + 1) * ST_TR + lr);
          u64[0] = wv.x; u64[1] = wv.y;
          wn[0] = vv.x * vsc; wn[1] = vv.y * vsc;
        }
        const int c0 = c * ST_CH;
        const int ncol = k - c0 < ST_CH ? (k - c0 > 0 ? k - c0 : 0) : ST_CH;
        for (int j = 0; j < ncol; j++) {
          const double2 q = *reinterpret_cast<const double2*>(st + j * ST_TR + lr);
          const int col = c0 + j;
          wn[0] = fma(-q.x, sT[col], wn[0]);
          wn[1] = fma(-q.y, sT[col], wn[1]);
          if (OFF) {
            float h0, l0, h1, l1;
            const bool okc = split_df(q.x, h0, l0) & split_df(q.y, h1, l1) & cok;
            if (__all_sync(__activemask(), okc)) {     // warp-uniform: no predicated DFMA
              df_mac(zh[0], zl[0], h0, l0, cH[col], cL[col]);
              df_mac(zh[1], zl[1], h1, l1, cH[col], cL[col]);
            } else {
              u64[0] = fma(-q.x, sC[col], u64[0]);
              u64[1] = fma(-q.y, sC[col], u64[1]);
            }
          } else {
            u64[0] = fma(-q.x, sC[col], u64[0]);
            u64[1] = fma(-q.y, sC[col], u64[1]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (++s == ST_NST) { s = 0; pass ^= 1u; }
    }
    if (!ok) break;
    if (lr < (rows & ~1)) {
      double qn[2], wo[2];
#pragma unroll
      for (int r = 0; r < 2; r++) {
        double u = u64[r];
        if (OFF) u = fma(-f2d_bits(zh[r]), scale, fma(-f2d_bits(zl[r]), scale, u));
        qn[r] = u * inva;
        wo[r] = fma(-qn[r], sT[k], wn[r]);
      }
      *reinterpret_cast<double2*>(qk + r0 + lr) = make_double2(qn[0], qn[1]);
      *reinterpret_cast<double2*>(w + r0 + lr) = make_double2(wo[0], wo[1]);
    } else if ((rows & 1) && lr == (rows & ~1)) {     // the odd last row of the last tile
      const int64_t row = r0 + lr;
      double u = __ldcg(w + row), wn1 = __ldcg(v + row) * vsc;
      for (int i = 0; i < k; i++) {
        const double q = __ldcg(Q + (int64_t)i * ldq + row);
        u = fma(-q, sC[i], u);
        wn1 = fma(-q, sT[i], wn1);
      }
      const double qn1 = u * inva;
      qk[row] = qn1;
      w[row] = fma(-qn1, sT[k], wn1);
    }
    (void)warp;
  }
}

kc_status launch_update_staged(kc_ctx* ctx, double* Q, int64_t ldq, int k, double* w,
                               const double* v, int64_t m) {
  static std::atomic<unsigned long long> attr_done[2];
  const int off = ctx->fp64_mode >= 1 ? 1 : 0;
  if (off) KC_TRY(smem_attr_once(ctx, attr_done[1], k_update_staged<true>, (int)ST_SMEM, "staged update"));
  else KC_TRY(smem_attr_once(ctx, attr_done[0], k_update_staged<false>, (int)ST_SMEM, "staged update"));
  const int64_t ntiles = (m + ST_TR - 1) / ST_TR;
  const int grid = (int)(ntiles < ctx->num_sms ? ntiles : ctx->num_sms);
  timing_begin(ctx, KID_UPDATE);
  if (off)
    k_update_staged<true><<<grid, ST_THREADS, ST_SMEM, ctx->stream>>>(Q, ldq, k, w, v, m, ctx->scal);
  else
    k_update_staged<false><<<grid, ST_THREADS, ST_SMEM, ctx->stream>>>(Q, ldq, k, w, v, m, ctx->scal);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

}  // namespace kc
