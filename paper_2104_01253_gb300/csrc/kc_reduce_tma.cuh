// TMA-staged fused DCGS2 reduction (the single reduction of Algorithm 4: C = Q^T w, S = Q^T v,
// beta = w^T w, s = w^T v, then the scalar step in the last CTA).
//
// One producer thread streams tiles of RT_TR rows: for every chunk of RT_CH basis columns
// one 2D tensor copy (cp.async.bulk.tensor) of an RT_TR x RT_CH box of Q, and with the
// first chunk of a tile two 1D tensor copies of the w and v rows, into a ring of RT_NST
// shared-memory stages completed on mbarriers.  Sixteen consumer warps compute from shared
// memory: warp (h, j) owns task j of every chunk (task c RT_CH + j: a column, beta or s)
// on row half h of the tile, and keeps its sums in registers across tiles.  The bytes in
// flight (RT_NST stages) no longer depend on registers, which bounded the register-streaming
// kernel once half of its FP64 work had moved to the FP32 pipes.  Rows and columns outside
// the tensors read as zero (tensor-copy fill), so there is no ragged-tail code.  Every wait
// is bounded: on a timeout the kernel records KC_ERR_TIMEOUT, stops issuing copies and
// drains the ones in flight before it exits.
//
// Included at the end of kc_ortho.cu (it uses that file's reduction epilogue).
#pragma once
#include <cuda.h>

#include "kc_internal.cuh"
#include "kc_dfloat.cuh"
#include "kc_tma.cuh"

namespace kc {

constexpr int RT_TR = 128;                  // rows per tile
constexpr int RT_CH = 8;                    // tasks per chunk
constexpr int RT_NST = 8;                   // ring stages
constexpr int RT_CW = 2 * RT_CH;            // consumer warps: RT_CH tasks x 2 row halves
constexpr int RT_THREADS = (RT_CW + 1) * 32;
constexpr int RT_STAGE_DOUBLES = (RT_CH + 2) * RT_TR;   // Q box, then w rows, then v rows
constexpr size_t RT_SMEM = 128 + (size_t)RT_NST * RT_STAGE_DOUBLES * 8 + 2 * RT_NST * 8;
static_assert(RT_TR % 128 == 0, "each row half must be whole pairs of rows for all 32 lanes");
static_assert(RT_TR <= 256 && RT_CH <= 256, "a tensor-copy box has at most 256 elements per dimension");

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y),
        "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, int x,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2}], [%3];\n"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x),
        "r"(smem_u32(bar))
      : "memory");
}

// OFF: S in float-float (FP64 with offload); !OFF: every product in FP64.
// MAXCH: compile-time bound on the number of chunks, ceil((k + 2) / RT_CH).
template <bool OFF, int MAXCH>
__global__ void __launch_bounds__(RT_THREADS, 1)
k_reduce_tma(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tx,
             const __grid_constant__ CUtensorMap ty, int k, int64_t m,
             double* __restrict__ partials, unsigned int* __restrict__ counter,
             Scalars* __restrict__ sc, StepArgs sa) {
  if (sc->stop) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  double* stage = reinterpret_cast<double*>(base);
  unsigned long long* full =
      reinterpret_cast<unsigned long long*>(base + (size_t)RT_NST * RT_STAGE_DOUBLES * 8);
  unsigned long long* empty = full + RT_NST;
  __shared__ double s_part[2][MAXCH][RT_CH][2];
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < RT_NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], RT_CW);
    }
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  const int ntask = k + 2;
  const int nch = (ntask + RT_CH - 1) / RT_CH;
  const int64_t ntiles = (m + RT_TR - 1) / RT_TR;

  if (warp == RT_CW) {
    // ---- producer (one thread) ----
    if (lane == 0) {
      int s = 0;
      unsigned int pass = 0;
      int last_par[RT_NST];
      for (int i = 0; i < RT_NST; i++) last_par[i] = -1;
      for (int64_t tile = blockIdx.x; tile < ntiles && !*(volatile int*)&s_abort;
           tile += gridDim.x) {
        const int r0 = (int)(tile * RT_TR);
        for (int c = 0; c < nch; c++) {
          if (!mbar_wait(&empty[s], pass ^ 1u, WAIT_LIMIT)) {
            s_abort = 1;
            atomicExch(&sc->status, (int)KC_ERR_TIMEOUT);
            break;
          }
          double* st = stage + (size_t)s * RT_STAGE_DOUBLES;
          const bool has_q = c * RT_CH < k;
          const unsigned int bytes = (has_q ? RT_TR * RT_CH * 8u : 0u) + (c == 0 ? 2u * RT_TR * 8u : 0u);
          if (bytes == 0) {
            mbar_arrive(&full[s]);              // a chunk of beta / s only, after the first
          } else {
            mbar_arrive_expect_tx(&full[s], bytes);
            if (has_q) tma_load_2d(st, &tq, r0, c * RT_CH, &full[s]);
            if (c == 0) {
              tma_load_1d(st + RT_CH * RT_TR, &tx, r0, &full[s]);
              tma_load_1d(st + (RT_CH + 1) * RT_TR, &ty, r0, &full[s]);
            }
          }
          last_par[s] = (int)pass;
          if (++s == RT_NST) { s = 0; pass ^= 1u; }
        }
      }
      // every copy issued has landed before the CTA (and its shared memory) goes away
      for (int i = 0; i < RT_NST; i++)
        if (last_par[i] >= 0) (void)mbar_wait(&full[i], (unsigned int)last_par[i], WAIT_LIMIT);
    }
  } else {
    // ---- consumers ----
    constexpr int RG = RT_TR / 128;                      // row pairs per lane (half: RT_TR / 2 rows)
    const int h = warp / RT_CH, j = warp % RT_CH;
    const int lr0 = h * (RT_TR / 2) + 2 * lane;          // rows lr0 + 64 g, + 1
    double ac[MAXCH], as64[MAXCH];
    float sh[MAXCH], sl[MAXCH];
#pragma unroll
    for (int c = 0; c < MAXCH; c++) { ac[c] = 0.0; as64[c] = 0.0; sh[c] = 0.0f; sl[c] = 0.0f; }
    int s = 0;
    unsigned int pass = 0;
    bool alive = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
      double xr[RG][2], yr[RG][2];
      float yh[RG][2], yl[RG][2];
      bool yok = true;
#pragma unroll
      for (int c = 0; c < MAXCH; c++) {
        if (c >= nch) break;
        if (!mbar_wait(&full[s], pass, WAIT_LIMIT)) {
          atomicExch(&sc->status, (int)KC_ERR_TIMEOUT);
          s_abort = 1;
          alive = false;
          break;
        }
        const double* st = stage + (size_t)s * RT_STAGE_DOUBLES;
        if (c == 0) {
#pragma unroll
          for (int g = 0; g < RG; g++) {
            const int lr = lr0 + 64 * g;
            const double2 xv = *reinterpret_cast<const double2*>(st + RT_CH * RT_TR + lr);
            const double2 yv = *reinterpret_cast<const double2*>(st + (RT_CH + 1) * RT_TR + lr);
            xr[g][0] = xv.x; xr[g][1] = xv.y; yr[g][0] = yv.x; yr[g][1] = yv.y;
            if (OFF) yok = yok & split_df(yr[g][0], yh[g][0], yl[g][0]) &
                           split_df(yr[g][1], yh[g][1], yl[g][1]);
          }
        }
        const int t = c * RT_CH + j;
        if (t < k) {
          double2 q[RG];
#pragma unroll
          for (int g = 0; g < RG; g++)
            q[g] = *reinterpret_cast<const double2*>(st + j * RT_TR + lr0 + 64 * g);
#pragma unroll
          for (int g = 0; g < RG; g++) {
            ac[c] = fma(q[g].x, xr[g][0], ac[c]);
            ac[c] = fma(q[g].y, xr[g][1], ac[c]);
          }
          if (OFF) {
            bool ok = yok;
#pragma unroll
            for (int g = 0; g < RG; g++) ok = ok & df_in_range(q[g].x) & df_in_range(q[g].y);
            if (__builtin_expect(__all_sync(0xffffffffu, ok), 1)) {
#pragma unroll
              for (int g = 0; g < RG; g++) {
                float qh[2], ql[2];
                split_df(q[g].x, qh[0], ql[0]);
                split_df(q[g].y, qh[1], ql[1]);
                df_mac(sh[c], sl[c], qh[0], ql[0], yh[g][0], yl[g][0]);
                df_mac(sh[c], sl[c], qh[1], ql[1], yh[g][1], yl[g][1]);
              }
            } else {
#pragma unroll
              for (int g = 0; g < RG; g++) {
                as64[c] = fma(q[g].x, yr[g][0], as64[c]);
                as64[c] = fma(q[g].y, yr[g][1], as64[c]);
              }
            }
          } else {
#pragma unroll
            for (int g = 0; g < RG; g++) {
              as64[c] = fma(q[g].x, yr[g][0], as64[c]);
              as64[c] = fma(q[g].y, yr[g][1], as64[c]);
            }
          }
        } else if (t == k) {                   // beta = w^T w
#pragma unroll
          for (int g = 0; g < RG; g++) {
            ac[c] = fma(xr[g][0], xr[g][0], ac[c]);
            ac[c] = fma(xr[g][1], xr[g][1], ac[c]);
          }
        } else if (t == k + 1) {               // s = w^T v
#pragma unroll
          for (int g = 0; g < RG; g++) {
            ac[c] = fma(xr[g][0], yr[g][0], ac[c]);
            ac[c] = fma(xr[g][1], yr[g][1], ac[c]);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == RT_NST) { s = 0; pass ^= 1u; }
      }
    }
#pragma unroll
    for (int c = 0; c < MAXCH; c++) {
      if (c >= nch) break;
      const double cv = warp_sum(ac[c]);
      const double sv = warp_sum(as64[c] + (f2d_bits(sh[c]) + f2d_bits(sl[c])));
      if (lane == 0) {
        s_part[h][c][j][0] = cv;
        s_part[h][c][j][1] = sv;
      }
    }
  }
  __syncthreads();
  // combine the two row halves in a fixed order and publish this CTA's partial sums
  for (int t = tid; t < ntask; t += blockDim.x) {
    const int c = t / RT_CH, jj = t % RT_CH;
    const double cv = s_part[0][c][jj][0] + s_part[1][c][jj][0];
    double* pp = partials + (int64_t)blockIdx.x * PSTRIDE;
    if (t < k) {
      pp[2 * t] = cv;
      pp[2 * t + 1] = s_part[0][c][jj][1] + s_part[1][c][jj][1];
    } else {
      pp[2 * k + (t - k)] = cv;                // beta -> [2k], s -> [2k + 1]
    }
  }
  if (!last_cta(counter)) return;
  reduce_epilogue(partials, k, 2, sc, EPI_DCGS2, sa);
}

// ---- host side --------------------------------------------------------------------------

// FP64 tensor of `cols` columns of `rows` elements (column stride ld elements), box
// RT_TR x box_cols; cols == 0 encodes a 1D tensor of `rows` elements with box RT_TR.
static bool encode_f64(CUtensorMap* map, const double* p, int64_t rows, int64_t ld, int cols,
                       int box_cols) {
  EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)(cols > 0 ? cols : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {(cuuint32_t)RT_TR, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1, 1};
  const cuuint32_t rank = cols > 0 ? 2 : 1;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank, const_cast<double*>(p), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <bool OFF, int MAXCH>
static kc_status launch_tma_inst(kc_ctx* ctx, int grid, const CUtensorMap& tq,
                                 const CUtensorMap& tx, const CUtensorMap& ty, int k, int64_t m,
                                 const StepArgs& sa) {
  static std::atomic<unsigned long long> attr_done{0};   // per instantiation and device
  KC_TRY(smem_attr_once(ctx, attr_done, k_reduce_tma<OFF, MAXCH>, (int)RT_SMEM, "reduce"));
  k_reduce_tma<OFF, MAXCH><<<grid, RT_THREADS, RT_SMEM, ctx->stream>>>(
      tq, tx, ty, k, m, ctx->partials, ctx->counters, ctx->scal, sa);
  return KC_OK;
}

bool reduce_tma_supported(int k, int64_t m) {
  return k + 2 <= 17 * RT_CH && m >= RT_TR && m < ((int64_t)1 << 31) && tensor_map_encoder() != nullptr;
}

kc_status launch_reduce_tma(kc_ctx* ctx, const double* Q, int64_t ldq, int k, const double* x,
                            const double* y, int64_t m, bool off, const StepArgs& sa) {
  CUtensorMap tq, tx, ty;
  if (!encode_f64(&tq, Q, m, ldq, k > 0 ? k : 1, RT_CH) || !encode_f64(&tx, x, m, m, 0, 1) ||
      !encode_f64(&ty, y, m, m, 0, 1))
    return fail(ctx, KC_ERR_CUDA, "reduce: tensor map encoding failed");
  const int nch = (k + 2 + RT_CH - 1) / RT_CH;
  const int64_t ntiles = (m + RT_TR - 1) / RT_TR;
  const int grid = (int)(ntiles < ctx->num_sms ? ntiles : ctx->num_sms);
  kc_status st = KC_OK;
  if (off) {
    if (nch <= 8) st = launch_tma_inst<true, 8>(ctx, grid, tq, tx, ty, k, m, sa);
    else st = launch_tma_inst<true, 17>(ctx, grid, tq, tx, ty, k, m, sa);
  } else {
    if (nch <= 8) st = launch_tma_inst<false, 8>(ctx, grid, tq, tx, ty, k, m, sa);
    else st = launch_tma_inst<false, 17>(ctx, grid, tq, tx, ty, k, m, sa);
  }
  return st;
}

}  // namespace kc
