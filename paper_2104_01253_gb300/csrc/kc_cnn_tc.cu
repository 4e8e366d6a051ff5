// 32 -> 32 3x3 convolution on the 5th-generation tensor cores (tcgen05, accumulator in
// tensor memory), the implicit GEMM of the learned preconditioner's hidden layers:
// rows = 128 output pixels of a 16 x 8 tile, N = 32 output channels, K = 9 taps x 32
// input channels, as 18 MMAs of K = 16 (BF16 x BF16 -> FP32).
//
// A persistent CTA of six warps runs a three-role pipeline over its tiles:
//   warp 0 (one thread): four 4D tensor copies per tile (one per 8-channel plane) bring
//     the 18 x 10 input tile with its one-pixel halo into a ring of TP_NS stages; the
//     copies start at the tile origin minus one pixel and read zeros outside the image;
//   warp 1 (one thread): 18 tcgen05.mma per tile into one of two 32-column accumulators
//     in tensor memory, then commits that free the stage and publish the accumulator;
//   warps 2-5: read the accumulator back (tcgen05.ld, one pixel per thread), release it,
//     and apply ReLU (forward) or the ReLU mask (backward data pass) while storing BF16
//     NHWC.
// Shared memory (no swizzle, K-major core matrices of 8 rows x 16 bytes):
//   weights, once per CTA: block (tap, chunk of 8 input channels) of 32 output channels x
//     16 bytes; a K = 16 step is two adjacent blocks (LBO 512 B, SBO 128 B);
//   a stage: four planes of 8 channels, 16 bytes per halo pixel (2944-byte planes, so
//     every copy lands 128-byte aligned).  Eight consecutive output pixels of a tile row
//     are eight consecutive halo pixels and the next row is 10 pixels further, so every
//     tap is the same descriptor (LBO = one plane, SBO = 160 B) with a start address
//     shifted by (dy * 10 + dx) * 16 bytes: no im2col copy.
// Every wait is bounded: on a timeout the kernel records KC_ERR_TIMEOUT, stops, waits
// (bounded) for its copies and MMAs in flight, frees its tensor memory and returns.
#include "kc_internal.cuh"
#include "kc_tcgen05.cuh"
#include "kc_tma.cuh"

namespace kc {

typedef __nv_bfloat16 bf16;

constexpr int TC_TH = 16, TC_TW = 8;                      // output tile: 128 pixels
constexpr int TC_HH = TC_TH + 2, TC_HW = TC_TW + 2;       // halo tile 18 x 10
constexpr int TP_PLANE = 2944;                            // 18 * 10 * 16 B, rounded to 128
constexpr int TP_STAGE = 4 * TP_PLANE;
constexpr int TP_BOX_BYTES = 4 * TC_HH * TC_HW * 16;      // 11520 bytes copied per stage
constexpr int TP_NS = 4;                                  // ring stages
constexpr int TC_WREGION = 20480;                         // weights (18432 B), 128-aligned
constexpr int TP_OUT = 4 * 32 * 64;                       // epilogue staging: 4 warps x 32 pixels
static_assert(TC_TW == 8 && TC_TH * TC_TW == 4 * 32, "each epilogue warp owns four 8-pixel tile rows");
constexpr int TP_SMEM = 128 + TC_WREGION + TP_NS * TP_STAGE + TP_OUT;
constexpr int TP_THREADS = 192;
constexpr int TP_TMEM_COLS = 64;                          // two 32-column accumulators
constexpr int TC_CTAS_PER_SM = 2;
constexpr uint32_t TC_IDESC = idesc_bf16_f32(128, 32);
static_assert(TP_PLANE % 128 == 0 && TP_PLANE >= TC_HH * TC_HW * 16, "plane size");
static_assert(TC_WREGION % 128 == 0 && TC_WREGION >= 9 * 4 * 512, "weight region");

__device__ __forceinline__ unsigned int tc_bfbits(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1),
        "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// out = ReLU(conv(in, w)) (epi 0) or conv(in, w) * (mask > 0) (epi 1); NHWC BF16.
// tin: 4D tensor map of `in` (dims C = 32, W, H, B; box 8 x 10 x 18 x 1).
__global__ void __launch_bounds__(TP_THREADS, 1)
k_cnn_conv32_tc(const __grid_constant__ CUtensorMap tin, bf16* __restrict__ out,
                const bf16* __restrict__ w, int B, int H, int W, int epi,
                const bf16* __restrict__ mask, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char* sW = base;
  unsigned char* sStage = base + TC_WREGION;
  unsigned char* sOut = base + TC_WREGION + TP_NS * TP_STAGE;
  __shared__ unsigned long long full[TP_NS], empty[TP_NS], tfull[2], tempty[2];
  __shared__ unsigned int tmem_sh;
  __shared__ int s_err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights: w[co][tap][ci] -> block (tap * 4 + ci / 8) of [co][8 ci]
  for (int i = tid; i < 32 * 36; i += blockDim.x) {
    const int co = i / 36, blk = i % 36;
    *reinterpret_cast<uint4*>(sW + (blk * 32 + co) * 16) =
        *reinterpret_cast<const uint4*>(w + co * 288 + blk * 8);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(smem_u32(&tmem_sh)), "r"(TP_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TP_NS; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    fence_barrier_init();
    s_err = 0;
  }
  fence_async_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned int tmem = tmem_sh;
  volatile int* err = &s_err;

  const int tiles_x = (W + TC_TW - 1) / TC_TW, tiles_y = (H + TC_TH - 1) / TC_TH;
  const int64_t per_img = (int64_t)tiles_x * tiles_y;
  const int64_t ntile = per_img * B;

  if (warp == 0) {
    // ---- producer: tensor copies of the halo tiles ----
    if (lane == 0) {
      int s = 0;
      unsigned int ph = 0;
      int last_par[TP_NS];
      for (int i = 0; i < TP_NS; i++) last_par[i] = -1;
      for (int64_t tile = blockIdx.x; tile < ntile && !*err; tile += gridDim.x) {
        const int b = (int)(tile / per_img), rem = (int)(tile % per_img);
        const int y0 = (rem / tiles_x) * TC_TH, x0 = (rem % tiles_x) * TC_TW;
        if (!mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT)) {
          *err = 1;
          atomicExch(status, (int)KC_ERR_TIMEOUT);
          break;
        }
        unsigned char* st = sStage + s * TP_STAGE;
        mbar_arrive_expect_tx(&full[s], TP_BOX_BYTES);
#pragma unroll
        for (int c8 = 0; c8 < 4; c8++)
          tma_load_4d(st + c8 * TP_PLANE, &tin, c8 * 8, x0 - 1, y0 - 1, b, &full[s]);
        last_par[s] = (int)ph;
        if (++s == TP_NS) { s = 0; ph ^= 1u; }
      }
      // every copy issued has landed before the CTA's shared memory goes away
      for (int i = 0; i < TP_NS; i++)
        if (last_par[i] >= 0) (void)mbar_wait(&full[i], (unsigned int)last_par[i], WAIT_LIMIT);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const unsigned int sw = smem_u32(sW);
      int s = 0, bb = 0;
      unsigned int ph = 0, tph = 0;
      int last_bb = -1;
      unsigned int last_tph = 0;
      for (int64_t tile = blockIdx.x; tile < ntile && !*err; tile += gridDim.x) {
        if (!mbar_wait(&full[s], ph, WAIT_LIMIT) || !mbar_wait(&tempty[bb], tph ^ 1u, WAIT_LIMIT)) {
          *err = 1;
          atomicExch(status, (int)KC_ERR_TIMEOUT);
          break;
        }
        tc_fence_after();
        const unsigned int sa = smem_u32(sStage + s * TP_STAGE);
        const unsigned int d = tmem + (unsigned int)(bb * 32);
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
          const int dy = tap / 3, dx = tap % 3;
#pragma unroll
          for (int kk = 0; kk < 2; kk++) {
            const unsigned long long ad =
                umma_desc(sa + 2 * kk * TP_PLANE + (dy * TC_HW + dx) * 16, TP_PLANE, TC_HW * 16);
            const unsigned long long bd = umma_desc(sw + (tap * 4 + 2 * kk) * 512, 512, 128);
            tc_mma(d, ad, bd, TC_IDESC, (tap | kk) ? 1u : 0u);
          }
        }
        tc_commit(&empty[s]);               // the stage is free once these MMAs are done
        tc_commit(&tfull[bb]);              // and the accumulator is ready
        last_bb = bb;
        last_tph = tph;
        if (++s == TP_NS) { s = 0; ph ^= 1u; }
        bb ^= 1;
        if (bb == 0) tph ^= 1u;
      }
      if (last_bb >= 0)                     // MMAs in flight are done before teardown
        (void)mbar_wait(&tfull[last_bb], last_tph, WAIT_LIMIT);
    }
  } else {
    // ---- epilogue: warps 2..5, tensor-memory lane quarter warp % 4 ----
    const int q = warp & 3;
    int bb = 0;
    unsigned int tph = 0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
      if (!mbar_wait(&tfull[bb], tph, WAIT_LIMIT)) {
        *err = 1;
        atomicExch(status, (int)KC_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      float v[32];
      tc_ld32(tmem + (unsigned int)(bb * 32) + ((unsigned int)(q * 32) << 16), v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[bb]);
      const int b = (int)(tile / per_img), rem = (int)(tile % per_img);
      const int y0 = (rem / tiles_x) * TC_TH, x0 = (rem % tiles_x) * TC_TW;
      const int m = q * 32 + lane;
      const int gy = y0 + m / TC_TW, gx = x0 + m % TC_TW;
      // this warp's 32 pixels = tile rows 4q .. 4q + 3; stage them in shared memory (16-byte
      // chunks swizzled by pixel, conflict-free) and write whole 512-byte rows
      unsigned char* so = sOut + q * 32 * 64;
      if (epi == 0) {
#pragma unroll
        for (int c = 0; c < 32; c++) v[c] = fmaxf(v[c], 0.0f);
      } else if (gy < H && gx < W) {
        const size_t p = (((size_t)b * H + gy) * W + gx) * 32;
#pragma unroll
        for (int qq = 0; qq < 4; qq++) {
          const uint4 mk = *reinterpret_cast<const uint4*>(mask + p + qq * 8);
          const unsigned int mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
          for (int t = 0; t < 4; t++) {
            if (!(__uint_as_float(mw[t] << 16) > 0.0f)) v[qq * 8 + 2 * t] = 0.0f;
            if (!(__uint_as_float(mw[t] & 0xffff0000u) > 0.0f)) v[qq * 8 + 2 * t + 1] = 0.0f;
          }
        }
      }
#pragma unroll
      for (int qq = 0; qq < 4; qq++) {
        uint4 o;
        o.x = tc_bfbits(v[qq * 8 + 0]) | (tc_bfbits(v[qq * 8 + 1]) << 16);
        o.y = tc_bfbits(v[qq * 8 + 2]) | (tc_bfbits(v[qq * 8 + 3]) << 16);
        o.z = tc_bfbits(v[qq * 8 + 4]) | (tc_bfbits(v[qq * 8 + 5]) << 16);
        o.w = tc_bfbits(v[qq * 8 + 6]) | (tc_bfbits(v[qq * 8 + 7]) << 16);
        *reinterpret_cast<uint4*>(so + lane * 64 + ((qq ^ ((lane >> 1) & 3)) * 16)) = o;
      }
      __syncwarp();
#pragma unroll
      for (int row = 0; row < 4; row++) {
        const int pix = row * 8 + (lane >> 2), qq = lane & 3;
        const int ry = y0 + 4 * q + row, rx = x0 + (lane >> 2);
        const uint4 o = *reinterpret_cast<const uint4*>(so + pix * 64 + ((qq ^ ((pix >> 1) & 3)) * 16));
        if (ry < H && rx < W)
          *reinterpret_cast<uint4*>(out + (((size_t)b * H + ry) * W + rx) * 32 + qq * 8) = o;
      }
      __syncwarp();
      bb ^= 1;
      if (bb == 0) tph ^= 1u;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 ::"r"(tmem), "r"(TP_TMEM_COLS) : "memory");
}

kc_status cnn_conv32_tc(kc_ctx* ctx, const bf16* in, bf16* out, const bf16* w, int B, int H,
                        int W, int epi, const bf16* mask) {
  static std::atomic<unsigned long long> attr_done{0};
  KC_TRY(smem_attr_once(ctx, attr_done, k_cnn_conv32_tc, TP_SMEM, "conv"));
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return fail(ctx, KC_ERR_CUDA, "conv: no tensor map encoder");
  CUtensorMap tin;
  const cuuint64_t dims[4] = {32, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {64, (cuuint64_t)W * 64, (cuuint64_t)H * W * 64};
  const cuuint32_t box[4] = {8, TC_HW, TC_HH, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (enc(&tin, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(in), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return fail(ctx, KC_ERR_CUDA, "conv: tensor map encoding failed");
  const int64_t ntile = (int64_t)((W + TC_TW - 1) / TC_TW) * ((H + TC_TH - 1) / TC_TH) * B;
  const int64_t cap = (int64_t)ctx->num_sms * TC_CTAS_PER_SM;
  const int grid = (int)(ntile < cap ? ntile : cap);
  timing_begin(ctx, KID_OTHER);
  k_cnn_conv32_tc<<<grid, TP_THREADS, TP_SMEM, ctx->stream>>>(tin, out, w, B, H, W, epi, mask,
                                                              &ctx->scal->status);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

}  // namespace kc
