// The learned right preconditioner (an addition, not in the paper): a 6-layer 3x3
// convolutional network 1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, zero padding, no bias,
// ReLU after layers 0..4, with BF16 weights and activations and FP32 accumulation.
//
// Layout.  Activations are NHWC in BF16 (32 channels = 64 bytes per pixel).  Weights are
// kept by the caller in FP32 ("master" copy, updated by Adam), per layer [Cout][3][3][Cin],
// layers concatenated (37,440 values); every call converts them to BF16.
//
// The four 32 -> 32 layers are implicit GEMMs on the tensor cores (mma.sync m16n8k16
// BF16 x BF16 -> FP32): rows = output pixels, K = (tap, input channel) = 288, N = 32
// output channels.  A CTA computes an 8 x 32 pixel tile; its input tile with a one-pixel
// halo and the layer's weights sit in shared memory, padded so that ldmatrix rows and
// the B-fragment loads are free of bank conflicts.  The backward data pass is the same
// kernel with flipped, transposed weights; its epilogue applies the ReLU mask.  Weight
// gradients and the 1-channel end layers run on the FP32 CUDA cores.
#include "kc_internal.cuh"

namespace kc {

constexpr int CNN_C = 32;
constexpr int CNN_TAPS = 9;
constexpr int CNN_K = CNN_TAPS * CNN_C;              // 288
constexpr int CNN_W0 = 0;                            // layer offsets in the packed weights
constexpr int CNN_WMID = CNN_C * CNN_TAPS;           // 288: start of layer 1
constexpr int CNN_WMID_SZ = CNN_C * CNN_K;           // 9216 per 32 -> 32 layer
constexpr int CNN_W5 = CNN_WMID + 4 * CNN_WMID_SZ;   // 37152: start of layer 5
constexpr int CNN_NPARAM = CNN_W5 + CNN_K;           // 37440

constexpr int CT_H = 8, CT_W = 32;                   // output pixels per CTA
constexpr int CPAD = 40;                             // BF16 per pixel in shared memory
constexpr int KPAD = 296;                            // BF16 per weight row in shared memory
constexpr int HALO_PIX = (CT_H + 2) * (CT_W + 2);

typedef __nv_bfloat16 bf16;

// float -> bfloat16 bits, round to nearest even (finite inputs)
__device__ __forceinline__ unsigned int bfbits(float f) {
  unsigned int u = __float_as_uint(f);
  return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ unsigned int pack_bf16x2(float a, float b) {
  return bfbits(a) | (bfbits(b) << 16);
}
__device__ __forceinline__ float bf_lo(unsigned int w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned int w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float bfload(const bf16* p) {
  return __uint_as_float(((unsigned int)*reinterpret_cast<const unsigned short*>(p)) << 16);
}

// ---- weights -----------------------------------------------------------------------------

// FP32 master weights -> BF16 forward weights (same layout) and, for the four 32 -> 32
// layers, the flipped transposes used by the backward data pass:
// Wt[l][ci][tap'][co] = W[l][co][8 - tap'][ci].
__global__ void k_cnn_prep_weights(const float* __restrict__ w32, bf16* __restrict__ wf,
                                   bf16* __restrict__ wt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < CNN_NPARAM; i += gridDim.x * blockDim.x) {
    const unsigned short b = (unsigned short)bfbits(w32[i]);
    reinterpret_cast<unsigned short*>(wf)[i] = b;
    if (i >= CNN_WMID && i < CNN_W5) {
      const int l = (i - CNN_WMID) / CNN_WMID_SZ, r = (i - CNN_WMID) % CNN_WMID_SZ;
      const int co = r / CNN_K, tap = (r % CNN_K) / CNN_C, ci = r % CNN_C;
      reinterpret_cast<unsigned short*>(wt)[l * CNN_WMID_SZ + ci * CNN_K + (8 - tap) * CNN_C + co] = b;
    }
  }
}

// ---- 32 -> 32 convolution on the tensor cores ---------------------------------------------

__device__ __forceinline__ void ldmatrix_x4(unsigned int (&r)[4], const void* smem) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned int (&a)[4],
                                         unsigned int b0, unsigned int b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

enum ConvEpi : int { CONV_RELU = 0, CONV_MASK = 1 };

// out[b][y][x][co] = sum_{tap, ci} w[co][tap][ci] * in[b][y+dy-1][x+dx-1][ci], then either
// ReLU (forward) or multiplication by (mask > 0) (backward data pass).
__global__ void __launch_bounds__(256)
k_cnn_conv32(const bf16* __restrict__ in, bf16* __restrict__ out, const bf16* __restrict__ w,
             int H, int W, int epi, const bf16* __restrict__ mask) {
  __shared__ __align__(16) bf16 sIn[HALO_PIX * CPAD];
  __shared__ __align__(16) bf16 sW[CNN_C * KPAD];
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * CT_H, tx0 = blockIdx.x * CT_W;
  const size_t plane = (size_t)H * W;
  const bf16* inb = in + (size_t)b * plane * CNN_C;
  for (int i = threadIdx.x; i < CNN_C * (CNN_K / 8); i += blockDim.x) {
    const int co = i / (CNN_K / 8), c = i % (CNN_K / 8);
    *reinterpret_cast<uint4*>(&sW[co * KPAD + c * 8]) =
        *reinterpret_cast<const uint4*>(&w[co * CNN_K + c * 8]);
  }
  for (int i = threadIdx.x; i < HALO_PIX * 4; i += blockDim.x) {
    const int pix = i >> 2, ch = i & 3;
    const int py = pix / (CT_W + 2), px = pix % (CT_W + 2);
    const int gy = ty0 + py - 1, gx = tx0 + px - 1;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (gy >= 0 && gy < H && gx >= 0 && gx < W)
      val = *reinterpret_cast<const uint4*>(&inb[((size_t)gy * W + gx) * CNN_C + ch * 8]);
    *reinterpret_cast<uint4*>(&sIn[pix * CPAD + ch * 8]) = val;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 2, tid = lane & 3;
  // warp `warp` owns output row `warp` of the tile: two m16 tiles of 16 pixels each
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8;    // ldmatrix row supplied by this lane
  const int lk = (lane >> 4) * 8;                          // and its k offset
  float acc[2][4][4];
#pragma unroll
  for (int j = 0; j < 2; j++)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[j][nt][e] = 0.0f;
#pragma unroll 1
  for (int tap = 0; tap < CNN_TAPS; tap++) {
    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
    for (int kc = 0; kc < 2; kc++) {
      unsigned int a[2][4];
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int pix = (warp + dy) * (CT_W + 2) + j * 16 + lrow + dx;
        ldmatrix_x4(a[j], &sIn[pix * CPAD + kc * 16 + lk]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const bf16* wp = &sW[(nt * 8 + grp) * KPAD + tap * CNN_C + kc * 16 + tid * 2];
        const unsigned int b0 = *reinterpret_cast<const unsigned int*>(wp);
        const unsigned int b1 = *reinterpret_cast<const unsigned int*>(wp + 8);
        mma_bf16(acc[0][nt], a[0], b0, b1);
        mma_bf16(acc[1][nt], a[1], b0, b1);
      }
    }
  }
  bf16* outb = out + (size_t)b * plane * CNN_C;
  const bf16* maskb = mask ? mask + (size_t)b * plane * CNN_C : nullptr;
  const int gy = ty0 + warp;
  if (gy >= H) return;
#pragma unroll
  for (int j = 0; j < 2; j++)
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const int gx = tx0 + j * 16 + grp + half * 8;
      if (gx >= W) continue;
      const size_t pbase = ((size_t)gy * W + gx) * CNN_C;
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const int co = nt * 8 + tid * 2;
        float v0 = acc[j][nt][half * 2], v1 = acc[j][nt][half * 2 + 1];
        if (epi == CONV_RELU) {
          v0 = fmaxf(v0, 0.0f);
          v1 = fmaxf(v1, 0.0f);
        } else {
          const unsigned int mk = *reinterpret_cast<const unsigned int*>(&maskb[pbase + co]);
          if (!(bf_lo(mk) > 0.0f)) v0 = 0.0f;
          if (!(bf_hi(mk) > 0.0f)) v1 = 0.0f;
        }
        *reinterpret_cast<unsigned int*>(&outb[pbase + co]) = pack_bf16x2(v0, v1);
      }
    }
}

}  // namespace kc

namespace kc {

// ---- end layers and their backward passes (FP32 CUDA cores) ------------------------------

// layer 0: x (1 channel, FP32) -> a1 = ReLU(conv), BF16 NHWC.  A CTA computes an
// 8 x 32 pixel tile: the haloed input tile and the weights sit in shared memory, each
// thread computes one pixel's 32 channels into a shared output tile, and the tile rows
// (2 KB each) leave in coalesced 16-byte stores.
__global__ void __launch_bounds__(256)
k_cnn_in(const float* __restrict__ x, bf16* __restrict__ a1, const bf16* __restrict__ wf,
         int H, int W, int B) {
  __shared__ float w0[CNN_C * CNN_TAPS];
  __shared__ float sx[(CT_H + 2) * (CT_W + 2)];
  __shared__ __align__(16) unsigned int so[CT_H * CT_W * 16];
  for (int i = threadIdx.x; i < CNN_C * CNN_TAPS; i += blockDim.x) w0[i] = bfload(&wf[CNN_W0 + i]);
  const int b = blockIdx.z, ty0 = blockIdx.y * CT_H, tx0 = blockIdx.x * CT_W;
  const float* xb = x + (size_t)b * H * W;
  for (int i = threadIdx.x; i < (CT_H + 2) * (CT_W + 2); i += blockDim.x) {
    const int gy = ty0 + i / (CT_W + 2) - 1, gx = tx0 + i % (CT_W + 2) - 1;
    sx[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xb[(size_t)gy * W + gx] : 0.0f;
  }
  __syncthreads();
  const int py = threadIdx.x / CT_W, px = threadIdx.x % CT_W;
  float nb[9];
#pragma unroll
  for (int t = 0; t < 9; t++) nb[t] = sx[(py + t / 3) * (CT_W + 2) + px + t % 3];
#pragma unroll
  for (int c = 0; c < CNN_C; c += 2) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int t = 0; t < 9; t++) {
      s0 = fmaf(w0[c * 9 + t], nb[t], s0);
      s1 = fmaf(w0[(c + 1) * 9 + t], nb[t], s1);
    }
    // word (c / 2) of pixel threadIdx.x, rotated by the pixel index against bank conflicts
    so[threadIdx.x * 16 + ((c / 2 + threadIdx.x) & 15)] = pack_bf16x2(fmaxf(s0, 0.f), fmaxf(s1, 0.f));
  }
  __syncthreads();
  bf16* ob = a1 + (size_t)b * H * W * CNN_C;
  for (int i = threadIdx.x; i < CT_H * CT_W * 4; i += blockDim.x) {      // 16-byte pieces
    const int pix = i >> 2, q = i & 3;
    const int gy = ty0 + pix / CT_W, gx = tx0 + pix % CT_W;
    if (gy >= H || gx >= W) continue;
    uint4 v;
    v.x = so[pix * 16 + ((4 * q + 0 + pix) & 15)];
    v.y = so[pix * 16 + ((4 * q + 1 + pix) & 15)];
    v.z = so[pix * 16 + ((4 * q + 2 + pix) & 15)];
    v.w = so[pix * 16 + ((4 * q + 3 + pix) & 15)];
    *reinterpret_cast<uint4*>(ob + ((size_t)gy * W + gx) * CNN_C + q * 8) = v;
  }
}

// layer 5: a5 (32 channels, BF16) -> y (1 channel, FP32), no activation.  A CTA loads the
// haloed 10 x 34 input tile into shared memory in coalesced 16-byte pieces (pixel stride
// 40 BF16: conflict-free 16-byte reads) and each thread computes one output pixel.
__global__ void __launch_bounds__(256)
k_cnn_out(const bf16* __restrict__ a5, float* __restrict__ y, const bf16* __restrict__ wf,
          int H, int W, int B) {
  __shared__ float w5[CNN_K];
  __shared__ __align__(16) bf16 sIn[HALO_PIX * CPAD];
  for (int i = threadIdx.x; i < CNN_K; i += blockDim.x) w5[i] = bfload(&wf[CNN_W5 + i]);
  const int b = blockIdx.z, ty0 = blockIdx.y * CT_H, tx0 = blockIdx.x * CT_W;
  const bf16* ab = a5 + (size_t)b * H * W * CNN_C;
  for (int i = threadIdx.x; i < HALO_PIX * 4; i += blockDim.x) {
    const int pix = i >> 2, ch = i & 3;
    const int gy = ty0 + pix / (CT_W + 2) - 1, gx = tx0 + pix % (CT_W + 2) - 1;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gy >= 0 && gy < H && gx >= 0 && gx < W)
      v = *reinterpret_cast<const uint4*>(&ab[((size_t)gy * W + gx) * CNN_C + ch * 8]);
    *reinterpret_cast<uint4*>(&sIn[pix * CPAD + ch * 8]) = v;
  }
  __syncthreads();
  const int py = threadIdx.x / CT_W, px = threadIdx.x % CT_W;
  const int gy = ty0 + py, gx = tx0 + px;
  float s = 0.f;
#pragma unroll
  for (int t = 0; t < 9; t++) {
    const bf16* src = &sIn[((py + t / 3) * (CT_W + 2) + px + t % 3) * CPAD];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint4 v = *reinterpret_cast<const uint4*>(src + q * 8);
      const unsigned int u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int ci = q * 8 + e * 2;
        s = fmaf(w5[t * CNN_C + ci], bf_lo(u[e]), s);
        s = fmaf(w5[t * CNN_C + ci + 1], bf_hi(u[e]), s);
      }
    }
  }
  if (gy < H && gx < W) y[((size_t)b * H + gy) * W + gx] = s;
}

// backward of layer 5: dz4 = (conv^T(g, w5)) * (a5 > 0), BF16 NHWC
__global__ void __launch_bounds__(256)
k_cnn_out_bwd(const float* __restrict__ g, const bf16* __restrict__ a5, bf16* __restrict__ dz,
              const bf16* __restrict__ wf, int H, int W, int B) {
  __shared__ float w5[CNN_K];
  for (int i = threadIdx.x; i < CNN_K; i += blockDim.x) w5[i] = bfload(&wf[CNN_W5 + i]);
  __syncthreads();
  const int64_t n = (int64_t)B * H * W;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = p / ((int64_t)H * W);
    const int yx = (int)(p % ((int64_t)H * W)), y0 = yx / W, x0 = yx % W;
    float acc[CNN_C];
#pragma unroll
    for (int c = 0; c < CNN_C; c++) acc[c] = 0.f;
    for (int t = 0; t < 9; t++) {          // pixel q = p - off(t) received tap t
      const int yy = y0 - (t / 3 - 1), xc = x0 - (t % 3 - 1);
      if (yy < 0 || yy >= H || xc < 0 || xc >= W) continue;
      const float gv = g[(b * H + yy) * W + xc];
#pragma unroll
      for (int c = 0; c < CNN_C; c++) acc[c] = fmaf(w5[t * CNN_C + c], gv, acc[c]);
    }
    const uint4* ap = reinterpret_cast<const uint4*>(a5 + p * CNN_C);
    uint4* dp = reinterpret_cast<uint4*>(dz + p * CNN_C);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint4 av = ap[q];
      const unsigned int u[4] = {av.x, av.y, av.z, av.w};
      unsigned int o[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int c = q * 8 + e * 2;
        o[e] = pack_bf16x2(bf_lo(u[e]) > 0.f ? acc[c] : 0.f, bf_hi(u[e]) > 0.f ? acc[c + 1] : 0.f);
      }
      dp[q] = make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
}

// Weight gradients of the two 1-channel layers.  A thread owns (pixel, chunk of 8
// channels) pairs in a grid-stride loop and keeps 9 x 8 partial sums in registers; the CTA
// adds its threads' sums in shared memory (fixed order) and commits them with one atomic
// per weight.
constexpr int DW1_THREADS = 256;

// CTA-wide sum of acc[9][8] over the threads with the same chunk, then dw[off(t, j)] += sum
template <typename F>
__device__ __forceinline__ void dw1_commit(float (&acc)[9][8], int chunk, F index,
                                           float* __restrict__ dw) {
  __shared__ float red[DW1_THREADS / 32][4][72];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // lanes with equal chunk (lane % 4) first: xor 4, 8, 16
#pragma unroll
  for (int t = 0; t < 9; t++)
#pragma unroll
    for (int j = 0; j < 8; j++) {
      float v = acc[t][j];
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      acc[t][j] = v;
    }
  if (lane < 4)
#pragma unroll
    for (int t = 0; t < 9; t++)
#pragma unroll
      for (int j = 0; j < 8; j++) red[warp][chunk][t * 8 + j] = acc[t][j];
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 72; i += blockDim.x) {
    const int c = i / 72, tj = i % 72;
    float s = 0.f;
    for (int w = 0; w < DW1_THREADS / 32; w++) s += red[w][c][tj];
    atomicAdd(&dw[index(c * 8 + tj % 8, tj / 8)], s);
  }
}

// layer 5: dw5[tap][ci] += sum_p g[p] * a5[p + off(tap)][ci]; over input pixels q = p + off:
// sum_q a5[q][ci] * g[q - off(tap)]
__global__ void __launch_bounds__(DW1_THREADS)
k_cnn_dw_out(const float* __restrict__ g, const bf16* __restrict__ a5, float* __restrict__ dw,
             int H, int W, int B) {
  const int chunk = threadIdx.x & 3;
  float acc[9][8];
#pragma unroll
  for (int t = 0; t < 9; t++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[t][j] = 0.f;
  const int64_t n = (int64_t)B * H * W;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2; q < n;
       q += ((int64_t)gridDim.x * blockDim.x) >> 2) {
    const int64_t b = q / ((int64_t)H * W);
    const int yx = (int)(q - b * H * W), y = yx / W, xx = yx % W;
    const uint4 av = *reinterpret_cast<const uint4*>(a5 + q * CNN_C + chunk * 8);
    const unsigned int u[4] = {av.x, av.y, av.z, av.w};
    float a[8];
#pragma unroll
    for (int e = 0; e < 4; e++) { a[2 * e] = bf_lo(u[e]); a[2 * e + 1] = bf_hi(u[e]); }
#pragma unroll
    for (int t = 0; t < 9; t++) {
      const int py = y - (t / 3 - 1), px = xx - (t % 3 - 1);
      if (py < 0 || py >= H || px < 0 || px >= W) continue;
      const float gv = g[(b * H + py) * W + px];
#pragma unroll
      for (int j = 0; j < 8; j++) acc[t][j] = fmaf(gv, a[j], acc[t][j]);
    }
  }
  dw1_commit(acc, chunk, [](int ci, int t) { return CNN_W5 + t * CNN_C + ci; }, dw);
}

// layer 0: dw0[co][tap] += sum_p dz0[p][co] * x[p + off(tap)]
__global__ void __launch_bounds__(DW1_THREADS)
k_cnn_dw_in(const bf16* __restrict__ dz0, const float* __restrict__ x, float* __restrict__ dw,
            int H, int W, int B) {
  const int chunk = threadIdx.x & 3;
  float acc[9][8];
#pragma unroll
  for (int t = 0; t < 9; t++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[t][j] = 0.f;
  const int64_t n = (int64_t)B * H * W;
  for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2; p < n;
       p += ((int64_t)gridDim.x * blockDim.x) >> 2) {
    const int64_t b = p / ((int64_t)H * W);
    const int yx = (int)(p - b * H * W), y = yx / W, xx = yx % W;
    const uint4 dv = *reinterpret_cast<const uint4*>(dz0 + p * CNN_C + chunk * 8);
    const unsigned int u[4] = {dv.x, dv.y, dv.z, dv.w};
    float d[8];
#pragma unroll
    for (int e = 0; e < 4; e++) { d[2 * e] = bf_lo(u[e]); d[2 * e + 1] = bf_hi(u[e]); }
#pragma unroll
    for (int t = 0; t < 9; t++) {
      const int qy = y + t / 3 - 1, qx = xx + t % 3 - 1;
      if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
      const float xv = x[(b * H + qy) * W + qx];
#pragma unroll
      for (int j = 0; j < 8; j++) acc[t][j] = fmaf(d[j], xv, acc[t][j]);
    }
  }
  dw1_commit(acc, chunk, [](int co, int t) { return CNN_W0 + co * CNN_TAPS + t; }, dw);
}

}  // namespace kc

namespace kc {

// weight gradient of a 32 -> 32 layer: dw[co][tap][ci] += sum_p dz[p][co] * a[p + off(tap)][ci]
// CTA: an 8 x 32 pixel tile (dz) with its haloed input tile in shared memory; warp w owns
// output channels 4w..4w+3, lane = ci, and each thread keeps 4 x 9 partial sums.
__global__ void __launch_bounds__(256)
k_cnn_dw32(const bf16* __restrict__ dz, const bf16* __restrict__ a, float* __restrict__ dw,
           int H, int W) {
  __shared__ __align__(16) bf16 sA[HALO_PIX * CNN_C];
  __shared__ __align__(16) bf16 sG[CT_H * CT_W * CNN_C];
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * CT_H, tx0 = blockIdx.x * CT_W;
  const size_t plane = (size_t)H * W;
  const bf16* ab = a + (size_t)b * plane * CNN_C;
  const bf16* gb = dz + (size_t)b * plane * CNN_C;
  for (int i = threadIdx.x; i < HALO_PIX * 4; i += blockDim.x) {
    const int pix = i >> 2, ch = i & 3;
    const int gy = ty0 + pix / (CT_W + 2) - 1, gx = tx0 + pix % (CT_W + 2) - 1;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (gy >= 0 && gy < H && gx >= 0 && gx < W)
      val = *reinterpret_cast<const uint4*>(&ab[((size_t)gy * W + gx) * CNN_C + ch * 8]);
    *reinterpret_cast<uint4*>(&sA[pix * CNN_C + ch * 8]) = val;
  }
  for (int i = threadIdx.x; i < CT_H * CT_W * 4; i += blockDim.x) {
    const int pix = i >> 2, ch = i & 3;
    const int gy = ty0 + pix / CT_W, gx = tx0 + pix % CT_W;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);          // pixels outside the image add nothing
    if (gy < H && gx < W)
      val = *reinterpret_cast<const uint4*>(&gb[((size_t)gy * W + gx) * CNN_C + ch * 8]);
    *reinterpret_cast<uint4*>(&sG[pix * CNN_C + ch * 8]) = val;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, ci = threadIdx.x & 31;
  float acc[4][9];
#pragma unroll
  for (int c = 0; c < 4; c++)
#pragma unroll
    for (int t = 0; t < 9; t++) acc[c][t] = 0.f;
  for (int py = 0; py < CT_H; py++) {
    for (int px = 0; px < CT_W; px++) {
      const uint2 gv = *reinterpret_cast<const uint2*>(&sG[(py * CT_W + px) * CNN_C + warp * 4]);
      const float g0 = bf_lo(gv.x), g1 = bf_hi(gv.x), g2 = bf_lo(gv.y), g3 = bf_hi(gv.y);
#pragma unroll
      for (int t = 0; t < 9; t++) {
        const float av = bfload(&sA[((py + t / 3) * (CT_W + 2) + px + t % 3) * CNN_C + ci]);
        acc[0][t] = fmaf(g0, av, acc[0][t]);
        acc[1][t] = fmaf(g1, av, acc[1][t]);
        acc[2][t] = fmaf(g2, av, acc[2][t]);
        acc[3][t] = fmaf(g3, av, acc[3][t]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; c++)
#pragma unroll
    for (int t = 0; t < 9; t++)
      atomicAdd(&dw[(warp * 4 + c) * CNN_K + t * CNN_C + ci], acc[c][t]);
}

// per-sample sums of (y - e)^2 and e^2 (FP64 atomics)
__global__ void __launch_bounds__(256)
k_cnn_loss_sums(const float* __restrict__ y, const float* __restrict__ e, double* __restrict__ sums,
                int64_t npix) {
  const int b = blockIdx.y;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)y[b * npix + i] - (double)e[b * npix + i];
    s0 += d * d;
    s1 += (double)e[b * npix + i] * (double)e[b * npix + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[2 * b], s0);
    atomicAdd(&sums[2 * b + 1], s1);
  }
}

// g = (2/B) (y - e) / ||e||^2
__global__ void __launch_bounds__(256)
k_cnn_loss_grad(const float* __restrict__ y, const float* __restrict__ e,
                const double* __restrict__ sums, float* __restrict__ g, int64_t npix, int B) {
  const int b = blockIdx.y;
  const double sc = 2.0 / ((double)B * sums[2 * b + 1]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
       i += (int64_t)gridDim.x * blockDim.x)
    g[b * npix + i] = (float)(sc * ((double)y[b * npix + i] - (double)e[b * npix + i]));
}

// Residual loss (the preconditioner's training loss on an operator A shared by the batch):
// res_b = A (x_b + y_b) - r_b; sums[2b] += ||res_b||^2, sums[2b+1] += ||r_b||^2.
__global__ void __launch_bounds__(256)
k_cnn_res_sums(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
               const double* __restrict__ av, const float* __restrict__ x,
               const float* __restrict__ y, const float* __restrict__ r, float* __restrict__ res,
               double* __restrict__ sums, int64_t npix) {
  const int b = blockIdx.y;
  const float* xb = x + b * npix;
  const float* yb = y + b * npix;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; p++) {
      const int j = ci[p];
      acc += av[p] * ((double)xb[j] + (double)yb[j]);
    }
    const double ri = (double)r[b * npix + i];
    const double d = acc - ri;
    res[b * npix + i] = (float)d;
    s0 += d * d;
    s1 += ri * ri;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[2 * b], s0);
    atomicAdd(&sums[2 * b + 1], s1);
  }
}

// g_b = (2/B) A^T res_b / ||r_b||^2, scattered along the rows of A (g zeroed beforehand)
__global__ void __launch_bounds__(256)
k_cnn_res_grad(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
               const double* __restrict__ av, const float* __restrict__ res,
               const double* __restrict__ sums, float* __restrict__ g, int64_t npix, int B) {
  const int b = blockIdx.y;
  const double sc = 2.0 / ((double)B * sums[2 * b + 1]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double t = sc * (double)res[b * npix + i];
    for (int p = rp[i]; p < rp[i + 1]; p++)
      atomicAdd(&g[b * npix + ci[p]], (float)(av[p] * t));
  }
}

// Adam on the FP32 master weights
__global__ void k_cnn_adam(float* __restrict__ w, const float* __restrict__ g,
                           float* __restrict__ mo, float* __restrict__ ve, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < CNN_NPARAM; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float m = b1 * mo[i] + (1.f - b1) * gi;
    const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    w[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// ---- launchers (used by kc_cnn_api.cu) -------------------------------------------------------

static dim3 conv_grid(int H, int W, int B) {
  return dim3((W + CT_W - 1) / CT_W, (H + CT_H - 1) / CT_H, B);
}
// pixel-chunk threads (4 per pixel), at most 4 CTAs per SM
static int dw1_grid(const kc_ctx* ctx, int64_t n) {
  int64_t g = (4 * n + DW1_THREADS - 1) / DW1_THREADS, cap = (int64_t)ctx->num_sms * 4;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}
static int pix_grid(const kc_ctx* ctx, int64_t n) {
  int64_t g = (n + 255) / 256, cap = (int64_t)ctx->num_sms * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// One 32 -> 32 layer on the kernel the context selects (tcgen05 or mma.sync).
static kc_status conv32(kc_ctx* ctx, const bf16* in, bf16* out, const bf16* w, int B, int H,
                        int W, int epi, const bf16* mask) {
  if (ctx->conv_tc) return cnn_conv32_tc(ctx, in, out, w, B, H, W, epi, mask);
  timing_begin(ctx, KID_OTHER);
  k_cnn_conv32<<<conv_grid(H, W, B), 256, 0, ctx->stream>>>(in, out, w, H, W, epi, mask);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

// Forward pass.  wf/wt: BF16 weights prepared by cnn_prep.  acts: 5 activation buffers of
// B*H*W*32 BF16 each when `keep` (training), else 2 used as ping-pong.  Returns in y.
kc_status cnn_forward(kc_ctx* ctx, const bf16* wf, const float* x, float* y, bf16* const* acts,
                      bool keep, int B, int H, int W) {
  const int64_t n = (int64_t)B * H * W;
  timing_begin(ctx, KID_OTHER);
  k_cnn_in<<<conv_grid(H, W, B), 256, 0, ctx->stream>>>(x, acts[0], wf, H, W, B);
  KC_LAUNCHED(ctx);
  for (int l = 0; l < 4; l++) {
    const bf16* src = keep ? acts[l] : acts[l & 1];
    bf16* dst = keep ? acts[l + 1] : acts[(l + 1) & 1];
    kc_status s = conv32(ctx, src, dst, wf + CNN_WMID + l * CNN_WMID_SZ, B, H, W, CONV_RELU,
                         nullptr);
    if (s != KC_OK) return s;
  }
  timing_begin(ctx, KID_OTHER);
  k_cnn_out<<<conv_grid(H, W, B), 256, 0, ctx->stream>>>(keep ? acts[4] : acts[0], y, wf, H, W, B);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status cnn_prep(kc_ctx* ctx, const float* w32, bf16* wf, bf16* wt) {
  timing_begin(ctx, KID_SMALL);
  k_cnn_prep_weights<<<64, 256, 0, ctx->stream>>>(w32, wf, wt);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

// Backward pass after a kept forward: g (dL/dy, FP32) -> dw (FP32, accumulated).
// dz: two ping-pong BF16 gradient buffers.
kc_status cnn_backward(kc_ctx* ctx, const bf16* wf, const bf16* wt, const float* x,
                       const float* g, bf16* const* acts, bf16* const* dz, float* dw, int B,
                       int H, int W) {
  const int64_t n = (int64_t)B * H * W;
  const int nblk = (int)((n + 255) / 256);
  timing_begin(ctx, KID_OTHER);
  k_cnn_dw_out<<<dw1_grid(ctx, n), DW1_THREADS, 0, ctx->stream>>>(g, acts[4], dw, H, W, B);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_OTHER);
  k_cnn_out_bwd<<<pix_grid(ctx, n), 256, 0, ctx->stream>>>(g, acts[4], dz[0], wf, H, W, B);
  KC_LAUNCHED(ctx);
  int cur = 0;
  for (int l = 3; l >= 0; l--) {      // 32 -> 32 layer l maps acts[l] -> acts[l+1]
    timing_begin(ctx, KID_OTHER);
    k_cnn_dw32<<<conv_grid(H, W, B), 256, 0, ctx->stream>>>(
        dz[cur], acts[l], dw + CNN_WMID + l * CNN_WMID_SZ, H, W);
    KC_LAUNCHED(ctx);
    kc_status s = conv32(ctx, dz[cur], dz[cur ^ 1], wt + l * CNN_WMID_SZ, B, H, W, CONV_MASK,
                         acts[l]);
    if (s != KC_OK) return s;
    cur ^= 1;
  }
  timing_begin(ctx, KID_OTHER);
  k_cnn_dw_in<<<dw1_grid(ctx, n), DW1_THREADS, 0, ctx->stream>>>(dz[cur], x, dw, H, W, B);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status cnn_loss_grad(kc_ctx* ctx, const float* y, const float* e, double* sums, float* g,
                        int B, int64_t npix) {
  KC_CUDA(ctx, cudaMemsetAsync(sums, 0, 2 * B * sizeof(double), ctx->stream));
  dim3 grid((unsigned)((npix + 255) / 256 < 64 ? (npix + 255) / 256 : 64), B);
  timing_begin(ctx, KID_SMALL);
  k_cnn_loss_sums<<<grid, 256, 0, ctx->stream>>>(y, e, sums, npix);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_SMALL);
  k_cnn_loss_grad<<<grid, 256, 0, ctx->stream>>>(y, e, sums, g, npix, B);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status cnn_residual_loss_grad(kc_ctx* ctx, const kc_csr* A, const float* x, const float* y,
                                 const float* r, float* res, double* sums, float* g, int B,
                                 int64_t npix) {
  KC_CUDA(ctx, cudaMemsetAsync(sums, 0, 2 * B * sizeof(double), ctx->stream));
  KC_CUDA(ctx, cudaMemsetAsync(g, 0, (size_t)B * npix * sizeof(float), ctx->stream));
  dim3 grid((unsigned)((npix + 255) / 256 < 64 ? (npix + 255) / 256 : 64), B);
  const double* av = (const double*)A->val;
  timing_begin(ctx, KID_SMALL);
  k_cnn_res_sums<<<grid, 256, 0, ctx->stream>>>(A->row_ptr, A->col_idx, av, x, y, r, res, sums,
                                                npix);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_SMALL);
  k_cnn_res_grad<<<grid, 256, 0, ctx->stream>>>(A->row_ptr, A->col_idx, av, res, sums, g, npix, B);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status cnn_adam(kc_ctx* ctx, float* w, const float* g, float* m, float* v, int64_t t,
                   float lr, float b1, float b2, float eps) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  timing_begin(ctx, KID_SMALL);
  k_cnn_adam<<<64, 256, 0, ctx->stream>>>(w, g, m, v, lr, b1, b2, eps, c1, c2);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

int64_t cnn_nparam() { return CNN_NPARAM; }

}  // namespace kc
