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
// kernel with flipped, transposed weights; its epilogue applies the ReLU mask.  The weight
// gradient of the 32 -> 32 layers is a tensor-core product too (K = pixels); the
// 1-channel end layers and their weight gradients run on the FP32 CUDA cores.
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

// ---- end layers and their backward passes -----------------------------------------------

// The 1-channel end layers.  Layers 0 and 5-backward run on the FP32 CUDA cores as tile
// kernels on a persistent grid: the scalar field's haloed 8 x 32 tile (zero outside the
// image) sits in shared memory, four threads share a pixel, each owns 8 of the 32 channels
// with their 9 x 8 weights in registers, and a thread's 8 channels leave or arrive as one
// 16-byte piece (a warp covers 8 whole pixels, 512 contiguous bytes).  The next tile's
// halo values and first piece are loaded into registers while the current tile computes,
// so the persistent CTAs do not wait on global memory at each tile.
constexpr int END_THREADS = 256;                     // 64 pixels x 4 channel chunks per pass
constexpr int END_PASSES = CT_H * CT_W / 64;
constexpr int HALO1 = (CT_H + 2) * (CT_W + 2);       // values of a scalar field's halo tile
static_assert(2 * END_THREADS >= HALO1, "two halo values per thread");

struct Tile { int b, ty0, tx0; };
__device__ __forceinline__ Tile tile_at(int64_t t, int per_img, int tiles_x) {
  const int b = (int)(t / per_img), rem = (int)(t % per_img);
  return {b, (rem / tiles_x) * CT_H, (rem % tiles_x) * CT_W};
}
// this thread's two values of the scalar field's haloed tile (zero outside the image)
__device__ __forceinline__ void halo1_fetch(const float* __restrict__ f, Tile t, int H, int W,
                                            float (&h)[2]) {
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int i = threadIdx.x + r * END_THREADS;
    float v = 0.0f;
    if (i < HALO1) {
      const int gy = t.ty0 + i / (CT_W + 2) - 1, gx = t.tx0 + i % (CT_W + 2) - 1;
      if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = f[((size_t)t.b * H + gy) * W + gx];
    }
    h[r] = v;
  }
}
__device__ __forceinline__ void halo1_store(float* s, const float (&h)[2]) {
  s[threadIdx.x] = h[0];
  if (threadIdx.x + END_THREADS < HALO1) s[threadIdx.x + END_THREADS] = h[1];
}
// the 16-byte piece (channels 8 chunk .. 8 chunk + 7) of pass `pass`'s pixel of tile t
// (pq = thread / 4), zeros outside the image
__device__ __forceinline__ uint4 piece_at(const bf16* __restrict__ t32, Tile t, int pass,
                                          int pq, int chunk, int H, int W) {
  const int lp = pass * 64 + pq, gy = t.ty0 + lp / CT_W, gx = t.tx0 + lp % CT_W;
  return (gy < H && gx < W)
             ? *reinterpret_cast<const uint4*>(t32 + (((size_t)t.b * H + gy) * W + gx) * CNN_C +
                                               chunk * 8)
             : make_uint4(0u, 0u, 0u, 0u);
}

// layer 0: x (1 channel, FP32) -> a1 = ReLU(conv), BF16 NHWC
__global__ void __launch_bounds__(END_THREADS)
k_cnn_in(const float* __restrict__ x, bf16* __restrict__ a1, const bf16* __restrict__ wf,
         int H, int W, int B) {
  __shared__ float sx[HALO1];
  const int chunk = threadIdx.x & 3, pq = threadIdx.x >> 2;
  float w[8][9];                                     // w0[co = 8 chunk + j][tap]
#pragma unroll
  for (int j = 0; j < 8; j++)
#pragma unroll
    for (int t = 0; t < 9; t++) w[j][t] = bfload(&wf[CNN_W0 + (chunk * 8 + j) * CNN_TAPS + t]);
  const int tiles_x = (W + CT_W - 1) / CT_W, tiles_y = (H + CT_H - 1) / CT_H;
  const int per_img = tiles_x * tiles_y;
  const int64_t ntiles = (int64_t)per_img * B;
  float h[2] = {0.0f, 0.0f};
  if (blockIdx.x < ntiles) halo1_fetch(x, tile_at(blockIdx.x, per_img, tiles_x), H, W, h);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tt = tile_at(tile, per_img, tiles_x);
    __syncthreads();                                 // the previous tile's reads are done
    halo1_store(sx, h);
    __syncthreads();
    if (tile + gridDim.x < ntiles)
      halo1_fetch(x, tile_at(tile + gridDim.x, per_img, tiles_x), H, W, h);
#pragma unroll 1
    for (int pass = 0; pass < END_PASSES; pass++) {
      const int lp = pass * 64 + pq, ly = lp / CT_W, lx = lp % CT_W;
      const int gy = tt.ty0 + ly, gx = tt.tx0 + lx;
      if (gy >= H || gx >= W) continue;
      float nb[9];
#pragma unroll
      for (int t = 0; t < 9; t++) nb[t] = sx[(ly + t / 3) * (CT_W + 2) + lx + t % 3];
      unsigned int o[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int t = 0; t < 9; t++) {
          s0 = fmaf(w[2 * e][t], nb[t], s0);
          s1 = fmaf(w[2 * e + 1][t], nb[t], s1);
        }
        o[e] = pack_bf16x2(fmaxf(s0, 0.f), fmaxf(s1, 0.f));
      }
      *reinterpret_cast<uint4*>(a1 + (((size_t)tt.b * H + gy) * W + gx) * CNN_C + chunk * 8) =
          make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
}

// layer 5: a5 (32 channels, BF16) -> y (1 channel, FP32), no activation.  The same implicit
// GEMM on the tensor cores as the 32 -> 32 layers (rows = pixels of an 8 x 32 tile,
// K = (tap, ci) = 288, mma.sync m16n8k16 BF16 x BF16 -> FP32) with one 8-column B tile
// whose column 0 holds w5 and the other columns zero; the lanes holding column 0 store y.
__global__ void __launch_bounds__(256)
k_cnn_out(const bf16* __restrict__ a5, float* __restrict__ y, const bf16* __restrict__ wf,
          int H, int W, int B) {
  __shared__ __align__(16) bf16 sIn[HALO_PIX * CPAD];
  __shared__ __align__(16) bf16 sW5[CNN_K];
  for (int i = threadIdx.x; i < CNN_K; i += blockDim.x) sW5[i] = wf[CNN_W5 + i];
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 2, tid = lane & 3;
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8;    // ldmatrix row supplied by this lane
  const int lk = (lane >> 4) * 8;                          // and its k offset
  float acc[2][4];
#pragma unroll
  for (int j = 0; j < 2; j++)
#pragma unroll
    for (int e = 0; e < 4; e++) acc[j][e] = 0.0f;
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
      const bf16* wp = &sW5[tap * CNN_C + kc * 16 + tid * 2];
      const unsigned int b0 = grp == 0 ? *reinterpret_cast<const unsigned int*>(wp) : 0u;
      const unsigned int b1 = grp == 0 ? *reinterpret_cast<const unsigned int*>(wp + 8) : 0u;
      mma_bf16(acc[0], a[0], b0, b1);
      mma_bf16(acc[1], a[1], b0, b1);
    }
  }
  const int gy = ty0 + warp;
  if (tid != 0 || gy >= H) return;                         // column 0: lanes with tid 0
#pragma unroll
  for (int j = 0; j < 2; j++)
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const int gx = tx0 + j * 16 + grp + half * 8;
      if (gx < W) y[((size_t)b * H + gy) * W + gx] = acc[j][half * 2];
    }
}

// backward of layer 5: dz4[p][ci] = (a5[p][ci] > 0) * sum_tap w5[tap][ci] g[p - off(tap)],
// BF16 NHWC; the haloed g tile in shared memory, 72 weights per thread in registers
__global__ void __launch_bounds__(END_THREADS)
k_cnn_out_bwd(const float* __restrict__ g, const bf16* __restrict__ a5, bf16* __restrict__ dz,
              const bf16* __restrict__ wf, int H, int W, int B) {
  __shared__ float sg[HALO1];
  const int chunk = threadIdx.x & 3, pq = threadIdx.x >> 2;
  float w[8][9];                                     // w5[tap][ci = 8 chunk + j]
#pragma unroll
  for (int j = 0; j < 8; j++)
#pragma unroll
    for (int t = 0; t < 9; t++) w[j][t] = bfload(&wf[CNN_W5 + t * CNN_C + chunk * 8 + j]);
  const int tiles_x = (W + CT_W - 1) / CT_W, tiles_y = (H + CT_H - 1) / CT_H;
  const int per_img = tiles_x * tiles_y;
  const int64_t ntiles = (int64_t)per_img * B;
  float h[2] = {0.0f, 0.0f};
  uint4 nxt = make_uint4(0u, 0u, 0u, 0u);            // the a5 piece (ReLU mask), one pass ahead
  if (blockIdx.x < ntiles) {
    const Tile t0 = tile_at(blockIdx.x, per_img, tiles_x);
    halo1_fetch(g, t0, H, W, h);
    nxt = piece_at(a5, t0, 0, pq, chunk, H, W);
  }
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tt = tile_at(tile, per_img, tiles_x);
    __syncthreads();                                 // the previous tile's reads are done
    halo1_store(sg, h);
    __syncthreads();
    const bool more = tile + gridDim.x < ntiles;
    const Tile tn = more ? tile_at(tile + gridDim.x, per_img, tiles_x) : tt;
    if (more) halo1_fetch(g, tn, H, W, h);
#pragma unroll 1
    for (int pass = 0; pass < END_PASSES; pass++) {
      const uint4 av = nxt;
      if (pass + 1 < END_PASSES) nxt = piece_at(a5, tt, pass + 1, pq, chunk, H, W);
      else if (more) nxt = piece_at(a5, tn, 0, pq, chunk, H, W);
      const int lp = pass * 64 + pq, ly = lp / CT_W, lx = lp % CT_W;
      const int gy = tt.ty0 + ly, gx = tt.tx0 + lx;
      if (gy >= H || gx >= W) continue;
      float acc[8];
#pragma unroll
      for (int j = 0; j < 8; j++) acc[j] = 0.f;
#pragma unroll
      for (int t = 0; t < 9; t++) {                  // pixel p - off(t) received tap t
        const float gv = sg[(ly + 2 - t / 3) * (CT_W + 2) + lx + 2 - t % 3];
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] = fmaf(w[j][t], gv, acc[j]);
      }
      const unsigned int u[4] = {av.x, av.y, av.z, av.w};
      unsigned int o[4];
#pragma unroll
      for (int e = 0; e < 4; e++)
        o[e] = pack_bf16x2(bf_lo(u[e]) > 0.f ? acc[2 * e] : 0.f,
                           bf_hi(u[e]) > 0.f ? acc[2 * e + 1] : 0.f);
      *reinterpret_cast<uint4*>(dz + (((size_t)tt.b * H + gy) * W + gx) * CNN_C + chunk * 8) =
          make_uint4(o[0], o[1], o[2], o[3]);
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

// Weight gradients of the 1-channel end layers (FP32 CUDA cores), as tile kernels on a
// persistent grid.  Both are sums over pixels of a 32-channel BF16 tensor times a shifted
// scalar field:
//   layer 5 (OUT): dw5[tap][ci] += sum_q a5[q][ci] * g[q - off(tap)]
//   layer 0 (IN):  dw0[co][tap] += sum_p dz0[p][co] * x[p + off(tap)]
// A CTA loops over 8 x 32 pixel tiles: the scalar field's haloed tile (zero outside the
// image) sits in shared memory, so the nine shifted values of a pixel are fixed offsets
// with no bounds tests; four threads share a pixel (8 channels each, one 16-byte load)
// and keep 9 x 8 partial sums across all their tiles, reduced over the CTA once.
template <bool OUT>
__global__ void __launch_bounds__(DW1_THREADS)
k_cnn_dw1(const bf16* __restrict__ t32, const float* __restrict__ f, float* __restrict__ dw,
          int H, int W, int B) {
  static_assert(DW1_THREADS == END_THREADS, "the halo helpers assume END_THREADS threads");
  __shared__ float sf[HALO1];
  const int chunk = threadIdx.x & 3, pq = threadIdx.x >> 2;     // 64 pixels per pass
  const int tiles_x = (W + CT_W - 1) / CT_W, tiles_y = (H + CT_H - 1) / CT_H;
  const int per_img = tiles_x * tiles_y;
  const int64_t ntiles = (int64_t)per_img * B;
  float acc[9][8];
#pragma unroll
  for (int t = 0; t < 9; t++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[t][j] = 0.f;
  float h[2] = {0.0f, 0.0f};
  uint4 nxt = make_uint4(0u, 0u, 0u, 0u);            // the 32-channel piece, one pass ahead
  if (blockIdx.x < ntiles) {
    const Tile t0 = tile_at(blockIdx.x, per_img, tiles_x);
    halo1_fetch(f, t0, H, W, h);
    nxt = piece_at(t32, t0, 0, pq, chunk, H, W);
  }
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile tt = tile_at(tile, per_img, tiles_x);
    __syncthreads();                                 // the previous tile's reads are done
    halo1_store(sf, h);
    __syncthreads();
    const bool more = tile + gridDim.x < ntiles;
    const Tile tn = more ? tile_at(tile + gridDim.x, per_img, tiles_x) : tt;
    if (more) halo1_fetch(f, tn, H, W, h);
#pragma unroll 1
    for (int pass = 0; pass < END_PASSES; pass++) {
      const uint4 tv = nxt;
      if (pass + 1 < END_PASSES) nxt = piece_at(t32, tt, pass + 1, pq, chunk, H, W);
      else if (more) nxt = piece_at(t32, tn, 0, pq, chunk, H, W);
      const int lp = pass * 64 + pq, ly = lp / CT_W, lx = lp % CT_W;
      if (tt.ty0 + ly >= H || tt.tx0 + lx >= W) continue;
      const unsigned int u[4] = {tv.x, tv.y, tv.z, tv.w};
      float a[8];
#pragma unroll
      for (int e = 0; e < 4; e++) { a[2 * e] = bf_lo(u[e]); a[2 * e + 1] = bf_hi(u[e]); }
#pragma unroll
      for (int t = 0; t < 9; t++) {
        const int dy = t / 3, dx = t % 3;
        // OUT: g at (y - (dy - 1), x - (dx - 1)); IN: x at (y + dy - 1, x + dx - 1)
        const float fv = OUT ? sf[(ly + 2 - dy) * (CT_W + 2) + lx + 2 - dx]
                             : sf[(ly + dy) * (CT_W + 2) + lx + dx];
#pragma unroll
        for (int j = 0; j < 8; j++) acc[t][j] = fmaf(fv, a[j], acc[t][j]);
      }
    }
  }
  if (OUT)
    dw1_commit(acc, chunk, [](int ci, int t) { return CNN_W5 + t * CNN_C + ci; }, dw);
  else
    dw1_commit(acc, chunk, [](int co, int t) { return CNN_W0 + co * CNN_TAPS + t; }, dw);
}

}  // namespace kc

namespace kc {

// weight gradient of a 32 -> 32 layer on the tensor cores (mma.sync m16n8k16, BF16 x BF16
// -> FP32): dw[co][tap][ci] += sum_p dz[p][co] * a[p + off(tap)][ci], i.e. for each tap the
// 32 x 32 product D = G^T X_tap with K = pixels.  A CTA loops over 8 x 32 pixel tiles
// (persistent grid) with the dz tile and the haloed input tile in shared memory (rows
// padded to 80 bytes: ldmatrix rows are conflict-free), two stages deep: the next tile's
// 16-byte cp.async copies (zero-filled outside the image) are in flight while the tensor
// cores work on the current one.  Warp w owns tap w: its A fragments are G^T
// (ldmatrix.trans of the pixel-major dz rows), its B fragments X_tap (ldmatrix.trans of the
// input rows at the tap-shifted halo pixels: every lane supplies its own row address, so
// the shift costs nothing).  The accumulators stay in registers across the CTA's tiles;
// one atomic per accumulator at the end.
constexpr int DW32_THREADS = 9 * 32;
constexpr int DW32_STAGE_A = HALO_PIX * CPAD;               // BF16 elements per stage
constexpr int DW32_STAGE_G = CT_H * CT_W * CPAD;
constexpr int DW32_SMEM = 2 * (DW32_STAGE_A + DW32_STAGE_G) * (int)sizeof(bf16);   // 95,360 B

__device__ __forceinline__ void ldmatrix_x4_trans(unsigned int (&r)[4], const void* smem) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros (src unread)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" :: "r"(d), "l"(src),
               "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" :: "n"(N) : "memory");
}

// issue the copies of one tile (haloed input rows and dz rows) into a stage
__device__ __forceinline__ void dw32_fetch(bf16* sA, bf16* sG, const bf16* __restrict__ dz,
                                           const bf16* __restrict__ a, int64_t tile,
                                           int per_img, int tiles_x, int H, int W) {
  const int b = (int)(tile / per_img), rem = (int)(tile % per_img);
  const int ty0 = (rem / tiles_x) * CT_H, tx0 = (rem % tiles_x) * CT_W;
  const size_t plane = (size_t)H * W;
  const bf16* ab = a + (size_t)b * plane * CNN_C;
  const bf16* gb = dz + (size_t)b * plane * CNN_C;
  for (int i = threadIdx.x; i < HALO_PIX * 4; i += blockDim.x) {
    const int pix = i >> 2, ch = i & 3;
    const int gy = ty0 + pix / (CT_W + 2) - 1, gx = tx0 + pix % (CT_W + 2) - 1;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    const bf16* src = in ? &ab[((size_t)gy * W + gx) * CNN_C + ch * 8] : ab;
    cp_async16(&sA[pix * CPAD + ch * 8], src, in ? 16 : 0);
  }
  for (int i = threadIdx.x; i < CT_H * CT_W * 4; i += blockDim.x) {
    const int pix = i >> 2, ch = i & 3;
    const int gy = ty0 + pix / CT_W, gx = tx0 + pix % CT_W;
    const bool in = gy < H && gx < W;                // pixels outside the image add nothing
    const bf16* src = in ? &gb[((size_t)gy * W + gx) * CNN_C + ch * 8] : gb;
    cp_async16(&sG[pix * CPAD + ch * 8], src, in ? 16 : 0);
  }
}

__global__ void __launch_bounds__(DW32_THREADS, 2)
k_cnn_dw32(const bf16* __restrict__ dz, const bf16* __restrict__ a, float* __restrict__ dw,
           int H, int W, int B) {
  extern __shared__ __align__(16) unsigned char dw32_smem[];
  bf16* const stA = reinterpret_cast<bf16*>(dw32_smem);                 // [2][DW32_STAGE_A]
  bf16* const stG = stA + 2 * DW32_STAGE_A;                              // [2][DW32_STAGE_G]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dy = warp / 3, dx = warp % 3;
  const int tiles_x = (W + CT_W - 1) / CT_W, tiles_y = (H + CT_H - 1) / CT_H;
  const int per_img = tiles_x * tiles_y;
  const int64_t ntiles = (int64_t)per_img * B;
  // ldmatrix row of this lane: matrix i = lane / 8, row r = lane % 8
  const int li = lane >> 3, lr = lane & 7;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.0f;
  int64_t tile = blockIdx.x;
  if (tile < ntiles) dw32_fetch(stA, stG, dz, a, tile, per_img, tiles_x, H, W);
  cp_async_commit();
  for (int it = 0; tile < ntiles; it++, tile += gridDim.x) {
    const int cur = it & 1;
    const int64_t next = tile + gridDim.x;
    if (next < ntiles)                                 // the other stage is free (barrier below)
      dw32_fetch(stA + (cur ^ 1) * DW32_STAGE_A, stG + (cur ^ 1) * DW32_STAGE_G, dz, a, next,
                 per_img, tiles_x, H, W);
    cp_async_commit();
    cp_async_wait<1>();                                // this tile's copies have landed
    __syncthreads();
    const bf16* sA = stA + cur * DW32_STAGE_A;
    const bf16* sG = stG + cur * DW32_STAGE_G;
#pragma unroll 2
    for (int ks = 0; ks < CT_H * 2; ks++) {            // 16 output pixels of one tile row
      const int py = ks >> 1, px0 = (ks & 1) * 16;
      // A = G^T (rows co, K = pixels): matrix i covers co + 8 (i & 1), pixels + 8 (i >= 2)
      const int pa = py * CT_W + px0 + lr + ((li >> 1) << 3);
      unsigned int a0[4], a1[4];
      ldmatrix_x4_trans(a0, &sG[pa * CPAD + (li & 1) * 8]);
      ldmatrix_x4_trans(a1, &sG[pa * CPAD + 16 + (li & 1) * 8]);
      // B = X_tap (K = pixels, N = ci): matrix i covers pixels + 8 (i & 1), ci + 8 (i >> 1)
      const int hb = (py + dy) * (CT_W + 2) + px0 + dx + lr + ((li & 1) << 3);
      unsigned int b0[4], b1[4];
      ldmatrix_x4_trans(b0, &sA[hb * CPAD + (li >> 1) * 8]);
      ldmatrix_x4_trans(b1, &sA[hb * CPAD + 16 + (li >> 1) * 8]);
      mma_bf16(acc[0][0], a0, b0[0], b0[1]);
      mma_bf16(acc[0][1], a0, b0[2], b0[3]);
      mma_bf16(acc[0][2], a0, b1[0], b1[1]);
      mma_bf16(acc[0][3], a0, b1[2], b1[3]);
      mma_bf16(acc[1][0], a1, b0[0], b0[1]);
      mma_bf16(acc[1][1], a1, b0[2], b0[3]);
      mma_bf16(acc[1][2], a1, b1[0], b1[1]);
      mma_bf16(acc[1][3], a1, b1[2], b1[3]);
    }
    __syncthreads();                                   // stage `cur` may be refilled next
  }
  cp_async_wait<0>();
  const int grp = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int co = mt * 16 + grp + (e >> 1) * 8, ci = nt * 8 + tq * 2 + (e & 1);
        atomicAdd(&dw[co * CNN_K + warp * CNN_C + ci], acc[mt][nt][e]);
      }
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
// persistent grid of a tile kernel: its resident CTAs on every SM, at most one per 8 x 32
// pixel tile
template <typename Kernel>
static int tile_grid(const kc_ctx* ctx, Kernel kernel, int threads, int smem, int H, int W,
                     int B) {
  const int64_t tiles = (int64_t)((W + CT_W - 1) / CT_W) * ((H + CT_H - 1) / CT_H) * B;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) !=
          cudaSuccess || occ < 1)
    occ = 1;
  const int64_t g = (int64_t)occ * ctx->num_sms;
  return (int)(tiles < g ? tiles : g);
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
  timing_begin(ctx, KID_OTHER);
  k_cnn_in<<<tile_grid(ctx, k_cnn_in, END_THREADS, 0, H, W, B), END_THREADS, 0, ctx->stream>>>(
      x, acts[0], wf, H, W, B);
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
  timing_begin(ctx, KID_OTHER);
  k_cnn_dw1<true><<<tile_grid(ctx, k_cnn_dw1<true>, DW1_THREADS, 0, H, W, B), DW1_THREADS, 0,
                    ctx->stream>>>(
      acts[4], g, dw, H, W, B);
  KC_LAUNCHED(ctx);
  timing_begin(ctx, KID_OTHER);
  k_cnn_out_bwd<<<tile_grid(ctx, k_cnn_out_bwd, END_THREADS, 0, H, W, B), END_THREADS, 0,
                  ctx->stream>>>(g, acts[4], dz[0], wf, H, W, B);
  KC_LAUNCHED(ctx);
  static std::atomic<unsigned long long> dw32_attr{0};
  KC_TRY(smem_attr_once(ctx, dw32_attr, k_cnn_dw32, DW32_SMEM, "weight gradient"));
  int cur = 0;
  for (int l = 3; l >= 0; l--) {      // 32 -> 32 layer l maps acts[l] -> acts[l+1]
    timing_begin(ctx, KID_OTHER);
    k_cnn_dw32<<<tile_grid(ctx, k_cnn_dw32, DW32_THREADS, DW32_SMEM, H, W, B), DW32_THREADS,
                 DW32_SMEM, ctx->stream>>>(
        dz[cur], acts[l], dw + CNN_WMID + l * CNN_WMID_SZ, H, W, B);
    KC_LAUNCHED(ctx);
    kc_status s = conv32(ctx, dz[cur], dz[cur ^ 1], wt + l * CNN_WMID_SZ, B, H, W, CONV_MASK,
                         acts[l]);
    if (s != KC_OK) return s;
    cur ^= 1;
  }
  timing_begin(ctx, KID_OTHER);
  k_cnn_dw1<false><<<tile_grid(ctx, k_cnn_dw1<false>, DW1_THREADS, 0, H, W, B), DW1_THREADS,
                     0, ctx->stream>>>(
      dz[cur], x, dw, H, W, B);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

// CTAs per sample of the loss kernels: about four per SM over all samples
static unsigned loss_grid(const kc_ctx* ctx, int64_t npix, int B) {
  const int64_t want = (4 * (int64_t)ctx->num_sms + B - 1) / B, blocks = (npix + 255) / 256;
  const int64_t g = blocks < want ? blocks : want;
  return (unsigned)(g < 1 ? 1 : g);
}

kc_status cnn_loss_grad(kc_ctx* ctx, const float* y, const float* e, double* sums, float* g,
                        int B, int64_t npix) {
  KC_CUDA(ctx, cudaMemsetAsync(sums, 0, 2 * B * sizeof(double), ctx->stream));
  dim3 grid(loss_grid(ctx, npix, B), B);
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
  dim3 grid(loss_grid(ctx, npix, B), B);
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
