// Fused DCGS2 reduction on the tensor cores (FP64 mode 2): C = Q^T w, S = Q^T v,
// beta = w^T w and s = w^T v (the single reduction of Algorithm 4) as exact integer dot products of
// fixed-point digit expansions, then the scalar step in the last CTA.
//
// Arithmetic (the Ozaki scheme on integer digits: Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 59, 2012; Ootomo, Ozaki and Yokota, IJHPCA 2024):
//   * a basis entry q becomes the integer X = round(q 2^56); w and v are scaled per chunk
//     of TX_R rows, Y = round(v 2^P) with P set by the chunk's largest exponent so that
//     |Y| < 2^58.  The w column of A (for beta and s) uses w's chunk scale less 1 bit,
//     so that every column of A has |X| < 2^57.
//   * X has six balanced 10-bit digits, X = sum_s d_s 1024^s, d_s in [-512, 511] (the
//     10-bit digits u_s of X + 512 sum_s 1024^s, less 512); Y has twelve balanced 5-bit
//     digits d_t in [-16, 15].
//   * the MMA operands are FP16 integers: A holds 1024 + u_s = 1536 + d_s (bit pattern
//     0x6400 | u_s: one OR), B holds d_t.  Over one chunk of 512 rows
//     D_st = sum_i (1536 + d_s,i) d_t,i stays within 2^24 in magnitude, so the FP32
//     accumulator in tensor memory holds it exactly; D_st - 1536 sum_i d_t,i is the digit
//     product sum, and sum_s,t 1024^s 32^t of those is the chunk's exact integer X^T Y
//     (taken mod 2^128, exact while |X^T Y| < 2^127: 512 2^57 2^58 = 2^124).  The
//     offset forms stay below 2^60: X + 512 sum 1024^s and Y + 16 sum 32^t.
// The roundings are the fixed-point conversions (2^-57 absolute for q, 2^-59 of the
// chunk's largest |v| for v) and one FP64 rounding of each chunk's exact sum; there is no
// FP64 arithmetic per basis entry, which is what bounds the FP64 kernels on this GPU.
// A basis entry of magnitude >= 2 (a column far from unit norm) or a non-finite operand
// sets KC_ERR_NONFINITE.
//
// Layout: per chunk of TX_R rows, B (N = 32: twelve w digits, twelve v digits, zero rows)
// in shared memory; per stage of TX_KS rows, A tiles of 128 rows = 21 columns x 6 digits
// and two more rows, at most TX_MT tiles (k + 1 <= 63 columns).  Row 126 of tile 0 holds
// FP16 ones, so its accumulator row is sum_i d_t,i of w and v (the bias to remove).  Both are K-major core
// matrices of 8 rows x 16 bytes without swizzle; the K-adjacent slabs are padded by 16
// bytes so that the 4-byte digit-pair stores of a warp hit 32 distinct banks.  One CTA
// per SM, 16 warps: warp w converts columns w, w + 16, ... (lane l: rows 2l, 2l + 1 of
// the stage); thread 0 issues the MMAs of a stage into the chunk's accumulators (two
// sets, 4 x 32 tensor-memory columns each); warp w drains tile w / 4, lanes of quarter
// w % 4, one chunk behind.  Every wait is bounded (KC_ERR_TIMEOUT, no fault).
//
// Included at the end of kc_ortho.cu (it uses that file's reduction epilogue).
#pragma once

#include "kc_internal.cuh"
#include "kc_tcgen05.cuh"

namespace kc {

constexpr int TX_THREADS = 512;
constexpr int TX_R = 512;                       // rows per chunk (one exact accumulation)
constexpr int TX_KS = 64;                       // rows per stage
constexpr int TX_NST = TX_R / TX_KS;            // stages per chunk
constexpr int TX_NA = 6, TX_BA = 10;            // A digits: six of 10 bits
constexpr int TX_NB = 12, TX_BB = 5;            // B digits: twelve of 5 bits
constexpr int TX_CPT = 128 / TX_NA;             // basis columns per 128-row A tile (21)
constexpr int TX_MT = 3;                        // A tiles
constexpr int TX_MAXC = TX_CPT * TX_MT;         // columns (k + 1) the kernel takes
constexpr int TX_NCW = (TX_MAXC + TX_THREADS / 32 - 1) / (TX_THREADS / 32);   // columns per warp
constexpr int TX_LBO_A = 128 * 16 + 16;         // bytes between K-adjacent slabs of A
constexpr int TX_ATILE = (TX_KS / 8) * TX_LBO_A;
constexpr int TX_ASTAGE = TX_MT * TX_ATILE;
constexpr int TX_LBO_B = 32 * 16 + 16;          // bytes between K-adjacent slabs of B
constexpr int TX_BTILE = (TX_R / 8) * TX_LBO_B;
constexpr int TX_NAB = 3;                      // A stage buffers
constexpr int TX_SP = TX_MT * 128 * 4 * 8;      // drained sums: tile x row x (w lo, hi, v lo, hi)
constexpr int TX_PB = 1080;                     // Y = v 2^(TX_PB - e_max): |Y| < 2^58
constexpr size_t TX_SMEM = 128 + TX_NAB * (size_t)TX_ASTAGE + 2 * (size_t)TX_BTILE;
constexpr int TX_TMEM_COLS = 256;               // two chunks x four tiles x 32 columns
constexpr int TX_QP = 56;                       // fixed-point scale of basis entries
constexpr int TX_WSHIFT = 1;                    // w as a column of A: |X| < 2^57 like q
constexpr unsigned long long TX_OFFA = 512ull * 0x0004010040100401ull;  // 512 sum_s 1024^s
constexpr unsigned long long TX_OFFB = 16ull * 0x0084210842108421ull;   // 16 sum_t 32^t
constexpr uint32_t TX_IDESC = idesc_f16_f32(128, 32);
static_assert(TX_ATILE % 16 == 0 && TX_BTILE % 16 == 0, "descriptor addresses are 16-byte units");
static_assert(TX_CPT * TX_NA <= 128 && 2 * TX_NB <= 32, "tile shapes");
static_assert(TX_R * 2047 * 16 <= (1 << 24), "exact FP32 accumulation over a chunk");
static_assert(TX_SMEM + 12 * 1024 <= 227 * 1024, "shared memory (with the static part)");
static_assert(TX_CPT * TX_NA <= 126, "row 126 of tile 0 is the row of ones");
static_assert(TX_SP <= TX_BTILE, "drained sums live in the drained chunk's B buffer");

__device__ __forceinline__ int tx_expo(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}

// a >> n, 0 for n >= 64 (the PTX shift clamps its count)
__device__ __forceinline__ unsigned long long tx_shr(unsigned long long a, unsigned int n) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(a), "r"(n));
  return r;
}

// off + round(v 2^P) in two's complement (|v| 2^P rounded half up), branch-free: the
// significand is aligned to bit 63 and shifted right once; the caller keeps |v| 2^P below
// 2^62, so the shift is at least 2.
__device__ __forceinline__ unsigned long long tx_fixed(double v, int P, unsigned long long off) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int e = (int)(bits >> 52) & 0x7FF;
  const unsigned long long mm = (bits << 11) | (e ? (1ull << 63) : 0ull);
  const int n = 1086 - P - (e ? e : 1);
  const unsigned long long a = (tx_shr(mm, (unsigned int)(n - 1)) + 1ull) >> 1;
  return (long long)bits < 0 ? off - a : off + a;
}

// A operand: FP16 pair of 1024 + u_s for 10-bit digit s of two offset integers
__device__ __forceinline__ unsigned int tx_adig(unsigned long long a, unsigned long long b,
                                                int s) {
  const unsigned int da = (unsigned int)(a >> (TX_BA * s)) & 1023u;
  const unsigned int db = (unsigned int)(b >> (TX_BA * s)) & 1023u;
  return 0x64006400u | da | (db << 16);
}

// B operand: FP16 bits of u - 16 (exact: |u - 16| <= 16)
__device__ __forceinline__ unsigned int tx_bdig(unsigned int u) {
  return (unsigned int)__half_as_ushort(__float2half_rn((float)((int)u - 16)));
}

__device__ __forceinline__ void tx_flag(int* s_flag) { atomicExch(s_flag, 1); }

__global__ void __launch_bounds__(TX_THREADS, 1)
k_reduce_tcx(const double* __restrict__ Q, int64_t ldq, int k, const double* __restrict__ x,
             const double* __restrict__ y, int64_t m, double* __restrict__ partials,
             unsigned int* __restrict__ counter, Scalars* __restrict__ sc, StepArgs sa) {
  if (sc->stop) return;
  extern __shared__ unsigned char tx_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tx_raw) + 127) & ~(uintptr_t)127);
  unsigned char* sA = base;                                   // TX_NAB stage buffers
  unsigned char* sB = base + TX_NAB * TX_ASTAGE;              // two chunk buffers
  __shared__ double s_acc[TX_MAXC][2];
  __shared__ int s_bsum[2 * TX_NB];             // sum_i d_t,i of the drained chunk (w, v)
  __shared__ unsigned int s_blut[1024];         // FP16 pair of two 5-bit digits, by u0 | u1 << 5
  __shared__ int s_emax[2][2];
  __shared__ unsigned long long bar_a[TX_NAB], bar_c[2];
  __shared__ unsigned int s_tmem;
  __shared__ int s_err, s_range;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols = k + 1, ntile = (ncols + TX_CPT - 1) / TX_CPT;
  const int64_t nchunk = (m + TX_R - 1) / TX_R;

  for (int i = tid; i < (TX_NAB * TX_ASTAGE + 2 * TX_BTILE) / 16; i += TX_THREADS)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < TX_MAXC * 2; i += TX_THREADS) (&s_acc[0][0])[i] = 0.0;
  for (int i = tid; i < 1024; i += TX_THREADS) s_blut[i] = tx_bdig(i & 31) | (tx_bdig(i >> 5) << 16);
  __syncthreads();
  // row 126 of tile 0 holds ones (FP16 1.0): its accumulator row is sum_i d_t,i of w and v
  for (int i = tid; i < TX_NAB * (TX_KS / 8); i += TX_THREADS)
    *reinterpret_cast<uint4*>(base + (i / (TX_KS / 8)) * TX_ASTAGE + (i % (TX_KS / 8)) * TX_LBO_A +
                              126 * 16) = make_uint4(0x3C003C00u, 0x3C003C00u, 0x3C003C00u, 0x3C003C00u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(smem_u32(&s_tmem)), "r"(TX_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TX_NAB; i++) mbar_init(&bar_a[i], 1);
    for (int i = 0; i < 2; i++) mbar_init(&bar_c[i], 1);
    fence_barrier_init();
    s_err = 0;
    s_range = 0;
  }
  fence_async_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned int tmem = s_tmem;

  // drain chunk nl (buffer nl & 1): exact digit sums -> one FP64 value per column and vector
  auto drain = [&](int nl) {
    const int bd = nl & 1;
    // the chunk's B buffer is idle from here until chunk nl + 2: it holds the drained sums
    long long* sP = reinterpret_cast<long long*>(sB + bd * TX_BTILE);
    if (tid == 0 && !mbar_wait(&bar_c[bd], (unsigned int)((nl >> 1) & 1), WAIT_LIMIT))
      tx_flag(&s_err);
    __syncthreads();
    tc_fence_after();
    const int tau = warp >> 2, qd = warp & 3;
    float D[32];
    if (tau < ntile) {
      tc_ld32(tmem + (unsigned int)(bd * 128 + tau * 32) + ((unsigned int)(qd * 32) << 16), D);
      if (tau == 0 && qd * 32 + lane == 126) {
#pragma unroll
        for (int t = 0; t < 2 * TX_NB; t++) s_bsum[t] = __float2int_rn(D[t]);
      }
    }
    __syncthreads();
    if (tau < ntile) {
      const int r = qd * 32 + lane, c = tau * TX_CPT + r / TX_NA;
      if (r < TX_CPT * TX_NA && c < ncols) {
#pragma unroll
        for (int vec = 0; vec < 2; vec++) {
          long long lo = 0, hi = 0;
#pragma unroll
          for (int t = 0; t < TX_NB; t++) {
            // D is an integer of magnitude <= 2^24 (exact in FP32 and through the conversion)
            const int di = __float2int_rn(D[TX_NB * vec + t]) - 1536 * s_bsum[TX_NB * vec + t];
            if (t < 7) lo += (long long)di * (1ll << (TX_BB * t));
            else hi += (long long)di * (1ll << (TX_BB * (t - 7)));
          }
          long long* p = sP + ((int64_t)(tau * 128 + r) * 4 + 2 * vec);
          p[0] = lo;
          p[1] = hi;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    if (tid < 2 * ncols) {
      const int c = tid >> 1, vec = tid & 1, tau = c / TX_CPT, j = c % TX_CPT;
      unsigned __int128 V = 0;
#pragma unroll
      for (int s = 0; s < TX_NA; s++) {
        const long long* p = sP + ((int64_t)(tau * 128 + TX_NA * j + s) * 4 + 2 * vec);
        V += (unsigned __int128)(__int128)p[0] << (TX_BA * s);
        V += (unsigned __int128)(__int128)p[1] << (7 * TX_BB + TX_BA * s);
      }
      const __int128 Vs = (__int128)V;
      const double dv = (double)(long long)(Vs >> 64) * 18446744073709551616.0 +
                        (double)(unsigned long long)V;
      const int py = TX_PB - s_emax[bd][vec];
      const int px = c < k ? TX_QP : TX_PB - TX_WSHIFT - s_emax[bd][0];
      s_acc[c][vec] += ldexp(dv, -(px + py));
    }
  };

  // A stage's columns are loaded into registers one stage ahead of their conversion, and
  // bulk L2 prefetches run three stages ahead; w and v of the next chunk are loaded a
  // chunk ahead.
  auto load_stage = [&](double2 (&dst)[TX_NCW], int64_t chk, int st) {
    const int64_t row = chk * TX_R + st * TX_KS + 2 * lane;
#pragma unroll
    for (int i = 0; i < TX_NCW; i++) {
      const int c = warp + (TX_THREADS / 32) * i;
      double2 v = make_double2(0.0, 0.0);
      if (c < ncols && chk < nchunk) {
        const double* col = c < k ? Q + (int64_t)c * ldq : x;
        if (row + 1 < m) v = __ldg(reinterpret_cast<const double2*>(col + row));
        else if (row < m) v.x = __ldg(col + row);
      }
      dst[i] = v;
    }
  };
  auto prefetch_stage = [&](int64_t chk, int st) {
    if (st >= TX_NST) { chk += gridDim.x; st -= TX_NST; }
    const int64_t row = chk * TX_R + st * TX_KS;
    if (lane != 0 || chk >= nchunk || row >= m) return;
    const int64_t nrow = m - row < TX_KS ? m - row : TX_KS;
    const unsigned int bytes = (unsigned int)(nrow * 8) & ~15u;
    if (bytes == 0) return;
#pragma unroll
    for (int i = 0; i < TX_NCW; i++) {
      const int c = warp + (TX_THREADS / 32) * i;
      if (c >= ncols) break;
      const double* col = c < k ? Q + (int64_t)c * ldq : x;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(col + row), "r"(bytes)
                   : "memory");
    }
  };
  const int vec = tid >> 8, p = tid & 255;         // B: vector, row pair
  auto load_vecs = [&](double& o0, double& o1, int64_t chk) {
    o0 = 0.0;
    o1 = 0.0;
    if (chk >= nchunk) return;
    const double* src = vec ? y : x;
    const int64_t row = chk * TX_R + 2 * p;
    if (row + 1 < m) {
      const double2 t2 = __ldg(reinterpret_cast<const double2*>(src + row));
      o0 = t2.x;
      o1 = t2.y;
    } else if (row < m) {
      o0 = __ldg(src + row);
    }
  };

  int64_t g = 0;                   // stages issued by this CTA
  int nloc = 0;                    // chunks begun by this CTA
  int last_sb = -1;
  unsigned int last_par = 0;
  double2 cur[TX_NCW];
  double nb0, nb1;
  load_vecs(nb0, nb1, blockIdx.x);
  load_stage(cur, blockIdx.x, 0);
  for (int d = 1; d < 3; d++) prefetch_stage(blockIdx.x, d);
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x, nloc++) {
    const int b = nloc & 1;
    // ---- B: digits of w and v over the chunk (threads 0-255: vector, row pair) ----
    if (tid < 2) s_emax[b][tid] = 0;
    __syncthreads();
    const double b0 = nb0, b1 = nb1;
    load_vecs(nb0, nb1, ch + gridDim.x);
    {
      int e = max(tx_expo(b0), tx_expo(b1));
      e = __reduce_max_sync(0xffffffffu, e);
      if (lane == 0) atomicMax(&s_emax[b][vec], e);
    }
    __syncthreads();
    {
      const int E = s_emax[b][vec];
      if (E == 0x7FF) tx_flag(&s_range);
      const int P = TX_PB - E;
      const unsigned long long a0 = tx_fixed(b0, P, TX_OFFB);
      const unsigned long long a1 = tx_fixed(b1, P, TX_OFFB);
      // row n of a slab sits at 16 n bytes (core matrices of 8 rows x 16 bytes, SBO 128)
      unsigned char* bt = sB + b * TX_BTILE + (p >> 2) * TX_LBO_B + (p & 3) * 4 + 16 * TX_NB * vec;
#pragma unroll
      for (int t = 0; t < TX_NB; t++) {
        const unsigned int u0 = (unsigned int)(a0 >> (TX_BB * t)) & 31u;
        const unsigned int u1 = (unsigned int)(a1 >> (TX_BB * t)) & 31u;
        *reinterpret_cast<unsigned int*>(bt + 16 * t) = s_blut[u0 | (u1 << 5)];
      }
      fence_async_shared();
    }
    const int pw = TX_PB - TX_WSHIFT - s_emax[b][0];   // (read after the barrier above)
    // ---- the chunk's stages ----
    for (int st = 0; st < TX_NST; st++, g++) {
      const int sb = (int)(g % TX_NAB);
      double2 nxt[TX_NCW];
      if (st + 1 < TX_NST) load_stage(nxt, ch, st + 1);
      else load_stage(nxt, ch + gridDim.x, 0);
      prefetch_stage(ch, st + 3);
      unsigned char* at = sA + sb * TX_ASTAGE;
#pragma unroll
      for (int i = 0; i < TX_NCW; i++) {
        const int c = warp + (TX_THREADS / 32) * i;
        if (c >= ncols) break;
        double v0 = cur[i].x, v1 = cur[i].y;
        if (c < k && max(tx_expo(v0), tx_expo(v1)) >= 1024) {   // |q| >= 2 or not finite
          tx_flag(&s_range);
          v0 = 0.0;
          v1 = 0.0;
        }
        const int P = c < k ? TX_QP : pw;
        const unsigned long long a0 = tx_fixed(v0, P, TX_OFFA);
        const unsigned long long a1 = tx_fixed(v1, P, TX_OFFA);
        const int tau = c / TX_CPT, j = c % TX_CPT;
        // row r = 6 j + s of a slab sits at 16 r bytes
        unsigned char* tb = at + tau * TX_ATILE + (lane >> 2) * TX_LBO_A + (lane & 3) * 4 +
                            16 * TX_NA * j;
#pragma unroll
        for (int s = 0; s < TX_NA; s++)
          *reinterpret_cast<unsigned int*>(tb + 16 * s) = tx_adig(a0, a1, s);
      }
#pragma unroll
      for (int i = 0; i < TX_NCW; i++) cur[i] = nxt[i];
      fence_async_shared();
      // the buffer of the next stage is free once the MMAs of its previous use are done
      if (tid == 0 && g + 1 >= TX_NAB &&
          !mbar_wait(&bar_a[(g + 1) % TX_NAB], (unsigned int)(((g + 1) / TX_NAB - 1) & 1),
                     WAIT_LIMIT))
        tx_flag(&s_err);
      tc_fence_before();
      __syncthreads();
      if (s_err) break;
      if (tid == 0) {
        tc_fence_after();
        const unsigned int abase = smem_u32(at), bbase = smem_u32(sB + b * TX_BTILE);
        for (int tau = 0; tau < ntile; tau++)
#pragma unroll
          for (int kk = 0; kk < TX_KS / 16; kk++) {
            const unsigned long long ad =
                umma_desc(abase + tau * TX_ATILE + 2 * kk * TX_LBO_A, TX_LBO_A, 128);
            const unsigned long long bdsc =
                umma_desc(bbase + (st * (TX_KS / 8) + 2 * kk) * TX_LBO_B, TX_LBO_B, 128);
            tc_mma(tmem + (unsigned int)(b * 128 + tau * 32), ad, bdsc, TX_IDESC,
                   (st | kk) ? 1u : 0u);
          }
        tc_commit(&bar_a[sb]);
        if (st == TX_NST - 1) tc_commit(&bar_c[b]);
        last_sb = sb;
        last_par = (unsigned int)((g / TX_NAB) & 1);
      }
      if (st == 1 && nloc >= 1) drain(nloc - 1);
    }
    __syncthreads();
    if (s_err) break;
  }
  if (!s_err && nloc >= 1) drain(nloc - 1);
  // every MMA issued has completed before the tensor memory is freed
  if (tid == 0 && last_sb >= 0) (void)mbar_wait(&bar_a[last_sb], last_par, WAIT_LIMIT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 ::"r"(tmem), "r"(TX_TMEM_COLS) : "memory");
  if (tid == 0) {
    if (s_err) atomicCAS(&sc->status, (int)KC_OK, (int)KC_ERR_TIMEOUT);
    else if (s_range) atomicCAS(&sc->status, (int)KC_OK, (int)KC_ERR_NONFINITE);
  }
  double* pp = partials + (int64_t)blockIdx.x * PSTRIDE;
  for (int c = tid; c < ncols; c += TX_THREADS) {
    const int i = c < k ? 2 * c : 2 * k;         // beta -> [2k], s -> [2k + 1]
    pp[i] = s_acc[c][0];
    pp[i + 1] = s_acc[c][1];
  }
  if (!last_cta(counter)) return;
  reduce_epilogue(partials, k, 2, sc, EPI_DCGS2, sa);
}

// ---- host side --------------------------------------------------------------------------

bool reduce_tcx_supported(int k, int64_t m, const void* Q, int64_t ldq, const void* x,
                          const void* y) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return k >= 0 && k + 1 <= TX_MAXC && m >= 1 && (ldq & 1) == 0 && al(Q) && al(x) && al(y);
}

kc_status launch_reduce_tcx(kc_ctx* ctx, const double* Q, int64_t ldq, int k, const double* x,
                            const double* y, int64_t m, const StepArgs& sa) {
  static std::atomic<unsigned long long> attr_done{0};
  KC_TRY(smem_attr_once(ctx, attr_done, k_reduce_tcx, (int)TX_SMEM, "reduce"));
  const int64_t nchunk = (m + TX_R - 1) / TX_R;
  const int grid = (int)(nchunk < ctx->num_sms ? nchunk : ctx->num_sms);
  k_reduce_tcx<<<grid, TX_THREADS, TX_SMEM, ctx->stream>>>(Q, ldq, k, x, y, m, ctx->partials,
                                                          ctx->counters, ctx->scal, sa);
  return KC_OK;
}

}  // namespace kc
