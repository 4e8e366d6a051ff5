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
// in shared memory; per stage of TX_KS rows, A tiles of 128 rows: each 32-row quarter of a
// tile holds TX_CPQ columns x 6 digits (row 32 qd + 6 jj + s for column 20 tau + 5 qd + jj,
// digit s) and two spare rows, so that the six digit rows of a column sit in one warp's
// tensor-memory lanes.  Row 30 of tile 0 holds FP16 ones: its accumulator row is
// sum_i d_t,i of w and v (the bias to remove).  Both operands are K-major core matrices
// of 8 rows x 16 bytes without swizzle; the K-adjacent slabs are padded by 16 bytes so
// that the 4-byte digit-pair stores of a warp hit 32 distinct banks.
//
// Warp roles (one CTA per SM, persistent over chunks), all hand-offs on mbarriers with
// bounded waits (KC_ERR_TIMEOUT, never a hang):
//   warps 0..TX_PW-1   A producers: load their columns' rows of a stage (one stage ahead
//                      in registers, bulk L2 prefetches three ahead), convert to digits
//                      into the stage's A buffer (a ring of TX_NAB), arrive on a_full;
//   warps TX_PW..+3    B producers and drain: the digits of w and v one chunk ahead (the
//                      chunk's largest exponents through shared memory), then the drain of
//                      the previous chunk's accumulators (tcgen05.ld, bias removal, digit
//                      combination across the six lanes of a column by shuffles, one FP64
//                      rounding per chunk) into per-column FP64 sums;
//   warp TX_PW+4       MMA issue (one thread): per stage and tile four MMAs of K = 16 into
//                      the chunk's accumulators (two sets in tensor memory), commits that
//                      free the A buffer and, at a chunk's end, publish its accumulators.
//
// Included at the end of kc_ortho.cu (it uses that file's reduction epilogue).
#pragma once

#include "kc_internal.cuh"
#include "kc_tcgen05.cuh"

namespace kc {

constexpr int TX_PW = 12;                       // A producer warps
constexpr int TX_DW = 4;                        // B producer / drain warps
constexpr int TX_THREADS = 32 * (TX_PW + TX_DW + 1);
constexpr int TX_R = 512;                       // rows per chunk (one exact accumulation)
constexpr int TX_KS = 64;                       // rows per stage
constexpr int TX_NST = TX_R / TX_KS;            // stages per chunk
constexpr int TX_NA = 6, TX_BA = 10;            // A digits: six of 10 bits
constexpr int TX_NB = 12, TX_BB = 5;            // B digits: twelve of 5 bits
constexpr int TX_CPQ = 5;                       // basis columns per 32-row quarter of a tile
constexpr int TX_CPT = 4 * TX_CPQ;              // basis columns per 128-row A tile (20)
constexpr int TX_MT = 3;                        // A tiles
constexpr int TX_MAXC = TX_CPT * TX_MT;         // columns (k + 1) the kernel takes
constexpr int TX_NCW = (TX_MAXC + TX_PW - 1) / TX_PW;   // columns per producer warp
constexpr int TX_ONES = 30;                     // row of tile 0 that holds the ones
constexpr int TX_LBO_A = 128 * 16 + 16;         // bytes between K-adjacent slabs of A
constexpr int TX_ATILE = (TX_KS / 8) * TX_LBO_A;
constexpr int TX_ASTAGE = TX_MT * TX_ATILE;
constexpr int TX_LBO_B = 32 * 16 + 16;          // bytes between K-adjacent slabs of B
constexpr int TX_BTILE = (TX_R / 8) * TX_LBO_B;
constexpr int TX_NAB = 3;                      // A stage buffers
constexpr int TX_PB = 1080;                     // Y = v 2^(TX_PB - e_max): |Y| < 2^58
constexpr size_t TX_SMEM = 128 + TX_NAB * (size_t)TX_ASTAGE + 2 * (size_t)TX_BTILE;
constexpr int TX_TMEM_COLS = 256;               // two chunks x four tiles x 32 columns
constexpr int TX_QP = 56;                       // fixed-point scale of basis entries
constexpr int TX_WSHIFT = 1;                    // w as a column of A: |X| < 2^57 like q
constexpr unsigned long long TX_OFFA = 512ull * 0x0004010040100401ull;  // 512 sum_s 1024^s
constexpr unsigned long long TX_OFFB = 16ull * 0x0084210842108421ull;   // 16 sum_t 32^t
constexpr uint32_t TX_IDESC = idesc_f16_f32(128, 32);
static_assert(TX_ATILE % 16 == 0 && TX_BTILE % 16 == 0, "descriptor addresses are 16-byte units");
static_assert(TX_CPQ * TX_NA <= 30 && 2 * TX_NB <= 32, "tile shapes");
static_assert(TX_R * 2047 * 16 <= (1 << 24), "exact FP32 accumulation over a chunk");
static_assert(TX_SMEM + 12 * 1024 <= 227 * 1024, "shared memory (with the static part)");
static_assert(TX_DW == 4, "the drain warps cover the four 32-lane quarters of tensor memory");

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
__device__ __forceinline__ int tx_read(const int* s_flag) {
  return *reinterpret_cast<const volatile int*>(s_flag);
}

// A wait whose outcome the whole warp shares: lane 0 polls (bounded), the result is
// broadcast, so the warp stays converged whatever the outcome.
__device__ __forceinline__ bool warp_wait(unsigned long long* bar, unsigned int parity) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, WAIT_LIMIT) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// A-tile row of column c's digit s: tile c / 20, quarter (c % 20) / 5, slot c % 5
__device__ __forceinline__ int tx_arow(int c, int s) {
  const int jl = c % TX_CPT;
  return 32 * (jl / TX_CPQ) + TX_NA * (jl % TX_CPQ) + s;
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

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
  __shared__ unsigned int s_blut[1024];         // FP16 pair of two 5-bit digits, by u0 | u1 << 5
  __shared__ int s_emax[4][2];                  // largest exponents of w, v, by chunk mod 4
  __shared__ int s_bsum[2 * TX_NB];             // sum_i d_t,i of the drained chunk (w, v)
  __shared__ unsigned long long a_full[TX_NAB], a_empty[TX_NAB], b_full[2], c_done[2],
      t_free[2];
  __shared__ unsigned int s_tmem;
  __shared__ int s_err, s_range, s_dok[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols = k + 1, ntile = (ncols + TX_CPT - 1) / TX_CPT;
  const int64_t nchunk = (m + TX_R - 1) / TX_R;
  const int nloc = (int)((nchunk - blockIdx.x + gridDim.x - 1) / gridDim.x);   // >= 1
  const int MMAW = TX_PW + TX_DW;

  for (int i = tid; i < (TX_NAB * TX_ASTAGE + 2 * TX_BTILE) / 16; i += TX_THREADS)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < 1024; i += TX_THREADS) s_blut[i] = tx_bdig(i & 31) | (tx_bdig(i >> 5) << 16);
  __syncthreads();
  // row TX_ONES of tile 0 holds ones (FP16 1.0) in every stage buffer
  for (int i = tid; i < TX_NAB * (TX_KS / 8); i += TX_THREADS)
    *reinterpret_cast<uint4*>(base + (i / (TX_KS / 8)) * TX_ASTAGE + (i % (TX_KS / 8)) * TX_LBO_A +
                              TX_ONES * 16) = make_uint4(0x3C003C00u, 0x3C003C00u, 0x3C003C00u, 0x3C003C00u);
  if (warp == MMAW) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(smem_u32(&s_tmem)), "r"(TX_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TX_NAB; i++) {
      mbar_init(&a_full[i], TX_PW);
      mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&b_full[i], TX_DW);
      mbar_init(&c_done[i], 1);
      mbar_init(&t_free[i], TX_DW);
    }
    fence_barrier_init();
    s_err = 0;
    s_range = 0;
  }
  fence_async_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned int tmem = s_tmem;
  double acc[TX_MT][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};   // drain lanes: column sums

  if (warp < TX_PW) {
    // ---------------- A producers ----------------
    auto load_stage = [&](double2 (&dst)[TX_NCW], int cl, int st) {
      const int64_t chk = blockIdx.x + (int64_t)cl * gridDim.x;
      const int64_t row = chk * TX_R + st * TX_KS + 2 * lane;
#pragma unroll
      for (int i = 0; i < TX_NCW; i++) {
        const int c = warp + TX_PW * i;
        double2 v = make_double2(0.0, 0.0);
        if (c < ncols && cl < nloc) {
          const double* col = c < k ? Q + (int64_t)c * ldq : x;
          if (row + 1 < m) v = __ldg(reinterpret_cast<const double2*>(col + row));
          else if (row < m) v.x = __ldg(col + row);
        }
        dst[i] = v;
      }
    };
    auto prefetch_stage = [&](int cl, int st) {
      cl += st / TX_NST;
      st %= TX_NST;
      const int64_t chk = blockIdx.x + (int64_t)cl * gridDim.x;
      const int64_t row = chk * TX_R + st * TX_KS;
      if (lane != 0 || cl >= nloc || row >= m) return;
      const int64_t nrow = m - row < TX_KS ? m - row : TX_KS;
      const unsigned int bytes = (unsigned int)(nrow * 8) & ~15u;
      if (bytes == 0) return;
#pragma unroll
      for (int i = 0; i < TX_NCW; i++) {
        const int c = warp + TX_PW * i;
        if (c >= ncols) break;
        const double* col = c < k ? Q + (int64_t)c * ldq : x;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(col + row), "r"(bytes)
                     : "memory");
      }
    };
    const bool owns_w = (k % TX_PW) == warp;       // the warp that converts the w column
    double2 cur[TX_NCW];
    load_stage(cur, 0, 0);
    prefetch_stage(0, 1);
    prefetch_stage(0, 2);
    int64_t g = 0;
    bool stop = false;
    for (int cl = 0; cl < nloc && !stop; cl++) {
      int pw = 0;
      if (owns_w) {                                  // w's chunk scale comes with B
        if (!warp_wait(&b_full[cl & 1], (unsigned int)((cl >> 1) & 1))) {
          if (lane == 0) tx_flag(&s_err);
          break;
        }
        pw = TX_PB - TX_WSHIFT - s_emax[cl & 3][0];
      }
      for (int st = 0; st < TX_NST; st++, g++) {
        const int sb = (int)(g % TX_NAB);
        double2 nxt[TX_NCW];
        if (st + 1 < TX_NST) load_stage(nxt, cl, st + 1);
        else load_stage(nxt, cl + 1, 0);
        prefetch_stage(cl, st + 3);
        if (g >= TX_NAB && !warp_wait(&a_empty[sb], (unsigned int)((g / TX_NAB - 1) & 1))) {
          if (lane == 0) tx_flag(&s_err);
          stop = true;
          break;
        }
        unsigned char* at = sA + sb * TX_ASTAGE;
#pragma unroll
        for (int i = 0; i < TX_NCW; i++) {
          const int c = warp + TX_PW * i;
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
          // row r of a slab sits at 16 r bytes; lane l holds K positions 2l, 2l + 1
          unsigned char* tb = at + (c / TX_CPT) * TX_ATILE + (lane >> 2) * TX_LBO_A +
                              (lane & 3) * 4 + 16 * tx_arow(c, 0);
#pragma unroll
          for (int s = 0; s < TX_NA; s++)
            *reinterpret_cast<unsigned int*>(tb + 16 * s) = tx_adig(a0, a1, s);
        }
#pragma unroll
        for (int i = 0; i < TX_NCW; i++) cur[i] = nxt[i];
        fence_async_shared();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[sb]);
        if (__shfl_sync(0xffffffffu, tx_read(&s_err), 0)) {
          stop = true;
          break;
        }
      }
    }
  } else if (warp < MMAW) {
    // ---------------- B producers and drain ----------------
    const int dw = warp - TX_PW, dt = tid - 32 * TX_PW;        // 0..3, 0..127
    auto produce_b = [&](int cl) {
      const int64_t chk = blockIdx.x + (int64_t)cl * gridDim.x;
      const int slot = cl & 3, b = cl & 1;
      double vals[8];
      int emx[2] = {0, 0};
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int item = dt + 128 * u;                // vector (item >> 8), row pair
        const int vec = item >> 8, p = item & 255;
        const double* src = vec ? y : x;
        const int64_t row = chk * TX_R + 2 * p;
        double o0 = 0.0, o1 = 0.0;
        if (row + 1 < m) {
          const double2 t2 = __ldg(reinterpret_cast<const double2*>(src + row));
          o0 = t2.x;
          o1 = t2.y;
        } else if (row < m) {
          o0 = __ldg(src + row);
        }
        vals[2 * u] = o0;
        vals[2 * u + 1] = o1;
        emx[vec] = max(emx[vec], max(tx_expo(o0), tx_expo(o1)));
      }
      if (dt < 2) s_emax[slot][dt] = 0;
      named_sync(1, 32 * TX_DW);
#pragma unroll
      for (int vec = 0; vec < 2; vec++) {
        const int e = __reduce_max_sync(0xffffffffu, emx[vec]);
        if (lane == 0) atomicMax(&s_emax[slot][vec], e);
      }
      named_sync(1, 32 * TX_DW);
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int item = dt + 128 * u;
        const int vec = item >> 8, p = item & 255;
        const int E = s_emax[slot][vec];
        if (E == 0x7FF) tx_flag(&s_range);
        const int P = TX_PB - E;
        const unsigned long long a0 = tx_fixed(vals[2 * u], P, TX_OFFB);
        const unsigned long long a1 = tx_fixed(vals[2 * u + 1], P, TX_OFFB);
        // row n of a slab sits at 16 n bytes (core matrices of 8 rows x 16 bytes, SBO 128)
        unsigned char* bt = sB + b * TX_BTILE + (p >> 2) * TX_LBO_B + (p & 3) * 4 + 16 * TX_NB * vec;
#pragma unroll
        for (int t = 0; t < TX_NB; t++) {
          const unsigned int u0 = (unsigned int)(a0 >> (TX_BB * t)) & 31u;
          const unsigned int u1 = (unsigned int)(a1 >> (TX_BB * t)) & 31u;
          *reinterpret_cast<unsigned int*>(bt + 16 * t) = s_blut[u0 | (u1 << 5)];
        }
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(&b_full[b]);
    };
    // A wait whose outcome all four warps share: thread 0 of the group polls (bounded) and
    // publishes the result before a group barrier (a ring of two slots: a slot is rewritten
    // only after every thread has passed the next group barrier).
    int ncall = 0;
    auto group_wait = [&](unsigned long long* bar, unsigned int parity) -> bool {
      const int slot = ncall++ & 1;
      if (dt == 0) {
        const bool ok = mbar_wait(bar, parity, WAIT_LIMIT);
        if (!ok) tx_flag(&s_err);
        s_dok[slot] = ok ? 1 : 0;
      }
      named_sync(1, 32 * TX_DW);
      return s_dok[slot] != 0;
    };
    // drain chunk cl (its accumulators are complete): exact digit sums -> FP64 column sums,
    // one tile at a time
    auto drain = [&](int cl) {
      const int b = cl & 1, slot = cl & 3;
      const int jj = lane / TX_NA, s = lane % TX_NA;
      const bool live = lane < TX_CPQ * TX_NA;
      tc_fence_after();
#pragma unroll 1
      for (int tau = 0; tau < ntile; tau++) {
        float D[32];
        tc_ld32(tmem + (unsigned int)(b * 128 + tau * 32) + ((unsigned int)(dw * 32) << 16), D);
        if (tau == ntile - 1) {                       // every accumulator of the set is read
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&t_free[b]);
        }
        if (tau == 0) {
          if (dw == 0 && lane == TX_ONES) {
#pragma unroll
            for (int t = 0; t < 2 * TX_NB; t++) s_bsum[t] = __float2int_rn(D[t]);
          }
          named_sync(1, 32 * TX_DW);
        }
        const int c = tau * TX_CPT + dw * TX_CPQ + jj;
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
          // this lane's digit-s term of X^T Y, mod 2^128
          unsigned __int128 V = (unsigned __int128)(__int128)lo << (TX_BA * s);
          V += (unsigned __int128)(__int128)hi << (7 * TX_BB + TX_BA * s);
          if (!live) V = 0;
          // the six lanes of a column add their terms into the first one
          const unsigned long long v0 = (unsigned long long)V, v1 = (unsigned long long)(V >> 64);
#pragma unroll
          for (int d = 1; d < TX_NA; d++) {
            const int src = (lane + d) & 31;
            const unsigned long long o0 = __shfl_sync(0xffffffffu, v0, src);
            const unsigned long long o1 = __shfl_sync(0xffffffffu, v1, src);
            if (s == 0) V += ((unsigned __int128)o1 << 64) | o0;
          }
          if (s == 0 && live && c < ncols) {
            const __int128 Vs = (__int128)V;
            const double dv = (double)(long long)(Vs >> 64) * 18446744073709551616.0 +
                              (double)(unsigned long long)V;
            const int py = TX_PB - s_emax[slot][vec];
            const int px = c < k ? TX_QP : TX_PB - TX_WSHIFT - s_emax[slot][0];
            const double term = ldexp(dv, -(px + py));
            if (tau == 0) acc[0][vec] += term;
            else if (tau == 1) acc[1][vec] += term;
            else acc[2][vec] += term;
          }
        }
      }
      named_sync(1, 32 * TX_DW);                      // s_bsum is rewritten by the next drain
    };
    produce_b(0);
    bool ok = true;
    for (int cl = 0; cl < nloc && ok; cl++) {
      if (cl >= 1) {
        ok = group_wait(&c_done[(cl - 1) & 1], (unsigned int)(((cl - 1) >> 1) & 1));
        if (!ok) break;
      }
      if (cl + 1 < nloc) produce_b(cl + 1);           // its buffer was chunk cl - 1's
      if (cl >= 1) drain(cl - 1);
    }
    if (ok && group_wait(&c_done[(nloc - 1) & 1], (unsigned int)(((nloc - 1) >> 1) & 1)))
      drain(nloc - 1);
  } else if (lane == 0) {
    // ---------------- MMA issue ----------------
    int64_t g = 0;
    bool stop = false;
    for (int cl = 0; cl < nloc && !stop && !tx_read(&s_err); cl++) {
      const int b = cl & 1;
      if (!mbar_wait(&b_full[b], (unsigned int)((cl >> 1) & 1), WAIT_LIMIT) ||
          (cl >= 2 && !mbar_wait(&t_free[b], (unsigned int)(((cl - 2) >> 1) & 1), WAIT_LIMIT))) {
        tx_flag(&s_err);
        break;
      }
      for (int st = 0; st < TX_NST; st++, g++) {
        const int sb = (int)(g % TX_NAB);
        if (!mbar_wait(&a_full[sb], (unsigned int)((g / TX_NAB) & 1), WAIT_LIMIT)) {
          tx_flag(&s_err);
          stop = true;
          break;
        }
        tc_fence_after();
        const unsigned int abase = smem_u32(sA + sb * TX_ASTAGE), bbase = smem_u32(sB + b * TX_BTILE);
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
        tc_commit(&a_empty[sb]);
        if (st == TX_NST - 1) tc_commit(&c_done[b]);
      }
    }
    // every MMA issued has completed before the tensor memory is freed: the last commit
    // covers all earlier ones
    if (g >= 1) {
      const int64_t gl = g - 1;
      (void)mbar_wait(&a_empty[gl % TX_NAB], (unsigned int)((gl / TX_NAB) & 1), WAIT_LIMIT);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == MMAW)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n"
                 ::"r"(tmem), "r"(TX_TMEM_COLS) : "memory");
  if (tid == 0) {
    if (s_err) atomicCAS(&sc->status, (int)KC_OK, (int)KC_ERR_TIMEOUT);
    else if (s_range) atomicCAS(&sc->status, (int)KC_OK, (int)KC_ERR_NONFINITE);
  }
  // the drain lanes that lead a column write its sums: beta -> [2k], s -> [2k + 1]
  double* pp = partials + (int64_t)blockIdx.x * PSTRIDE;
  if (warp >= TX_PW && warp < MMAW) {
    const int dw = warp - TX_PW, jj = lane / TX_NA, s = lane % TX_NA;
    if (lane < TX_CPQ * TX_NA && s == 0) {
#pragma unroll
      for (int tau = 0; tau < TX_MT; tau++) {
        const int c = tau * TX_CPT + dw * TX_CPQ + jj;
        if (tau < ntile && c < ncols) {
          const int i = c < k ? 2 * c : 2 * k;
          pp[i] = acc[tau][0];
          pp[i + 1] = acc[tau][1];
        }
      }
    }
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
