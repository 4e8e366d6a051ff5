// Hot kernels of the DCGS2 Arnoldi step (Algorithm 4) and of the CGS2 / MGS baselines:
//   K4' CSR SpMV, K1' fused multi-column transposed GEMV with in-launch deterministic
//   cross-CTA reduction and the scalar step, K2' fused GEMV + axpy update, plus the
//   projection, norm and scaling kernels of the CGS2 finish and of the baselines.
//
// Vector element types: FP64 (accumulate FP64) or FP32 (accumulate FP32 within a thread,
// FP64 across warps and CTAs).  Basis element types: FP64, FP32, or BF16 (FP32 vectors).
// Every kernel streams 16-byte groups of rows: 2 rows of FP64, 4 rows of FP32.
#include "kc_internal.cuh"
#include "kc_dfloat.cuh"

namespace kc {

constexpr int PSTRIDE = 2 * NMAX + 4;   // doubles per CTA in the partials buffer

// ----------------------------------------------------------------------------------------
// element helpers
// ----------------------------------------------------------------------------------------
template <typename TV> struct Acc;
template <> struct Acc<double> { using T = double; };
template <> struct Acc<float> { using T = float; };

template <typename TV> struct Grp { static constexpr int R = 16 / sizeof(TV); };

// load R consecutive vector rows of group g (read-only path, cached in L1: the vectors
// are re-read by every warp of the CTA)
__device__ __forceinline__ void ldv(const double* p, int64_t g, double (&o)[2]) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p) + g);
  o[0] = t.x; o[1] = t.y;
}
__device__ __forceinline__ void ldv(const float* p, int64_t g, float (&o)[4]) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p) + g);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
// plain (coherent) vector load: for vectors written earlier in the same kernel sequence
__device__ __forceinline__ void ldv_cg(const double* p, int64_t g, double (&o)[2]) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(p) + g);
  o[0] = t.x; o[1] = t.y;
}
__device__ __forceinline__ void ldv_cg(const float* p, int64_t g, float (&o)[4]) {
  float4 t = __ldcg(reinterpret_cast<const float4*>(p) + g);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void stv(double* p, int64_t g, const double (&o)[2]) {
  reinterpret_cast<double2*>(p)[g] = make_double2(o[0], o[1]);
}
__device__ __forceinline__ void stv(float* p, int64_t g, const float (&o)[4]) {
  reinterpret_cast<float4*>(p)[g] = make_float4(o[0], o[1], o[2], o[3]);
}

// basis loads: streamed once per pass (evict-first)
__device__ __forceinline__ void load_q(const double* p, int64_t g, double (&o)[2]) {
  double2 t = __ldcs(reinterpret_cast<const double2*>(p) + g);
  o[0] = t.x; o[1] = t.y;
}
__device__ __forceinline__ void load_q(const float* p, int64_t g, float (&o)[4]) {
  float4 t = __ldcs(reinterpret_cast<const float4*>(p) + g);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ float bf2f(unsigned short b) {
  return __uint_as_float(((unsigned int)b) << 16);
}
__device__ __forceinline__ void load_q(const __nv_bfloat16* p, int64_t g, float (&o)[4]) {
  uint2 t = __ldcs(reinterpret_cast<const uint2*>(p) + g);
  o[0] = __uint_as_float(t.x << 16);
  o[1] = __uint_as_float(t.x & 0xffff0000u);
  o[2] = __uint_as_float(t.y << 16);
  o[3] = __uint_as_float(t.y & 0xffff0000u);
}
// round to nearest even bfloat16, returned both as bits and as the rounded float
__device__ __forceinline__ unsigned int f2bf_bits(float f) {
  unsigned int u = __float_as_uint(f);
  u += 0x7fffu + ((u >> 16) & 1u);
  return u >> 16;
}
__device__ __forceinline__ void store_q(double* p, int64_t g, double (&o)[2]) {
  reinterpret_cast<double2*>(p)[g] = make_double2(o[0], o[1]);
}
__device__ __forceinline__ void store_q(float* p, int64_t g, float (&o)[4]) {
  reinterpret_cast<float4*>(p)[g] = make_float4(o[0], o[1], o[2], o[3]);
}
// BF16 store rounds o in place, so that the caller continues with the stored values
__device__ __forceinline__ void store_q(__nv_bfloat16* p, int64_t g, float (&o)[4]) {
  unsigned int b0 = f2bf_bits(o[0]), b1 = f2bf_bits(o[1]), b2 = f2bf_bits(o[2]),
               b3 = f2bf_bits(o[3]);
  o[0] = __uint_as_float(b0 << 16); o[1] = __uint_as_float(b1 << 16);
  o[2] = __uint_as_float(b2 << 16); o[3] = __uint_as_float(b3 << 16);
  reinterpret_cast<uint2*>(p)[g] = make_uint2(b0 | (b1 << 16), b2 | (b3 << 16));
}

// scalar (single-row) versions for ragged tails
__device__ __forceinline__ double ld1(const double* p, int64_t i) { return __ldcg(p + i); }
__device__ __forceinline__ float ld1(const float* p, int64_t i) { return __ldcg(p + i); }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p, int64_t i) {
  return bf2f(reinterpret_cast<const unsigned short*>(p)[i]);
}
__device__ __forceinline__ void st1(double* p, int64_t i, double& v) { p[i] = v; }
__device__ __forceinline__ void st1(float* p, int64_t i, float& v) { p[i] = v; }
__device__ __forceinline__ void st1(__nv_bfloat16* p, int64_t i, float& v) {
  unsigned int b = f2bf_bits(v);
  v = __uint_as_float(b << 16);
  reinterpret_cast<unsigned short*>(p)[i] = (unsigned short)b;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of V values (V a power of two, at most 32) over the 32 lanes of a warp in one
// butterfly.  At each of the first log2 V levels a lane keeps half of its values and adds
// its partner's copies of them (V - 1 adds in all), then the remaining levels add the one
// value left: V - 1 + 5 - log2 V adds per lane against 5 V for V separate trees, which counts
// where FP64 adds issue at two per clock per SM.  Lane l ends with the total of value
// l & (V - 1) in x[0], in a fixed order (bitwise the same in every lane that holds it).
template <int V>
__device__ __forceinline__ double warp_sum_multi(double (&x)[V]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = V / 2; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;               // this lane keeps the upper half
#pragma unroll
    for (int i = 0; i < h; i++) {
      const double send = up ? x[i] : x[i + h];
      const double keep = up ? x[i + h] : x[i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
#pragma unroll
  for (int o = V; o < 32; o <<= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
  return x[0];
}

// Column sums of an nrows x nval table (row c at base + c * stride) in a fixed order
// (deterministic) into tot[0:nval], by every thread of the CTA (it synchronises; tot may
// be read after a further __syncthreads).  The last CTA of a reduction runs this while
// the other SMs idle, so it is arranged for memory-level parallelism: with no more values
// than warps, G = nw / nval warps share a value (each over every G-th group of 32 rows,
// eight loads in flight per lane) and their sums are added in warp order; with more, each
// warp takes four values at a time, so that a lane has sixteen loads in flight.
__device__ void sum_rows(const double* __restrict__ base, int nrows, int stride, int nval,
                         double* tot) {
  __shared__ double gsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nval > 0 && nval <= nw) {
    const int G = nw / nval;
    const int vi = warp % nval, gi = warp / nval;
    double acc = 0.0;
    if (gi < G) {
#pragma unroll 8
      for (int c = gi * 32 + lane; c < nrows; c += 32 * G)
        acc += __ldcg(base + (int64_t)c * stride + vi);
    }
    acc = warp_sum(acc);
    if (lane == 0) gsum[warp] = acc;
    __syncthreads();
    if ((int)threadIdx.x < nval) {
      double t = 0.0;
      for (int g = 0; g < G; g++) t += gsum[g * nval + threadIdx.x];
      tot[threadIdx.x] = t;
    }
    return;
  }
  for (int v0 = warp; v0 < nval; v0 += 4 * nw) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int c = lane; c < nrows; c += 32) {
      const double* p = base + (int64_t)c * stride;
#pragma unroll
      for (int u = 0; u < 4; u++)
        if (v0 + u * nw < nval) acc[u] += __ldcg(p + v0 + u * nw);
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const double t = warp_sum(acc[u]);
      if (lane == 0 && v0 + u * nw < nval) tot[v0 + u * nw] = t;
    }
  }
}

// Sum the per-CTA partials in a fixed order (deterministic), into tot[0:nval].
__device__ void sum_partials(const double* __restrict__ partials, int nparts, int nval,
                             double* tot) {
  sum_rows(partials, nparts, PSTRIDE, nval, tot);
}

// Last-CTA election: returns true in every thread of the CTA that arrives last.
__device__ __forceinline__ bool last_cta(unsigned int* counter) {
  __shared__ unsigned int ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return false;
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;   // ready for the next launch on the stream
  return true;
}

// Column sums of a short nrows x nval table (row c at base + c * stride) into tot[0:nval]
// in a fixed order, by every thread of the CTA (no barrier inside): P threads per value
// (aligned lane groups, P = 8, 4, 2 or 1 as the CTA allows), each adding every P-th row in
// row order, their sums combined by a fixed xor tree.  Against sum_rows this issues about
// one FP64 add per table entry instead of the warp tree's five per lane and value, which
// matters on the one SM that runs a reduction's last steps (two FP64 adds per clock).
__device__ void sum_cols(const double* __restrict__ base, int nrows, int64_t stride, int nval,
                         double* tot) {
  const int nt = (int)blockDim.x;
  const int P = nval * 8 <= nt ? 8 : (nval * 4 <= nt ? 4 : (nval * 2 <= nt ? 2 : 1));
  for (int b = 0; b < nval; b += nt / P) {                   // uniform over the CTA
    const int v = b + (int)threadIdx.x / P, sub = (int)threadIdx.x % P;
    double acc = 0.0;
    if (v < nval) {
#pragma unroll 4
      for (int c = sub; c < nrows; c += P) acc += __ldcg(base + (int64_t)c * stride + v);
    }
    for (int o = P / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (v < nval && sub == 0) tot[v] = acc;
  }
}

// Two-level completion of a reduction whose CTAs wrote rows 0..nr-1 of the partials
// (cpr CTAs per row, each writing its own entries of the row; CTA b belongs to row
// b / cpr).  Rows form groups of RED_GROUP; the last CTA of a group to arrive (counted in
// gcount[group]) sums the group's rows in row order into the group's first row, and the
// last group to finish (counted in *counter) returns true in every thread of its CTA.
// The final sums then take ceil(nr / RED_GROUP) rows (stride RED_GROUP rows) instead of
// nr, and the groups' sums run on many SMs while the other CTAs still stream.
__device__ __noinline__ bool tree_arrive(double* __restrict__ partials, int nr, int cpr, int nval,
                            unsigned int* counter, unsigned int* gcount) {
  __shared__ unsigned int ticket;
  const int r = (int)blockIdx.x / cpr, g = r / RED_GROUP;
  const int r0 = g * RED_GROUP, r1 = r0 + RED_GROUP < nr ? r0 + RED_GROUP : nr;
  const int ng = (nr + RED_GROUP - 1) / RED_GROUP;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(gcount + g, 1u);
  __syncthreads();
  if (ticket != (unsigned int)((r1 - r0) * cpr - 1)) return false;
  __threadfence();
  if (r1 - r0 > 1) {
    double* row0 = partials + (int64_t)r0 * PSTRIDE;
    sum_cols(row0, r1 - r0, PSTRIDE, nval, row0);             // in place (per value)
  }
  if (threadIdx.x == 0) gcount[g] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != (unsigned int)(ng - 1)) return false;
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ void set_status(Scalars* sc, int st) {
  if (sc->status == KC_OK) sc->status = st;
}

// The scalar step of Algorithm 4 after alpha is known (all threads of one CTA), with
// inva = 1 / alpha.  Inputs: C (C_{0:k-1}) and S (raw S_{0:k-1} = Q_k^T v) from tot
// (tot[2i], tot[2i+1], shared memory) or, without tot, from sc; s (= w^T v), cs (= C^T S)
// from sc.
//   T_{0:k-1} = S/alpha, T_k = (s - C^T S)/alpha^2 (eq. 30);
//   H(0:k, k-1) = K(0:k, k-1) + C, H(k, k-1) = alpha;
//   K(0:k, k) = T - H(0:k, 0:k-1) C / alpha (the flexible variant keeps K = T);
//   GMRES: Givens rotation of the finalised column k-1.
__device__ void scalar_step(Scalars* sc, const StepArgs& sa, int k, double alpha,
                            double inva, const double* tot = nullptr) {
  // The last CTA runs this once per step, so its dependent FP64 chains (about 70 cycles a
  // link) are on the step's critical path: C, T, the finalised H column and the Givens
  // state are staged in shared memory, the divisions by alpha are products with its
  // reciprocal (computed beside the square root), the breakdown test compares squares, and
  // the K-column products unroll their loads.
  __shared__ double s_c[NMAX], s_h[NMAX + 2], s_gc[NMAX], s_gs[NMAX], s_t[NMAX + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool qr = (sa.flags & SF_QR) != 0;
  if (threadIdx.x == 0) {
    sc->alpha = alpha;
    sc->inv_alpha = inva;
    sc->vscale = qr ? 1.0 : inva;
    const double tk = qr ? (sc->s - sc->cs) * inva : (sc->s - sc->cs) * inva * inva;
    sc->T[k] = tk;
    s_t[k] = tk;
    if ((sa.flags & SF_GIVENS) && k == 0) { sc->g[0] = alpha; sc->ncols = 0; }
    if (sa.flags & SF_FLEXIBLE) sc->zscale[k] = inva;
    if (k >= 1 || qr) sa.H[k + (int64_t)(k - 1) * sa.ldh] = alpha;
    s_h[k] = alpha;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double c = tot ? tot[2 * i] : sc->C[i];
    const double si = tot ? tot[2 * i + 1] : sc->S[i];
    const double t = qr ? si : si * inva;
    sc->T[i] = t;
    s_t[i] = t;
    const double h = sa.K[i + (int64_t)(k - 1) * sa.ldk] + c;
    sa.H[i + (int64_t)(k - 1) * sa.ldh] = h;
    s_c[i] = c;
    s_h[i] = h;
    if (i < k - 1) { s_gc[i] = sc->gc[i]; s_gs[i] = sc->gs[i]; }
  }
  __syncthreads();
  if (warp == 0 && k >= 1) {
    double cn = 0.0;
    for (int i = lane; i <= k; i += 32) cn += s_h[i] * s_h[i];
    cn = warp_sum(cn);
    if (lane == 0 && alpha * alpha <= 1e-26 * cn) set_status(sc, KC_ERR_BREAKDOWN);
  }
  // K(i, k) = T_i - H(i, 0:k-1) C / alpha for i <= k: P lanes per row (aligned groups of a
  // warp), each over every P-th column, added by a fixed xor tree, so that each thread has
  // only k / P dependent-free loads of H to wait for
  {
    const int nt = (int)blockDim.x;
    const int P = (k + 1) * 8 <= nt ? 8 : ((k + 1) * 4 <= nt ? 4 : ((k + 1) * 2 <= nt ? 2 : 1));
    const bool corr = !(sa.flags & (SF_FLEXIBLE | SF_QR));
    for (int base = 0; base <= k; base += nt / P) {          // uniform over the CTA
      const int i = base + (int)threadIdx.x / P, sub = (int)threadIdx.x % P;
      double hc = 0.0;
      if (i <= k && corr) {
#pragma unroll 4
        for (int j = sub; j < k; j += P) hc += sa.H[i + (int64_t)j * sa.ldh] * s_c[j];
      }
      for (int o = P / 2; o > 0; o >>= 1) hc += __shfl_xor_sync(0xffffffffu, hc, o);
      if (i <= k && sub == 0) sa.K[i + (int64_t)k * sa.ldk] = s_t[i] - hc * inva;
    }
  }
  if (threadIdx.x == 0 && (sa.flags & SF_GIVENS) && k >= 1) {
    // Givens rotation of column k-1 on the staged copies (the column is s_h, stride 0)
    const int j = k - 1;
    const double e = givens_rotate(s_gc, s_gs, sc->g, s_h, 0, j, sa.R, sa.ldr);
    sc->gc[j] = s_gc[j];
    sc->gs[j] = s_gs[j];
    sc->resid_est = e;
    sc->ncols = j + 1;
    if (!(e > sc->rtol_abs)) sc->stop = 1;
  }
}

// ----------------------------------------------------------------------------------------
// K4': CSR SpMV, one thread per row.
// ----------------------------------------------------------------------------------------
// CTA sums of x^T x and x^T y (FP64, fixed order) into dots[2 b], dots[2 b + 1]
__device__ __forceinline__ void store_dots(double ab, double as, double* dots) {
  __shared__ double red[2][8];
  double x[2] = {ab, as};
  const double v = warp_sum_multi<2>(x);          // lane 0: x^T x, lane 1: x^T y
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < 2) red[lane][warp] = v;
  __syncthreads();
  if (threadIdx.x < 2) {
    double b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) b += red[threadIdx.x][i];
    dots[2 * blockIdx.x + threadIdx.x] = b;
  }
}

// (A x)_r of a CSR row, the products added in the row's stored order
template <typename TA, typename TV>
__device__ __forceinline__ TA csr_row(const int32_t* __restrict__ rp,
                                      const int32_t* __restrict__ ci, const TA* __restrict__ val,
                                      const TV* __restrict__ x, int64_t r) {
  const int b = __ldg(rp + r), e = __ldg(rp + r + 1);
  TA s = 0;
  for (int j = b; j < e; j++) s += __ldg(val + j) * (TA)__ldcg(x + __ldg(ci + j));
  return s;
}

// DOTS (FP64 DCGS2 step): the same pass also sums beta = x^T x and s = x^T y per CTA, the
// two FP64 tasks of the step's reduction, at the cost of one more load of x[r] (in cache)
// and two FMAs per row in this HBM-bound kernel.
template <typename TA, typename TV, bool DOTS = false>
__global__ void __launch_bounds__(256) k_spmv(const int32_t* __restrict__ rp,
                                              const int32_t* __restrict__ ci,
                                              const TA* __restrict__ val,
                                              const TV* __restrict__ x, TV* __restrict__ y,
                                              int64_t m, const Scalars* __restrict__ sc,
                                              double* __restrict__ dots = nullptr) {
  pdl_wait();
  if (sc->stop) return;
  double ab = 0.0, as = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const TA s = csr_row<TA>(rp, ci, val, x, r);
    y[r] = (TV)s;
    if (DOTS) {
      const double xr = (double)__ldcg(x + r);
      ab = fma(xr, xr, ab);
      as = fma(xr, (double)s, as);
    }
  }
  pdl_trigger();
  if (DOTS) store_dots(ab, as, dots);
}

// ----------------------------------------------------------------------------------------
// K4'': the matrix-free 7-point stencil, one thread per row.  The terms are summed in
// increasing column order (z-, y-, x-, centre, x+, y+, z+), the order of a CSR row, so on
// the same coefficients the result is bitwise that of k_spmv.  The x-neighbours come from
// the warp's own lines (L1), the y- and z-neighbours from L2 (one plane is nx ny elements).
// ----------------------------------------------------------------------------------------
template <typename T>
struct Stencil7 {
  T c[7];       // centre, x-1, x+1, y-1, y+1, z-1, z+1
};

// (A x)_r of the 7-point stencil, terms in CSR column order
template <typename T>
__device__ __forceinline__ T stencil_row(const T* __restrict__ x, int64_t r, int nx, int ny,
                                         int nz, const Stencil7<T>& c) {
  // 32-bit index arithmetic (m < 2^31 is checked at the boundary): a 64-bit division per
  // row costs more issue slots than the row's seven FMAs
  const int64_t pl = (int64_t)nx * ny;
  const unsigned int ur = (unsigned int)r, t = ur / (unsigned int)nx;
  const unsigned int q = t / (unsigned int)ny;
  const int ix = (int)(ur - t * (unsigned int)nx);
  const int iy = (int)(t - q * (unsigned int)ny), iz = (int)q;
  T s = 0;
  if (iz > 0) s += c.c[5] * __ldcg(x + r - pl);
  if (iy > 0) s += c.c[3] * __ldcg(x + r - nx);
  if (ix > 0) s += c.c[1] * __ldcg(x + r - 1);
  s += c.c[0] * __ldcg(x + r);
  if (ix < nx - 1) s += c.c[2] * __ldcg(x + r + 1);
  if (iy < ny - 1) s += c.c[4] * __ldcg(x + r + nx);
  if (iz < nz - 1) s += c.c[6] * __ldcg(x + r + pl);
  return s;
}

template <typename T, bool DOTS = false>
__global__ void __launch_bounds__(256) k_stencil7(const T* __restrict__ x, T* __restrict__ y,
                                                  int nx, int ny, int nz, Stencil7<T> c,
                                                  const Scalars* __restrict__ sc,
                                                  double* __restrict__ dots = nullptr) {
  pdl_wait();
  if (sc->stop) return;
  double ab = 0.0, as = 0.0;
  const int64_t m = (int64_t)nx * ny * nz;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const T s = stencil_row(x, r, nx, ny, nz, c);
    y[r] = s;
    if (DOTS) {
      const double xr = (double)__ldcg(x + r);
      ab = fma(xr, xr, ab);
      as = fma(xr, (double)s, as);
    }
  }
  pdl_trigger();
  if (DOTS) store_dots(ab, as, dots);
}

// The ICWY-MGS step (Section 5) from the summed [C, S, beta, s] of the fused reduction
// (all threads of one CTA): alpha = sqrt(beta) = ||w|| normalises the pending w into q_k
// (H(k, k-1) = alpha), row k of the strictly lower triangular L is C / alpha (stored in the
// K workspace, K(k, i)), and the projection coefficients of the next vector are
// y = (I + L)^{-1} r with r = [S / alpha; s / alpha^2] (QR of given columns: [S; s / alpha]),
// by forward substitution; y is H(0:k+1, k) and, with C = 0, the update's T.
__device__ void icwy_step(const double* tot, int k, Scalars* __restrict__ sc,
                          const StepArgs& sa) {
  __shared__ double s_r[NMAX + 1];
  __shared__ double s_a;
  const bool qr = (sa.flags & SF_QR) != 0;
  if (threadIdx.x == 0) {
    const double beta = tot[2 * k], s = tot[2 * k + 1];
    double alpha = sqrt(beta);
    if (!isfinite(beta) || !isfinite(s)) set_status(sc, KC_ERR_NONFINITE);
    if (!(alpha > 0.0)) {
      set_status(sc, KC_ERR_BREAKDOWN);
      alpha = 1e-300;
    }
    sc->alpha = alpha;
    sc->inv_alpha = 1.0 / alpha;
    sc->vscale = qr ? 1.0 : 1.0 / alpha;
    if (k >= 1 || qr) sa.H[k + (int64_t)(k - 1) * sa.ldh] = alpha;
    s_r[k] = qr ? s / alpha : s / (alpha * alpha);
    s_a = alpha;
  }
  __syncthreads();
  const double alpha = s_a;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    sa.K[k + (int64_t)i * sa.ldk] = tot[2 * i] / alpha;        // L(k, i)
    sc->C[i] = 0.0;                                            // the update projects with T only
    s_r[i] = qr ? tot[2 * i + 1] : tot[2 * i + 1] / alpha;
  }
  __syncthreads();
  for (int i = 0; i <= k; i++) {                               // (I + L) y = r, column by column
    const double yi = s_r[i];
    for (int l = i + 1 + threadIdx.x; l <= k; l += blockDim.x)
      s_r[l] -= __ldcg(sa.K + l + (int64_t)i * sa.ldk) * yi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    sc->T[i] = s_r[i];
    sa.H[i + (int64_t)k * sa.ldh] = s_r[i];
  }
  if (threadIdx.x == 0 && k >= 1) {                            // happy breakdown test
    double cn = alpha * alpha;
    for (int i = 0; i < k; i++) {
      const double h = sa.H[i + (int64_t)(k - 1) * sa.ldh];
      cn += h * h;
    }
    if (alpha <= 1e-13 * sqrt(cn)) set_status(sc, KC_ERR_BREAKDOWN);
  }
}

// The epilogue on the summed values tot[0 : (k + 1) NRHS] (shared memory; all threads of
// one CTA): a store of this rank's sums (row-partitioned step), a store of Q^T x, the
// ICWY-MGS step, or the scalar step of Algorithm 4.
__device__ void epilogue_from_tot(const double* tot, int k, int NRHS, Scalars* __restrict__ sc,
                                  int epilogue, const StepArgs& sa) {
  __shared__ double s_alpha, s_inva;
  const int nval = (k + 1) * NRHS;
  if (epilogue == EPI_PARTIAL) {
    for (int i = threadIdx.x; i < nval; i += blockDim.x) sa.part[i] = tot[i];
    return;
  }
  if (epilogue == EPI_ICWY) {
    icwy_step(tot, k, sc, sa);
    return;
  }
  if (epilogue != EPI_DCGS2) {
    double* dst = (epilogue == EPI_STORE_C || epilogue == EPI_STORE_C1)
                      ? sc->C
                      : (epilogue == EPI_STORE_C2 ? sc->C2 : sc->S);
    for (int i = threadIdx.x; i < k; i += blockDim.x) dst[i] = tot[i * NRHS];
    if (threadIdx.x == 0) {
      sc->norm_sq = tot[k * NRHS];
      if (!isfinite(tot[k * NRHS])) set_status(sc, KC_ERR_NONFINITE);
    }
    return;
  }

  // ---- scalar step of Algorithm 4, FP64 --------------------------------------------------
  // tot[2i] = C_i, tot[2i+1] = S_i (i < k); tot[2k] = beta, tot[2k+1] = s
  __shared__ int s_ok;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    sc->C[i] = tot[2 * i];
    sc->S[i] = tot[2 * i + 1];
  }
  if (threadIdx.x < 32) {                                   // C^T C and C^T S: warp 0
    double cc = 0.0, cs = 0.0;
    for (int i = threadIdx.x; i < k; i += 32) {
      cc += tot[2 * i] * tot[2 * i];
      cs += tot[2 * i] * tot[2 * i + 1];
    }
    cc = warp_sum(cc);
    cs = warp_sum(cs);
    if (threadIdx.x == 0) {
      const double beta = tot[2 * k], s = tot[2 * k + 1];
      double a2 = beta - cc;                                 // Pythagoras
      sc->beta = beta;
      sc->s = s;
      sc->cs = cs;
      s_ok = 1;
      if (!isfinite(a2) || !isfinite(s)) {
        set_status(sc, KC_ERR_NONFINITE);
      } else if (!(a2 > sa.pyth_tol * beta)) {
        if (sa.flags & SF_FALLBACK) {
          sc->fallback = 1;                                  // explicit norm pass follows
          s_ok = 0;
        } else {
          set_status(sc, KC_ERR_PYTHAGORAS_NEG);
          a2 = fmax(a2, 1e-300);
        }
      }
      s_alpha = sqrt(a2);
      s_inva = 1.0 / s_alpha;
    }
  }
  __syncthreads();
  if (s_ok) scalar_step(sc, sa, k, s_alpha, s_inva, tot);
}

// Last CTA of a reduction: deterministic sum of the per-CTA partials, then the epilogue.
// With `dots` (the DCGS2 step whose SpMV formed beta = w^T w and s = w^T v, ndots CTAs of
// two sums each), the partials hold the 2k column sums only and beta, s are the
// fixed-order sums of the SpMV's.
__device__ void reduce_epilogue(const double* __restrict__ partials, int k, int NRHS,
                                Scalars* __restrict__ sc, int epilogue, const StepArgs& sa,
                                int nparts = -1, const double* __restrict__ dots = nullptr,
                                int ndots = 0) {
  __shared__ double tot[PSTRIDE];
  const int nval = (k + 1) * NRHS;
  sum_partials(partials, nparts < 0 ? (int)gridDim.x : nparts, dots ? 2 * k : nval, tot);
  if (dots) {
    __syncthreads();                                           // sum_rows' scratch
    sum_rows(dots, ndots, 2, 2, tot + 2 * k);                  // beta -> [2k], s -> [2k+1]
  }
  __syncthreads();
  epilogue_from_tot(tot, k, NRHS, sc, epilogue, sa);
}

// Last CTA of a two-level reduction (tree_arrive over nr partials rows): the fixed-order
// sums of the group rows, then the epilogue.
__device__ void tree_epilogue(const double* __restrict__ partials, int nr, int k, int NRHS,
                              Scalars* __restrict__ sc, int epilogue, const StepArgs& sa) {
  __shared__ double tot[PSTRIDE];
  sum_cols(partials, (nr + RED_GROUP - 1) / RED_GROUP, (int64_t)RED_GROUP * PSTRIDE,
           (k + 1) * NRHS, tot);
  __syncthreads();
  epilogue_from_tot(tot, k, NRHS, sc, epilogue, sa);
}

// ----------------------------------------------------------------------------------------
// K1': fused reduction.  Tasks t = 0..k-1 are Q(:,t)^T [x, y]; task k is x^T [x, y].
// Warp w owns tasks w, w+16, w+32, ... (TPW of them) and keeps their partial sums in
// registers over all of the CTA's rows; the 16 warps of a CTA walk the same rows, so
// x and y are read from HBM once and served from L1 to the other warps.
// With rsub > 1 (a few tasks: one slot, nw = ntask task warps) the CTA's warps form rsub
// row sub-blocks: each walks its share of the CTA's rows with the whole task set, and the
// sub-block sums are added in shared memory in sub-block order.
// The partials are summed in a fixed order (deterministic): with gcount, in two levels
// (tree_arrive: groups of RED_GROUP rows, then the group rows), else by the last CTA to
// finish in CTA order (the allocation-free step).  The CTA that completes the sums runs
// the epilogue: the scalar step of Algorithm 4 or a plain store.
// ----------------------------------------------------------------------------------------
template <typename TQ, typename TV, int TPW, int NRHS>
__global__ void __launch_bounds__(RED_THREADS)
k_reduce(const TQ* __restrict__ Q, int64_t ldq, int k, const TV* __restrict__ x,
         const TV* __restrict__ y, int64_t m, double* __restrict__ partials,
         unsigned int* __restrict__ counter, Scalars* __restrict__ sc, int epilogue,
         StepArgs sa, int rsub, unsigned int* __restrict__ gcount) {
  using TA = typename Acc<TV>::T;
  constexpr int R = Grp<TV>::R;
  pdl_wait();
  if (sc->stop) return;
  // (one- to three-slot launches size their CTAs to the task count; a compile-time warp
  // count keeps the four- and eight-slot variants within 64 registers)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = TPW <= 3 ? (int)(blockDim.x >> 5) / rsub : RED_WARPS;
  const int wt = warp % nw, rs = warp / nw;        // task warp, row sub-block
  const int ntask = k + 1;
  TA acc[TPW][NRHS];
#pragma unroll
  for (int i = 0; i < TPW; i++)
#pragma unroll
    for (int r = 0; r < NRHS; r++) acc[i][r] = 0;

  const int64_t ngroups = m / R;
  const int64_t b0 = (int64_t)blockIdx.x * ngroups / gridDim.x;
  const int64_t b1 = (int64_t)(blockIdx.x + 1) * ngroups / gridDim.x;
  const int64_t g0 = b0 + (b1 - b0) * rs / rsub, g1 = b0 + (b1 - b0) * (rs + 1) / rsub;
  int64_t g = g0 + lane;
  // FP32 / BF16 vectors (HBM-bound): two row groups per iteration, every load issued
  // before the arithmetic, so twice the bytes are in flight per warp
  if (sizeof(TV) == 4 && TPW <= 4) {
    for (; g + 32 < g1; g += 64) {
      TV xa[R], ya[R], xb[R], yb[R];
      ldv(x, g, xa);
      ldv(x, g + 32, xb);
      if (NRHS == 2) { ldv(y, g, ya); ldv(y, g + 32, yb); }
      TA qa[TPW][R], qb[TPW][R];
#pragma unroll
      for (int i = 0; i < TPW; i++) {
        const int t = wt + nw * i;
        if (t < k) {
          load_q(Q + (int64_t)t * ldq, g, qa[i]);
          load_q(Q + (int64_t)t * ldq, g + 32, qb[i]);
        } else {
#pragma unroll
          for (int r = 0; r < R; r++) { qa[i][r] = xa[r]; qb[i][r] = xb[r]; }
        }
      }
#pragma unroll
      for (int i = 0; i < TPW; i++) {
        if (wt + nw * i >= ntask) continue;
#pragma unroll
        for (int r = 0; r < R; r++) {
          acc[i][0] += qa[i][r] * (TA)xa[r];
          acc[i][0] += qb[i][r] * (TA)xb[r];
          if (NRHS == 2) {
            acc[i][1] += qa[i][r] * (TA)ya[r];
            acc[i][1] += qb[i][r] * (TA)yb[r];
          }
        }
      }
    }
  }
  for (; g < g1; g += 32) {
    TV xv[R], yv[R];
    ldv(x, g, xv);
    if (NRHS == 2) ldv(y, g, yv);
#pragma unroll
    for (int i = 0; i < TPW; i++) {
      const int t = wt + nw * i;
      if (t < ntask) {
        TA qv[R];
        if (t < k) {
          load_q(Q + (int64_t)t * ldq, g, qv);
        } else {
#pragma unroll
          for (int r = 0; r < R; r++) qv[r] = xv[r];
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
          acc[i][0] += qv[r] * (TA)xv[r];
          if (NRHS == 2) acc[i][1] += qv[r] * (TA)yv[r];
        }
      }
    }
  }
  // ragged tail: rows ngroups*R .. m-1, taken by the last CTA's first row sub-block
  if (blockIdx.x == gridDim.x - 1 && rs == 0) {
    for (int64_t row = ngroups * R + lane; row < m; row += 32) {
      TA xs = (TA)__ldcg(x + row);
      TA ys = NRHS == 2 ? (TA)__ldcg(y + row) : (TA)0;
#pragma unroll
      for (int i = 0; i < TPW; i++) {
        const int t = wt + nw * i;
        if (t < ntask) {
          TA q = t < k ? (TA)ld1(Q + (int64_t)t * ldq, row) : xs;
          acc[i][0] += q * xs;
          if (NRHS == 2) acc[i][1] += q * ys;
        }
      }
    }
  }
  double sum[TPW][NRHS];
#pragma unroll
  for (int i = 0; i < TPW; i++)
#pragma unroll
    for (int r = 0; r < NRHS; r++) sum[i][r] = (double)warp_sum(acc[i][r]);
  __shared__ double red[RED_WARPS][TPW][NRHS];     // sub-block sums (rsub > 1)
  if (rsub > 1) {
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < TPW; i++)
#pragma unroll
        for (int r = 0; r < NRHS; r++) red[warp][i][r] = sum[i][r];
    __syncthreads();
    if (rs == 0)
#pragma unroll
      for (int i = 0; i < TPW; i++)
#pragma unroll
        for (int r = 0; r < NRHS; r++) {
          double t = red[wt][i][r];
          for (int q = 1; q < rsub; q++) t += red[q * nw + wt][i][r];
          sum[i][r] = t;
        }
  }
  if (rs == 0 && lane == 0)
#pragma unroll
    for (int i = 0; i < TPW; i++) {
      const int t = wt + nw * i;
      if (t < ntask)
#pragma unroll
        for (int r = 0; r < NRHS; r++)
          partials[(int64_t)blockIdx.x * PSTRIDE + t * NRHS + r] = sum[i][r];
    }
  pdl_trigger();
  if (gcount) {                                   // two-level completion
    if (!tree_arrive(partials, (int)gridDim.x, 1, ntask * NRHS, counter, gcount)) return;
    tree_epilogue(partials, (int)gridDim.x, k, NRHS, sc, epilogue, sa);
    return;
  }
  if (!last_cta(counter)) return;
  reduce_epilogue(partials, k, NRHS, sc, epilogue, sa);
}

// ----------------------------------------------------------------------------------------
// K2': fused update of Algorithm 4 (normalisation and projection).
//   u = w - Q_k C;  q_k = u / alpha -> Q(:,k);  w <- v/alpha - Q_k T(0:k) - q_k T_k
// One pass over Q_k; C and T are staged in shared memory.
// ----------------------------------------------------------------------------------------
template <typename TQ, typename TV>
__global__ void __launch_bounds__(UPD_THREADS)
k_dcgs2_update(TQ* __restrict__ Q, int64_t ldq, int k, TV* __restrict__ w,
               const TV* __restrict__ v, int64_t m, const Scalars* __restrict__ sc) {
  using TA = typename Acc<TV>::T;
  constexpr int R = Grp<TV>::R;
  pdl_wait();
  if (sc->stop) return;
  __shared__ TA sC[NMAX], sT[NMAX + 1];
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    if (i < k) sC[i] = (TA)sc->C[i];
    sT[i] = (TA)sc->T[i];
  }
  const TA inva = (TA)sc->inv_alpha;
  const TA vsc = (TA)sc->vscale;
  __syncthreads();
  TQ* qk = Q + (int64_t)k * ldq;
  const int64_t ngroups = m / R;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    TV wv[R], vv[R];
    ldv_cg(w, g, wv);
    ldv_cg(v, g, vv);
    TA u[R], wn[R];
#pragma unroll
    for (int r = 0; r < R; r++) { u[r] = wv[r]; wn[r] = vv[r] * vsc; }
    int i = 0;
    for (; i + 4 <= k; i += 4) {
      TA q0[R], q1[R], q2[R], q3[R];
      load_q(Q + (int64_t)(i + 0) * ldq, g, q0);
      load_q(Q + (int64_t)(i + 1) * ldq, g, q1);
      load_q(Q + (int64_t)(i + 2) * ldq, g, q2);
      load_q(Q + (int64_t)(i + 3) * ldq, g, q3);
#pragma unroll
      for (int r = 0; r < R; r++) {
        u[r] -= q0[r] * sC[i]; wn[r] -= q0[r] * sT[i];
        u[r] -= q1[r] * sC[i + 1]; wn[r] -= q1[r] * sT[i + 1];
        u[r] -= q2[r] * sC[i + 2]; wn[r] -= q2[r] * sT[i + 2];
        u[r] -= q3[r] * sC[i + 3]; wn[r] -= q3[r] * sT[i + 3];
      }
    }
    for (; i < k; i++) {
      TA q0[R];
      load_q(Q + (int64_t)i * ldq, g, q0);
#pragma unroll
      for (int r = 0; r < R; r++) { u[r] -= q0[r] * sC[i]; wn[r] -= q0[r] * sT[i]; }
    }
    TA qn[R];
#pragma unroll
    for (int r = 0; r < R; r++) qn[r] = u[r] * inva;
    store_q(qk, g, qn);                         // (BF16: qn now holds the rounded values)
    TV wo[R];
#pragma unroll
    for (int r = 0; r < R; r++) wo[r] = (TV)(wn[r] - qn[r] * sT[k]);
    stv(w, g, wo);
  }
  pdl_trigger();
  // ragged tail
  if (blockIdx.x == 0) {
    for (int64_t row = ngroups * R + threadIdx.x; row < m; row += blockDim.x) {
      TA u = (TA)w[row], wn = (TA)v[row] * vsc;
      for (int i = 0; i < k; i++) {
        TA q = (TA)ld1(Q + (int64_t)i * ldq, row);
        u -= q * sC[i];
        wn -= q * sT[i];
      }
      TA qn = u * inva;
      st1(qk, row, qn);
      w[row] = (TV)(wn - qn * sT[k]);
    }
  }
}

// x <- x - Q_k c, c = C (which 0), C2 (1) or S (2).  Used by CGS2 passes.
// With `allow32` (FP64 basis and vectors, FP64 offload mode) a launch whose coefficients
// are small against the result takes Q c in FP32, under the bound of
// k_dcgs2_update_f64x: (k + 3) 2^-24 ||c||_1 <= 2^-53 ||x - Q c||, where
// ||x - Q c||^2 = x^T x - ||c||^2 from the reduction that produced c (sc->norm_sq).  The
// second projection of the CGS2 finish (and the first, whose x is the pending vector,
// already projected once) meets it; a first projection (c = S) does not and stays FP64.
template <typename TQ, typename TV>
__global__ void __launch_bounds__(UPD_THREADS)
k_gemv_sub(const TQ* __restrict__ Q, int64_t ldq, int k, TV* __restrict__ x, int64_t m,
           const Scalars* __restrict__ sc, int which, int allow32) {
  using TA = typename Acc<TV>::T;
  constexpr int R = Grp<TV>::R;
  if (sc->stop) return;
  __shared__ TA sc_[NMAX];
  __shared__ float sf_[NMAX];
  __shared__ double s_scale;
  __shared__ int s_fast;
  const double* src = which == 0 ? sc->C : (which == 1 ? sc->C2 : sc->S);
  for (int i = threadIdx.x; i < k; i += blockDim.x) sc_[i] = (TA)src[i];
  if (threadIdx.x == 0) {
    int fast = 0;
    double sc2 = 1.0;
    if (allow32 && sizeof(TQ) == 8 && sizeof(TV) == 8) {
      double cmax = 0.0, l1 = 0.0, c2 = 0.0;
      for (int i = 0; i < k; i++) {
        const double c = src[i];
        cmax = fmax(cmax, fabs(c));
        l1 += fabs(c);
        c2 += c * c;
      }
      const double rest = sc->norm_sq - c2;
      int ex = 0;
      if (cmax > 0.0) frexp(cmax, &ex);
      sc2 = ldexp(1.0, ex);
      fast = (rest > 0.0 && cmax > 0.0 && ex > -900 &&
              l1 * (double)(k + 3) <= 0x1p-29 * sqrt(rest)) ? 1 : 0;
    }
    s_fast = fast;
    s_scale = sc2;
  }
  __syncthreads();
  const int64_t ngroups = m / R;
  if (sizeof(TQ) == 8 && sizeof(TV) == 8 && s_fast) {
    // powers of two: the inverse by its exponent (a division in every thread is a
    // sequence of FP64 operations on this pipe-bound GPU)
    const double scale = s_scale;
    int ex_s = 0;
    frexp(scale, &ex_s);
    const double inv = ldexp(1.0, 1 - ex_s);
    for (int i = threadIdx.x; i < k; i += blockDim.x) sf_[i] = d2f_trunc(src[i] * inv);
    __syncthreads();
    const double* Qd = reinterpret_cast<const double*>(Q);
    double* xd = reinterpret_cast<double*>(x);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < m / 2;
         g += (int64_t)gridDim.x * blockDim.x) {
      double xv[2];
      ldv_cg(xd, g, xv);
      float z[2] = {0.0f, 0.0f};
      int i = 0;
      for (; i + 4 <= k; i += 4) {
        double q[4][2];
#pragma unroll
        for (int j = 0; j < 4; j++) load_q(Qd + (int64_t)(i + j) * ldq, g, q[j]);
#pragma unroll
        for (int j = 0; j < 4; j++) {
          z[0] = fmaf(d2f_trunc(q[j][0]), sf_[i + j], z[0]);
          z[1] = fmaf(d2f_trunc(q[j][1]), sf_[i + j], z[1]);
        }
      }
      for (; i < k; i++) {
        double q[2];
        load_q(Qd + (int64_t)i * ldq, g, q);
        z[0] = fmaf(d2f_trunc(q[0]), sf_[i], z[0]);
        z[1] = fmaf(d2f_trunc(q[1]), sf_[i], z[1]);
      }
      xv[0] = fma(-f2d_bits(z[0]), scale, xv[0]);
      xv[1] = fma(-f2d_bits(z[1]), scale, xv[1]);
      stv(xd, g, xv);
    }
  } else
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    TV xv[R];
    ldv_cg(x, g, xv);
    TA u[R];
#pragma unroll
    for (int r = 0; r < R; r++) u[r] = xv[r];
    int i = 0;
    for (; i + 4 <= k; i += 4) {
      TA q0[R], q1[R], q2[R], q3[R];
      load_q(Q + (int64_t)(i + 0) * ldq, g, q0);
      load_q(Q + (int64_t)(i + 1) * ldq, g, q1);
      load_q(Q + (int64_t)(i + 2) * ldq, g, q2);
      load_q(Q + (int64_t)(i + 3) * ldq, g, q3);
#pragma unroll
      for (int r = 0; r < R; r++)
        u[r] -= q0[r] * sc_[i] + q1[r] * sc_[i + 1] + q2[r] * sc_[i + 2] + q3[r] * sc_[i + 3];
    }
    for (; i < k; i++) {
      TA q0[R];
      load_q(Q + (int64_t)i * ldq, g, q0);
#pragma unroll
      for (int r = 0; r < R; r++) u[r] -= q0[r] * sc_[i];
    }
#pragma unroll
    for (int r = 0; r < R; r++) xv[r] = (TV)u[r];
    stv(x, g, xv);
  }
  if (blockIdx.x == 0) {
    for (int64_t row = ngroups * R + threadIdx.x; row < m; row += blockDim.x) {
      TA u = (TA)x[row];
      for (int i = 0; i < k; i++) u -= (TA)ld1(Q + (int64_t)i * ldq, row) * sc_[i];
      x[row] = (TV)u;
    }
  }
}

// ----------------------------------------------------------------------------------------
// FP64 with offload.  This GPU executes about 2 FP64 FMAs per SM per clock against
// ~128 FP32 operations, so the two FP64 passes of a DCGS2 step are FP64-pipe bound.
// Only half of their products need FP64: the reorthogonalisation coefficients
// C = Q^T w (a tiny result of heavy cancellation that enters H and q
// directly) and the projection w <- v/alpha - Q T (its rounding error is the
// Arnoldi representation error).  The first-projection coefficients S = Q^T v
// only need to be accurate enough for the next step's delayed reorthogonalisation to
// remove what they leave behind (any error d in S reappears as -d/alpha in the next C and
// cancels in H = K + C), and the product Q C in q = (w - Q C)/alpha is
// multiplied by the tiny C.  Both are evaluated here in float-float arithmetic
// (operands split into two floats by integer operations, exact TwoProd products,
// TwoSum accumulation; about 2^-44 relative), on the FP32/INT pipes, concurrently with
// the FP64 FMAs of C and Q T.  Zeros and elements whose magnitude is outside [2^-80, 2^98) take
// the FP64 path.
// ----------------------------------------------------------------------------------------

// Offloaded reduction, task layout.  ntask = k + 2 tasks of equal FP64 cost (two FP64
// FMAs per group of two rows): task t < k is column t
// (C_t = q_t^T w in FP64 and S_t = q_t^T v in float-float), task k is beta = w^T w and
// task k + 1 is s = w^T v, both in FP64.  The tasks are cut into nsplit subsets of at most 48 (nt each); the grid is
// nsplit CTAs per row block, CTA (row block r, subset h) has nw = ceil(nt / TPW) warps and
// warp w takes the subset's tasks w, w + nw, ... (TPW slots, TPW <= 3), so at most TPW - 1
// slots of a CTA are idle and every CTA has at most 16 warps (two or more CTAs per SM
// with 64 registers).  All warps of a CTA walk the same rows; w and v come from L1 after
// the first warp has loaded them (and from L2 for the other subsets of the row block).

// the operand that task t multiplies into w: q_t, w itself (beta) or v (s); null if idle
__device__ __forceinline__ const double* f64x_operand(const double* Q, int64_t ldq, int k,
                                                      const double* x, const double* y,
                                                      int t) {
  return t < k ? Q + (int64_t)t * ldq : (t == k ? x : (t == k + 1 ? y : nullptr));
}

// One group of two rows for every slot: ac += a . w (FP64; C, beta and s); for columns
// S += a . v in float-float (OFF) or FP64 (!OFF, operands outside the float-float range).
// (s = w^T v in float-float as well measured slower: the warp that holds it then splits w.)
template <int TPW, bool OFF>
__device__ __forceinline__ void f64x_group(const int (&tk)[TPW], int k,
                                           const double (&xv)[2], const double (&yv)[2],
                                           const double (&av)[TPW][2], double* ac,
                                           double* as64, float* sh, float* sl) {
  float yh[2], yl[2];
  if (OFF) { split_fast(yv[0], yh[0], yl[0]); split_fast(yv[1], yh[1], yl[1]); }
#pragma unroll
  for (int i = 0; i < TPW; i++) {
    if (tk[i] > k + 1) continue;                 // idle slot (warp-uniform)
    ac[i] = fma(av[i][0], xv[0], ac[i]);
    ac[i] = fma(av[i][1], xv[1], ac[i]);
    if (tk[i] < k) {
      if (OFF) {
        float ah[2], al[2];
        split_fast(av[i][0], ah[0], al[0]);
        split_fast(av[i][1], ah[1], al[1]);
        df_mac(sh[i], sl[i], ah[0], al[0], yh[0], yl[0]);
        df_mac(sh[i], sl[i], ah[1], al[1], yh[1], yl[1]);
      } else {
        as64[i] = fma(av[i][0], yv[0], as64[i]);
        as64[i] = fma(av[i][1], yv[1], as64[i]);
      }
    }
  }
}

// true when every operand that the float-float path splits lies in its range (zero and
// magnitudes outside [2^-80, 2^98) take the FP64 path)
template <int TPW>
__device__ __forceinline__ bool f64x_in_range(const int (&tk)[TPW], int k,
                                              const double (&xv)[2], const double (&yv)[2],
                                              const double (&av)[TPW][2]) {
  bool ok = split_fast_ok(yv[0]) & split_fast_ok(yv[1]);
#pragma unroll
  for (int i = 0; i < TPW; i++)
    if (tk[i] < k) ok = ok & split_fast_ok(av[i][0]) & split_fast_ok(av[i][1]);
  (void)xv;
  return ok;
}

template <int TPW>
__device__ __forceinline__ void f64x_load(const double* const (&ap)[TPW], int64_t g,
                                          double (&av)[TPW][2]) {
#pragma unroll
  for (int i = 0; i < TPW; i++)
    if (ap[i]) load_q(ap[i], g, av[i]);
}

// beta and s from the SpMV (one warp): row block r of nr adds its share of the SpMV CTAs'
// sums (in CTA order) into dst[0] and dst[1] of its partials row, so that the final sums
// take them with the columns
__device__ __noinline__ void add_dots(double* __restrict__ dst, const double* __restrict__ dots,
                                      int r, int nr, int ndots) {
  const int lane = threadIdx.x & 31;
  const int c0 = (int)((int64_t)r * ndots / nr), c1 = (int)((int64_t)(r + 1) * ndots / nr);
  double ab = 0.0, as = 0.0;
  for (int c = c0 + lane; c < c1; c += 32) {
    ab += __ldcg(dots + 2 * c);
    as += __ldcg(dots + 2 * c + 1);
  }
  ab = warp_sum(ab);
  as = warp_sum(as);
  if (lane == 0) { dst[0] = ab; dst[1] = as; }
}

// most warps of a row-split offload reduction CTA (rsub > 1); the task counts that take
// the row split on long vectors, and the warps per CTA it aims at
constexpr int F64X_RSUB_MAXW = 16;
constexpr int F64X_RSUB_TASKS = 4;
constexpr int F64X_RSUB_WARPS = 8;

// Fused DCGS2 reduction, FP64 with offload (EPI_DCGS2 only).  The choice between the
// float-float and the FP64 evaluation of S is made once per loop iteration,
// warp-uniformly, around the whole iteration: a small per-column branch is turned into
// predicated code by the compiler, and an FP64 FMA issued with every lane predicated off
// still holds the FP64 pipe for its full issue time.  GR row groups per iteration (all
// loads issued before any arithmetic).
//
// With rsub > 1 (few tasks on long vectors) the CTA's warps form rsub row sub-blocks of
// nw / rsub task warps each: every sub-block walks its share of the CTA's rows with the
// whole task set, so that more warps per SM have loads in flight, and the sub-blocks'
// sums are added in shared memory in sub-block order before the CTA writes its partials.
//
// A warp's sums of its slots come from one butterfly (warp_sum_multi).  With beta and s
// from the SpMV (ndots > 0), the first warp of each row block's subset-0 CTA adds its share
// of the SpMV CTAs' sums into the row (add_dots).  The rows are then summed in two levels
// (tree_arrive, tree_epilogue) and the completing CTA runs the scalar step.
template <int TPW, int GR>
__global__ void __launch_bounds__(1024)
k_reduce_f64x(const double* __restrict__ Q, int64_t ldq, int k, const double* __restrict__ x,
              const double* __restrict__ y, int64_t m, double* __restrict__ partials,
              unsigned int* __restrict__ counter, Scalars* __restrict__ sc, StepArgs sa,
              int nsplit, int nt, int epi, const double* __restrict__ dots, int ndots,
              int rsub, unsigned int* __restrict__ gcount) {
  pdl_wait();
  if (sc->stop) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5) / rsub;     // task warps per row sub-block
  const int wt = warp % nw, rs = warp / nw;
  const int h = blockIdx.x % nsplit, r = blockIdx.x / nsplit, nr = gridDim.x / nsplit;
  const int tmax = ndots ? k : k + 2;             // tasks of this launch (columns first)
  int tk[TPW];
  const double* ap[TPW];
  double ac[TPW], as64[TPW];
  float sh[TPW], sl[TPW];
#pragma unroll
  for (int i = 0; i < TPW; i++) {
    const int tl = wt + nw * i;                        // task within the subset
    tk[i] = tl < nt && h * nt + tl < tmax ? h * nt + tl : k + 2;   // k + 2: idle slot
    ap[i] = f64x_operand(Q, ldq, k, x, y, tk[i]);
    ac[i] = 0.0; as64[i] = 0.0; sh[i] = 0.0f; sl[i] = 0.0f;
  }
  bool busy = false;                             // a warp without a task skips the rows
#pragma unroll
  for (int i = 0; i < TPW; i++) busy |= ap[i] != nullptr;
  const int64_t ngroups = m / 2;
  const int64_t b0 = (int64_t)r * ngroups / nr, b1 = (int64_t)(r + 1) * ngroups / nr;
  const int64_t g0 = b0 + (b1 - b0) * rs / rsub;
  const int64_t g1 = busy ? b0 + (b1 - b0) * (rs + 1) / rsub : g0;
  int64_t g = g0 + lane;
  if (GR == 2) {
    for (; g + 32 < g1; g += 64) {
      double xa[2], ya[2], xb[2], yb[2], qa[TPW][2], qb[TPW][2];
      ldv(x, g, xa);
      ldv(y, g, ya);
      ldv(x, g + 32, xb);
      ldv(y, g + 32, yb);
      f64x_load<TPW>(ap, g, qa);
      f64x_load<TPW>(ap, g + 32, qb);
      const bool ok = f64x_in_range<TPW>(tk, k, xa, ya, qa) & f64x_in_range<TPW>(tk, k, xb, yb, qb);
      if (__builtin_expect(__all_sync(__activemask(), ok), 1)) {
        f64x_group<TPW, true>(tk, k, xa, ya, qa, ac, as64, sh, sl);
        f64x_group<TPW, true>(tk, k, xb, yb, qb, ac, as64, sh, sl);
      } else {
        f64x_group<TPW, false>(tk, k, xa, ya, qa, ac, as64, sh, sl);
        f64x_group<TPW, false>(tk, k, xb, yb, qb, ac, as64, sh, sl);
      }
    }
  }
  for (; g < g1; g += 32) {
    double xa[2], ya[2], qa[TPW][2];
    ldv(x, g, xa);
    ldv(y, g, ya);
    f64x_load<TPW>(ap, g, qa);
    if (__builtin_expect(__all_sync(__activemask(), f64x_in_range<TPW>(tk, k, xa, ya, qa)), 1))
      f64x_group<TPW, true>(tk, k, xa, ya, qa, ac, as64, sh, sl);
    else
      f64x_group<TPW, false>(tk, k, xa, ya, qa, ac, as64, sh, sl);
  }
  if (r == nr - 1 && rs == 0 && busy) {          // ragged tail (m odd): FP64
    for (int64_t row = ngroups * 2 + lane; row < m; row += 32) {
      const double xs = __ldcg(x + row), ys1 = __ldcg(y + row);
#pragma unroll
      for (int i = 0; i < TPW; i++) {
        if (!ap[i]) continue;
        const double a = __ldcg(ap[i] + row);
        ac[i] = fma(a, xs, ac[i]);
        if (tk[i] < k) as64[i] = fma(a, ys1, as64[i]);   // S of columns only
      }
    }
  }
  // the warp's 2 TPW sums in one butterfly: value 2 i is C (or beta, s) of slot i, 2 i + 1
  // its S; lane l < 2 TPW ends with value l
  constexpr int V = TPW == 1 ? 2 : (TPW == 2 ? 4 : 8);
  double xs[V];
#pragma unroll
  for (int i = 0; i < V / 2; i++) {
    xs[2 * i] = i < TPW ? ac[i] : 0.0;
    xs[2 * i + 1] = i < TPW ? as64[i] + (f2d_bits(sh[i]) + f2d_bits(sl[i])) : 0.0;
  }
  double mine = warp_sum_multi<V>(xs);
  __shared__ double red[F64X_RSUB_MAXW][2 * TPW];   // sub-block sums (rsub > 1)
  if (rsub > 1) {
    if (lane < 2 * TPW) red[warp][lane] = mine;
    __syncthreads();
    if (rs == 0 && lane < 2 * TPW)
      for (int q = 1; q < rsub; q++) mine += red[q * nw + wt][lane];
  }
  if (rs == 0 && lane < 2 * TPW) {
    int t = k + 2;                                   // the task of slot lane / 2
#pragma unroll
    for (int i = 0; i < TPW; i++)
      if ((lane >> 1) == i) t = tk[i];
    double* pp = partials + (int64_t)r * PSTRIDE;    // row block r: one writer per entry
    if (t < k) pp[2 * t + (lane & 1)] = mine;
    else if (t <= k + 1 && (lane & 1) == 0) pp[2 * k + (t - k)] = mine;   // beta, s
  }
  if (ndots && h == 0 && warp == 0) add_dots(partials + (int64_t)r * PSTRIDE + 2 * k, dots, r, nr, ndots);
  pdl_trigger();
  if (!tree_arrive(partials, nr, nsplit, 2 * k + 2, counter, gcount)) return;
  tree_epilogue(partials, nr, k, 2, sc, epi, sa);
}

// The first DCGS2 steps in one pass (k <= FUSE_KMAX basis columns, FP64 offload mode): one
// thread per row forms v_r = (A w)_r with the row arithmetic of k_spmv / k_stencil7 (so v
// is bitwise the SpMV's), writes it, and adds to the step's sums: C_t = q_t^T w (FP64),
// S_t = q_t^T v (float-float; FP64 for the whole warp's row when an operand is outside the
// split's range), beta = w^T w and s = w^T v (FP64).  The CTA's sums are combined in warp
// order into its partials row ([C_0, S_0, ..., beta, s], as the fused reduction stores
// them) and the last CTA runs the scalar step.  Against the SpMV followed by the
// reduction this saves one launch with its tail and one read of w and of v, but the pass
// stays bound by its 9 + k FP64 operations per row: measured at m = 16 M it takes the time
// of the two launches it replaces (2.02 against 1.98 ms for k = 0..4), so it is opt-in
// (kc_set_staged flag 8).
constexpr int FUSE_KMAX = 4;

// K = k, the step's basis columns, is a template argument so that each step keeps only the
// accumulators it uses (the registers bound the resident warps of the matvec's gathers).
template <bool STENCIL, int K>
__global__ void __launch_bounds__(256, K <= 1 ? 8 : (K == 2 ? 6 : 5))
k_spmv_reduce_small(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                    const double* __restrict__ val, int nx, int ny, int nz, Stencil7<double> c,
                    const double* __restrict__ Q, int64_t ldq,
                    const double* __restrict__ x, double* __restrict__ y, int64_t m,
                    double* __restrict__ partials, unsigned int* __restrict__ counter,
                    Scalars* __restrict__ sc, StepArgs sa) {
  constexpr int KA = K > 0 ? K : 1;                 // (array extent; unused when K = 0)
  const int k = K;
  pdl_wait();
  if (sc->stop) return;
  double ac[KA], as64[KA];
  float sh[KA], sl[KA];
#pragma unroll
  for (int t = 0; t < KA; t++) { ac[t] = 0.0; as64[t] = 0.0; sh[t] = 0.0f; sl[t] = 0.0f; }
  double ab = 0.0, as = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    double qv[KA];
#pragma unroll
    for (int t = 0; t < K; t++) qv[t] = __ldcs(Q + (int64_t)t * ldq + r);
    const double vr = STENCIL ? stencil_row(x, r, nx, ny, nz, c)
                              : csr_row<double>(rp, ci, val, x, r);
    y[r] = vr;
    const double xr = __ldcg(x + r);
    ab = fma(xr, xr, ab);
    as = fma(xr, vr, as);
    if (K > 0) {
      bool ok = split_fast_ok(vr);
#pragma unroll
      for (int t = 0; t < K; t++) ok = ok & split_fast_ok(qv[t]);
      if (__builtin_expect(__all_sync(__activemask(), ok), 1)) {
        float vh, vl;
        split_fast(vr, vh, vl);
#pragma unroll
        for (int t = 0; t < K; t++) {
          ac[t] = fma(qv[t], xr, ac[t]);
          float qh, ql;
          split_fast(qv[t], qh, ql);
          df_mac(sh[t], sl[t], qh, ql, vh, vl);
        }
      } else {
#pragma unroll
        for (int t = 0; t < K; t++) {
          ac[t] = fma(qv[t], xr, ac[t]);
          as64[t] = fma(qv[t], vr, as64[t]);
        }
      }
    }
  }
  pdl_trigger();
  // CTA sums in warp order: [2t] = C_t, [2t + 1] = S_t, [2k] = beta, [2k + 1] = s
  __shared__ double red[8][2 * FUSE_KMAX + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < K; t++) {
    const double cv = warp_sum(ac[t]);
    const double sv = warp_sum(as64[t] + (f2d_bits(sh[t]) + f2d_bits(sl[t])));
    if (lane == 0) { red[warp][2 * t] = cv; red[warp][2 * t + 1] = sv; }
  }
  ab = warp_sum(ab);
  as = warp_sum(as);
  if (lane == 0) { red[warp][2 * k] = ab; red[warp][2 * k + 1] = as; }
  __syncthreads();
  if ((int)threadIdx.x < 2 * k + 2) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * PSTRIDE + threadIdx.x] = t;
  }
  if (!last_cta(counter)) return;
  reduce_epilogue(partials, k, 2, sc, EPI_DCGS2, sa, (int)gridDim.x);
}

// One group of two rows of the one-vector reduction for every slot: ac += a . x in FP64,
// or for a column with OFF, (sh, sl) += a . x in float-float.
template <int TPW, bool OFF>
__device__ __forceinline__ void r1_group(const int (&tk)[TPW], int k, const double (&xv)[2],
                                         const double (&av)[TPW][2], double* ac, float* sh,
                                         float* sl) {
  float xh[2], xl[2];
  if (OFF) { split_fast(xv[0], xh[0], xl[0]); split_fast(xv[1], xh[1], xl[1]); }
#pragma unroll
  for (int i = 0; i < TPW; i++) {
    if (tk[i] > k) continue;                     // idle slot (warp-uniform)
    if (OFF && tk[i] < k) {
      float ah[2], al[2];
      split_fast(av[i][0], ah[0], al[0]);
      split_fast(av[i][1], ah[1], al[1]);
      df_mac(sh[i], sl[i], ah[0], al[0], xh[0], xl[0]);
      df_mac(sh[i], sl[i], ah[1], al[1], xh[1], xl[1]);
    } else {
      ac[i] = fma(av[i][0], xv[0], ac[i]);
      ac[i] = fma(av[i][1], xv[1], ac[i]);
    }
  }
}

// true when x and every column operand of the group lie in split_fast's range
template <int TPW>
__device__ __forceinline__ bool r1_in_range(const int (&tk)[TPW], int k, const double (&xv)[2],
                                            const double (&av)[TPW][2]) {
  bool ok = split_fast_ok(xv[0]) & split_fast_ok(xv[1]);
#pragma unroll
  for (int i = 0; i < TPW; i++)
    if (tk[i] < k) ok = ok & split_fast_ok(av[i][0]) & split_fast_ok(av[i][1]);
  return ok;
}

// Q_k^T x and x^T x (one vector: the CGS2 finish's projections) with the offload
// reduction's task layout: tasks t < k are columns, task k is x^T x; GR row groups per
// iteration with all loads first.  Partials hold the k + 1 sums of each row block in task
// order.  With OFF (the first projection, C1 = Q^T w, whose error the second projection
// removes, as for S in the DCGS2 step) the columns are summed in float-float on the
// FP32/INT pipes (warp-uniformly per iteration, FP64 for operands outside the range);
// otherwise, and always for x^T x, every product is an FP64 FMA.
template <int TPW, int GR, bool OFF>
__global__ void __launch_bounds__(1024)
k_reduce1_f64(const double* __restrict__ Q, int64_t ldq, int k, const double* __restrict__ x,
              int64_t m, double* __restrict__ partials, unsigned int* __restrict__ counter,
              Scalars* __restrict__ sc, StepArgs sa, int nsplit, int nt, int epi) {
  if (sc->stop) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int h = blockIdx.x % nsplit, r = blockIdx.x / nsplit, nr = gridDim.x / nsplit;
  const double* ap[TPW];
  int tk[TPW];
  double ac[TPW];
  float sh[TPW], sl[TPW];
#pragma unroll
  for (int i = 0; i < TPW; i++) {
    const int tl = warp + nw * i;
    tk[i] = tl < nt ? h * nt + tl : k + 1;             // k + 1 and above: idle slot
    if (tk[i] > k) tk[i] = k + 1;
    ap[i] = tk[i] < k ? Q + (int64_t)tk[i] * ldq : (tk[i] == k ? x : nullptr);
    ac[i] = 0.0;
    sh[i] = 0.0f;
    sl[i] = 0.0f;
  }
  const int64_t ngroups = m / 2;
  const int64_t g0 = (int64_t)r * ngroups / nr;
  const int64_t g1 = (int64_t)(r + 1) * ngroups / nr;
  int64_t g = g0 + lane;
  if (GR == 2) {
    for (; g + 32 < g1; g += 64) {
      double xa[2], xb[2], qa[TPW][2], qb[TPW][2];
      ldv(x, g, xa);
      ldv(x, g + 32, xb);
#pragma unroll
      for (int i = 0; i < TPW; i++)
        if (ap[i]) { load_q(ap[i], g, qa[i]); load_q(ap[i], g + 32, qb[i]); }
      if (OFF && __builtin_expect(__all_sync(__activemask(), r1_in_range<TPW>(tk, k, xa, qa) &
                                                             r1_in_range<TPW>(tk, k, xb, qb)), 1)) {
        r1_group<TPW, OFF>(tk, k, xa, qa, ac, sh, sl);
        r1_group<TPW, OFF>(tk, k, xb, qb, ac, sh, sl);
      } else {
        r1_group<TPW, false>(tk, k, xa, qa, ac, sh, sl);
        r1_group<TPW, false>(tk, k, xb, qb, ac, sh, sl);
      }
    }
  }
  for (; g < g1; g += 32) {
    double xa[2], qa[TPW][2];
    ldv(x, g, xa);
#pragma unroll
    for (int i = 0; i < TPW; i++)
      if (ap[i]) load_q(ap[i], g, qa[i]);
    if (OFF && __builtin_expect(__all_sync(__activemask(), r1_in_range<TPW>(tk, k, xa, qa)), 1))
      r1_group<TPW, OFF>(tk, k, xa, qa, ac, sh, sl);
    else
      r1_group<TPW, false>(tk, k, xa, qa, ac, sh, sl);
  }
  if (r == nr - 1) {                             // ragged tail (m odd)
    for (int64_t row = ngroups * 2 + lane; row < m; row += 32) {
      const double xs = __ldcg(x + row);
#pragma unroll
      for (int i = 0; i < TPW; i++)
        if (ap[i]) ac[i] = fma(__ldcg(ap[i] + row), xs, ac[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < TPW; i++) {
    if (!ap[i]) continue;
    const double c = warp_sum(OFF ? ac[i] + (f2d_bits(sh[i]) + f2d_bits(sl[i])) : ac[i]);
    if (lane == 0) partials[(int64_t)r * PSTRIDE + tk[i]] = c;
  }
  if (!last_cta(counter)) return;
  reduce_epilogue(partials, k, 1, sc, epi, sa, nr);
}

// ----------------------------------------------------------------------------------------
// The CGS2 finish's middle passes in one: u = w - Q_k C1 (row-local) and the sums
// [Q_k^T u, u^T u] of the second projection, over tiles of PR_TR rows of Q staged in shared
// memory (double-buffered 16-byte asynchronous copies), so the basis is read once for both.
// u is formed as in k_gemv_sub with allow32: FP32 products of the truncated entries when
// (k + 3) 2^-24 ||C1||_1 <= 2^-53 ||w - Q C1||, else FP64 (decided per launch from the
// device scalars); the sums are FP64, accumulated per (task, row) slot across tiles and
// combined in a fixed order, then stored by the last CTA like a one-vector reduction
// (EPI_STORE_C2: C2 and the squared norm of u).
// ----------------------------------------------------------------------------------------
constexpr int PR_TR = 128;                      // rows per tile
constexpr int PR_THREADS = 4 * PR_TR;           // phase A: four column parts per row
constexpr int PR_MAXK = 64;                     // basis columns the fused pass takes
constexpr int PR_LD = PR_TR;                    // tile column stride (doubles)
constexpr int PR_TPW = (PR_MAXK + 1 + PR_THREADS / 32 - 1) / (PR_THREADS / 32);  // tasks per warp

__device__ __forceinline__ void pr_cp16(void* dst, const void* src) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(d), "l"(src) : "memory");
}

__global__ void __launch_bounds__(PR_THREADS)
k_proj_reduce(const double* __restrict__ Q, int64_t ldq, int k, double* __restrict__ w,
              int64_t m, double* __restrict__ partials, unsigned int* __restrict__ counter,
              Scalars* __restrict__ sc, StepArgs sa) {
  if (sc->stop) return;
  extern __shared__ double pr_smem[];
  double* tile = pr_smem;                                // 2 x k x PR_LD
  __shared__ double su[PR_TR];
  __shared__ float zp32[4][PR_TR];
  __shared__ double zp64[4][PR_TR];
  __shared__ float sf[PR_MAXK];
  __shared__ double sd[PR_MAXK];
  __shared__ double s_scale;
  __shared__ int s_fast;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < k; i += PR_THREADS) sd[i] = sc->C[i];
  if (tid == 0) {
    double cmax = 0.0, l1 = 0.0, c2 = 0.0;
    for (int i = 0; i < k; i++) {
      const double c = sc->C[i];
      cmax = fmax(cmax, fabs(c));
      l1 += fabs(c);
      c2 += c * c;
    }
    const double rest = sc->norm_sq - c2;
    int ex = 0;
    if (cmax > 0.0) frexp(cmax, &ex);
    s_scale = ldexp(1.0, ex);
    s_fast = (rest > 0.0 && cmax > 0.0 && ex > -900 &&
              l1 * (double)(k + 3) <= 0x1p-29 * sqrt(rest)) ? 1 : 0;
  }
  __syncthreads();
  const bool fast = s_fast;
  const double scale = s_scale;
  for (int i = tid; i < k; i += PR_THREADS) sf[i] = d2f_trunc(sd[i] / scale);
  // phase-B slots: warp w owns tasks w, w + 16, ... (columns, then u^T u as task k); its
  // lanes own rows lane, lane + 32, ... of every tile
  double acc[PR_TPW];
#pragma unroll
  for (int i = 0; i < PR_TPW; i++) acc[i] = 0.0;
  const int64_t ntiles = m / PR_TR;                       // whole tiles; the rest below
  auto fetch = [&](int64_t t, int buf) {
    const int64_t r0 = t * PR_TR;
    double* dst = tile + (size_t)buf * k * PR_LD;
    for (int e = tid; e < k * (PR_TR / 2); e += PR_THREADS) {
      const int j = e / (PR_TR / 2), c2 = e % (PR_TR / 2);
      pr_cp16(dst + j * PR_LD + 2 * c2, Q + (int64_t)j * ldq + r0 + 2 * c2);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int buf = 0;
  int64_t t = blockIdx.x;
  if (t < ntiles) fetch(t, 0);
  for (; t < ntiles; t += gridDim.x, buf ^= 1) {
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) {
      fetch(tn, buf ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const double* tb = tile + (size_t)buf * k * PR_LD;
    const int64_t r0 = t * PR_TR;
    // phase A: u = w - Q C1; thread (part, row) sums the columns j = part mod 4
    {
      const int row = tid % PR_TR, part = tid / PR_TR;
      if (fast) {
        float z = 0.0f;
        for (int j = part; j < k; j += 4) z = fmaf(d2f_trunc(tb[j * PR_LD + row]), sf[j], z);
        zp32[part][row] = z;
      } else {
        double z = 0.0;
        for (int j = part; j < k; j += 4) z = fma(tb[j * PR_LD + row], sd[j], z);
        zp64[part][row] = z;
      }
    }
    __syncthreads();
    if (tid < PR_TR) {
      double u;
      if (fast) {
        const float z = (zp32[0][tid] + zp32[1][tid]) + (zp32[2][tid] + zp32[3][tid]);
        u = fma(-f2d_bits(z), scale, __ldcg(w + r0 + tid));
      } else {
        u = __ldcg(w + r0 + tid) -
            ((zp64[0][tid] + zp64[1][tid]) + (zp64[2][tid] + zp64[3][tid]));
      }
      su[tid] = u;
      w[r0 + tid] = u;
    }
    __syncthreads();
    // phase B: the sums of the second projection
#pragma unroll
    for (int i = 0; i < PR_TPW; i++) {
      const int task = warp + (PR_THREADS / 32) * i;
      if (task > k) break;
      const double* col = task < k ? tb + task * PR_LD : su;
#pragma unroll
      for (int j = 0; j < PR_TR / 32; j++)
        acc[i] = fma(col[lane + 32 * j], su[lane + 32 * j], acc[i]);
    }
    __syncthreads();                                     // the buffer is refilled next
  }
  // rows past the last whole tile (fewer than PR_TR): the last CTA's warp 0, FP64
  if (blockIdx.x == gridDim.x - 1) {
    for (int64_t row = ntiles * PR_TR + tid; row < m; row += PR_THREADS) {
      double z = 0.0;
      for (int j = 0; j < k; j++) z = fma(__ldcg(Q + (int64_t)j * ldq + row), sd[j], z);
      w[row] = __ldcg(w + row) - z;
    }
    __syncthreads();
    for (int64_t row = ntiles * PR_TR + lane; row < m; row += 32) {
      const double u = __ldcg(w + row);
#pragma unroll
      for (int i = 0; i < PR_TPW; i++) {
        const int task = warp + (PR_THREADS / 32) * i;
        if (task > k) break;
        const double a = task < k ? __ldcg(Q + (int64_t)task * ldq + row) : u;
        acc[i] = fma(a, u, acc[i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < PR_TPW; i++) {
    const int task = warp + (PR_THREADS / 32) * i;
    if (task > k) break;
    const double v = warp_sum(acc[i]);
    if (lane == 0) partials[(int64_t)blockIdx.x * PSTRIDE + task] = v;
  }
  if (!last_cta(counter)) return;
  reduce_epilogue(partials, k, 1, sc, EPI_STORE_C2, sa);
}

// Two basis columns of the offloaded update for one group of two rows: u -= Q C in
// float-float (OFF) or FP64 (!OFF).
template <bool OFF>
__device__ __forceinline__ void f64x_update_pair(const double (&q)[2][2], const double* sC,
                                                 const float* cH, const float* cL, int i,
                                                 double (&u64)[2], float (&zh)[2],
                                                 float (&zl)[2]) {
#pragma unroll
  for (int j = 0; j < 2; j++) {
    if (OFF) {
      float h0, l0, h1, l1;
      split_df(q[j][0], h0, l0);
      split_df(q[j][1], h1, l1);
      df_mac(zh[0], zl[0], h0, l0, cH[i + j], cL[i + j]);
      df_mac(zh[1], zl[1], h1, l1, cH[i + j], cL[i + j]);
    } else {
      u64[0] = fma(-q[j][0], sC[i + j], u64[0]);
      u64[1] = fma(-q[j][1], sC[i + j], u64[1]);
    }
  }
}

// below this many basis columns the fast update takes two row groups per thread
constexpr int UPD_PAIR_K = 64;

// FP32 ("fast") products of the offloaded update for NG row groups gg: w <- v/alpha - Q T
// - q T_k in FP64 and q = w / alpha - (Q C) / alpha with the FP32 products, in chunks of CH
// columns whose loads are all issued before their arithmetic; the last, partial chunk is
// predicated so that its loads are in flight together too.  z = Q (C / scale) in FP32 is
// scaled by cf = scale / alpha in FP32 as well, so that q takes one FP64 FMA per row.
template <int NG, int CH>
__device__ __forceinline__ void upd_fast_rows(const double* __restrict__ Q, int64_t ldq, int k,
                                              double* __restrict__ w,
                                              const double* __restrict__ v,
                                              double* __restrict__ qk, const int64_t (&gg)[NG],
                                              const double* sT, const float* cH, double vsc,
                                              double inva, float cf) {
  double wv[NG][2], wn[NG][2];
  float z[NG][2];
#pragma unroll
  for (int n = 0; n < NG; n++) {
    double vv[2];
    ldv_cg(w, gg[n], wv[n]);
    ldv_cg(v, gg[n], vv);
    wn[n][0] = vv[0] * vsc;
    wn[n][1] = vv[1] * vsc;
    z[n][0] = 0.0f;
    z[n][1] = 0.0f;
  }
  int i = 0;
  for (; i + CH <= k; i += CH) {
    double q[CH][NG][2];
#pragma unroll
    for (int j = 0; j < CH; j++)
#pragma unroll
      for (int n = 0; n < NG; n++) load_q(Q + (int64_t)(i + j) * ldq, gg[n], q[j][n]);
#pragma unroll
    for (int j = 0; j < CH; j++)
#pragma unroll
      for (int n = 0; n < NG; n++)
#pragma unroll
        for (int r = 0; r < 2; r++) {
          wn[n][r] = fma(-q[j][n][r], sT[i + j], wn[n][r]);
          z[n][r] = fmaf(d2f_trunc(q[j][n][r]), cH[i + j], z[n][r]);
        }
  }
  if (i < k) {
    double q[CH][NG][2];
#pragma unroll
    for (int j = 0; j < CH; j++)
#pragma unroll
      for (int n = 0; n < NG; n++) {
        if (i + j < k) {
          load_q(Q + (int64_t)(i + j) * ldq, gg[n], q[j][n]);
        } else {
          q[j][n][0] = 0.0;
          q[j][n][1] = 0.0;
        }
      }
#pragma unroll
    for (int j = 0; j < CH; j++) {
      if (i + j < k) {
#pragma unroll
        for (int n = 0; n < NG; n++)
#pragma unroll
          for (int r = 0; r < 2; r++) {
            wn[n][r] = fma(-q[j][n][r], sT[i + j], wn[n][r]);
            z[n][r] = fmaf(d2f_trunc(q[j][n][r]), cH[i + j], z[n][r]);
          }
      }
    }
  }
#pragma unroll
  for (int n = 0; n < NG; n++) {
    double qn[2], wo[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      qn[r] = fma(wv[n][r], inva, -f2d_bits(z[n][r] * cf));
      wo[r] = fma(-qn[r], sT[k], wn[n][r]);
    }
    store_q(qk, gg[n], qn);
    stv(w, gg[n], wo);
  }
}

// DCGS2 update, FP64 with offload: u = w - Q C with C scaled by a power of two into float
// range, w <- v/alpha - Q T - q T_k in FP64.  Q C is small against w (C holds the delayed
// reorthogonalisation coefficients), so it needs far fewer correct digits than the FP64
// terms: in FP32 (basis entries truncated to 24 bits, k-term FP32 sums, the product by
// scale / alpha) its error per row of q is at most (k + 4) 2^-24 sum_j |q_j| |C_j| / alpha,
// whose 2-norm is at most (k + 4) 2^-24 ||C||_1 / alpha; when that is below 2^-53 (the FP64
// rounding of the unit vector q itself; alpha = ||w - Q C||) the
// launch takes the FP32 products ("fast"), otherwise float-float (split doubles, exact
// leading products), and FP64 for operands outside the float-float range (warp-uniform
// per pair of columns, see k_reduce_f64x).  The choice is made per launch from the device
// scalars, identically in every CTA.
__global__ void __launch_bounds__(UPD_THREADS, 4)
k_dcgs2_update_f64x(double* __restrict__ Q, int64_t ldq, int k, double* __restrict__ w,
                    const double* __restrict__ v, int64_t m, const Scalars* __restrict__ sc,
                    int allow32) {
  pdl_wait();
  if (sc->stop) return;
  __shared__ double sC[NMAX + 1], sT[NMAX + 1];
  __shared__ float cH[NMAX + 1], cL[NMAX + 1];
  __shared__ double s_scale;
  __shared__ float s_cf;
  __shared__ int s_cok, s_fast;
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    sC[i] = i < k ? sc->C[i] : 0.0;            // sC[k] = 0 pads an odd k to a column pair
    sT[i] = sc->T[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double cmax = 0.0, l1 = 0.0;
    for (int i = 0; i < k; i++) {
      cmax = fmax(cmax, fabs(sC[i]));
      l1 += fabs(sC[i]);
    }
    int ex = 0;
    if (cmax > 0.0) frexp(cmax, &ex);
    s_scale = ldexp(1.0, ex);                 // C / scale lies in (-1, 1)
    s_cok = 1;
    // 0x1p-29 = 2^-53 / 2^-24; l1 is FP64 (relative error far below the bound's margin);
    // the FP32 factor scale / alpha must be a normal float small enough that z cf (|z| <= k)
    // stays finite
    const double cf = s_scale * sc->inv_alpha;
    s_cf = (float)cf;
    s_fast = (allow32 && l1 * (double)(k + 4) <= 0x1p-29 * sc->alpha && fabs(cf) >= 0x1p-120 &&
              fabs(cf) <= 0x1p100) ? 1 : 0;
  }
  __syncthreads();
  __shared__ double s_inv_scale;
  if (threadIdx.x == 0) {                     // exact: a power of two, without a division
    int ex = 0;
    frexp(s_scale, &ex);
    s_inv_scale = ldexp(1.0, 1 - ex);
  }
  __syncthreads();
  const double inv_scale = s_inv_scale;
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    float h, l;
    if (!split_df(sC[i] * inv_scale, h, l)) { h = 0.0f; l = 0.0f; if (sC[i] != 0.0) s_cok = 0; }
    cH[i] = h;
    cL[i] = l;
  }
  __syncthreads();
  const bool cok = s_cok;
  const double inva = sc->inv_alpha, vsc = sc->vscale, scale = s_scale;
  double* qk = Q + (int64_t)k * ldq;
  const int64_t ngroups = m / 2;
  if (s_fast && cok) {
    // cH holds C / scale truncated to 24 bits (the leading float of its split); with the
    // truncated basis entries that is 2 x 2^-23 of each product, the FP32 sum adds at most
    // (k - 1) 2^-24, and cf and the product z cf two more roundings of 2^-24: together the
    // (k + 4) 2^-24 of the bound above (relative to sum_j |q_j| |C_j| / alpha)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < UPD_PAIR_K) {
      // few columns: the pass is HBM-latency bound, so each thread takes two row groups
      // a grid stride apart and issues all their loads before the arithmetic
      for (; g + stride < ngroups; g += 2 * stride) {
        const int64_t gg[2] = {g, g + stride};
        upd_fast_rows<2, 4>(Q, ldq, k, w, v, qk, gg, sT, cH, vsc, inva, s_cf);
      }
    }
    for (; g < ngroups; g += stride) {
      const int64_t gg[1] = {g};
      upd_fast_rows<1, 8>(Q, ldq, k, w, v, qk, gg, sT, cH, vsc, inva, s_cf);
    }
  } else
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    double wv[2], vv[2];
    ldv_cg(w, g, wv);
    ldv_cg(v, g, vv);
    double wn[2] = {vv[0] * vsc, vv[1] * vsc};
    double u64[2] = {wv[0], wv[1]};
    float zh[2] = {0.0f, 0.0f}, zl[2] = {0.0f, 0.0f};
    int i = 0;
    for (; i + 4 <= k; i += 4) {        // four columns' loads in flight before arithmetic
      double q[2][2], q2[2][2];
#pragma unroll
      for (int j = 0; j < 2; j++) load_q(Q + (int64_t)(i + j) * ldq, g, q[j]);
#pragma unroll
      for (int j = 0; j < 2; j++) load_q(Q + (int64_t)(i + 2 + j) * ldq, g, q2[j]);
#pragma unroll
      for (int j = 0; j < 2; j++) {
        wn[0] = fma(-q[j][0], sT[i + j], wn[0]);
        wn[1] = fma(-q[j][1], sT[i + j], wn[1]);
        wn[0] = fma(-q2[j][0], sT[i + 2 + j], wn[0]);
        wn[1] = fma(-q2[j][1], sT[i + 2 + j], wn[1]);
      }
      const bool ok = cok & df_in_range(q[0][0]) & df_in_range(q[0][1]) &
                      df_in_range(q[1][0]) & df_in_range(q[1][1]) &
                      df_in_range(q2[0][0]) & df_in_range(q2[0][1]) &
                      df_in_range(q2[1][0]) & df_in_range(q2[1][1]);
      if (__builtin_expect(__all_sync(__activemask(), ok), 1)) {
        f64x_update_pair<true>(q, sC, cH, cL, i, u64, zh, zl);
        f64x_update_pair<true>(q2, sC, cH, cL, i + 2, u64, zh, zl);
      } else {
        f64x_update_pair<false>(q, sC, cH, cL, i, u64, zh, zl);
        f64x_update_pair<false>(q2, sC, cH, cL, i + 2, u64, zh, zl);
      }
    }
    for (; i + 2 <= k; i += 2) {
      double q[2][2];
#pragma unroll
      for (int j = 0; j < 2; j++) load_q(Q + (int64_t)(i + j) * ldq, g, q[j]);
#pragma unroll
      for (int j = 0; j < 2; j++) {
        wn[0] = fma(-q[j][0], sT[i + j], wn[0]);
        wn[1] = fma(-q[j][1], sT[i + j], wn[1]);
      }
      const bool ok = cok & df_in_range(q[0][0]) & df_in_range(q[0][1]) &
                      df_in_range(q[1][0]) & df_in_range(q[1][1]);
      if (__builtin_expect(__all_sync(__activemask(), ok), 1))
        f64x_update_pair<true>(q, sC, cH, cL, i, u64, zh, zl);
      else
        f64x_update_pair<false>(q, sC, cH, cL, i, u64, zh, zl);
    }
    if (i < k) {                        // odd k: the last column, paired with a zero one
      double q[2][2];
      load_q(Q + (int64_t)i * ldq, g, q[0]);
      q[1][0] = 0.0;
      q[1][1] = 0.0;
      wn[0] = fma(-q[0][0], sT[i], wn[0]);
      wn[1] = fma(-q[0][1], sT[i], wn[1]);
      const bool ok = cok & df_in_range(q[0][0]) & df_in_range(q[0][1]);
      if (__all_sync(__activemask(), ok))
        f64x_update_pair<true>(q, sC, cH, cL, i, u64, zh, zl);
      else
        f64x_update_pair<false>(q, sC, cH, cL, i, u64, zh, zl);
    }
    double qn[2], wo[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const double u = fma(-f2d_bits(zh[r]), scale, fma(-f2d_bits(zl[r]), scale, u64[r]));
      qn[r] = u * inva;
      wo[r] = fma(-qn[r], sT[k], wn[r]);
    }
    store_q(qk, g, qn);
    stv(w, g, wo);
  }
  pdl_trigger();
  if (blockIdx.x == 0) {        // ragged tail: FP64
    for (int64_t row = ngroups * 2 + threadIdx.x; row < m; row += blockDim.x) {
      double u = w[row], wn1 = v[row] * vsc;
      for (int i = 0; i < k; i++) {
        const double q = __ldcg(Q + (int64_t)i * ldq + row);
        u = fma(-q, sC[i], u);
        wn1 = fma(-q, sT[i], wn1);
      }
      const double qn1 = u * inva;
      qk[row] = qn1;
      w[row] = fma(-qn1, sT[k], wn1);
    }
  }
}

// Explicit-norm fallback of the delayed normalisation: when the epilogue found
// beta - C^T C too small to trust (reduced precision), alpha = ||w - Q_k C|| is computed
// by one more pass and the scalar step runs here.  Returns at once otherwise.
template <typename TQ, typename TV>
__global__ void __launch_bounds__(UPD_THREADS)
k_fallback_norm(const TQ* __restrict__ Q, int64_t ldq, int k, const TV* __restrict__ w,
                int64_t m, double* __restrict__ partials, unsigned int* __restrict__ counter,
                Scalars* __restrict__ sc, StepArgs sa) {
  using TA = typename Acc<TV>::T;
  constexpr int R = Grp<TV>::R;
  if (sc->stop || !sc->fallback) return;
  __shared__ TA sc_[NMAX];
  for (int i = threadIdx.x; i < k; i += blockDim.x) sc_[i] = (TA)sc->C[i];
  __syncthreads();
  double acc = 0.0;
  const int64_t ngroups = m / R;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    TV xv[R];
    ldv_cg(w, g, xv);
    TA u[R];
#pragma unroll
    for (int r = 0; r < R; r++) u[r] = xv[r];
    for (int i = 0; i < k; i++) {
      TA q0[R];
      load_q(Q + (int64_t)i * ldq, g, q0);
#pragma unroll
      for (int r = 0; r < R; r++) u[r] -= q0[r] * sc_[i];
    }
#pragma unroll
    for (int r = 0; r < R; r++) acc += (double)u[r] * (double)u[r];
  }
  if (blockIdx.x == 0)
    for (int64_t row = ngroups * R + threadIdx.x; row < m; row += blockDim.x) {
      TA u = (TA)w[row];
      for (int i = 0; i < k; i++) u -= (TA)ld1(Q + (int64_t)i * ldq, row) * sc_[i];
      acc += (double)u * (double)u;
    }
  __shared__ double red[UPD_THREADS / 32];
  double v = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0;
    for (int i = 0; i < UPD_THREADS / 32; i++) s0 += red[i];
    partials[(int64_t)blockIdx.x * PSTRIDE] = s0;
  }
  if (!last_cta(counter)) return;
  __shared__ double tot[1];
  __shared__ double s_alpha, s_inva;
  sum_partials(partials, gridDim.x, 1, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    s_alpha = sqrt(tot[0]);
    s_inva = 1.0 / s_alpha;
    sc->fallback = 0;
    sc->pyth_fallbacks++;
    if (!(s_alpha > 0.0)) set_status(sc, KC_ERR_BREAKDOWN);
  }
  __syncthreads();
  scalar_step(sc, sa, k, s_alpha, s_inva);
}

// The epilogue of a norm / dot reduction from xx = x^T x and xy = x^T y (one thread).
__device__ void norm_epilogue(double xx, double xy, Scalars* __restrict__ sc, int nepi,
                              const StepArgs& sa) {
  const int k = sa.k;
  sc->norm_sq = xx;
  if (!isfinite(xx) || !isfinite(xy)) set_status(sc, KC_ERR_NONFINITE);
  if (nepi == NEPI_SQ) return;
  if (nepi == NEPI_DOT) {
    sc->h = xy;
    sa.H[sa.row + (int64_t)(k - 1) * sa.ldh] = xy;       // H(i, k-1), i = sa.row
    return;
  }
  double alpha = sqrt(xx);
  sc->alpha = alpha;
  sc->inv_alpha = 1.0 / alpha;
  sc->vscale = 1.0 / alpha;
  if (nepi == NEPI_INIT) {
    if (!(alpha > 0.0)) set_status(sc, KC_ERR_BREAKDOWN);
    return;
  }
  // finalise column k-1 of H
  double* Hc = sa.H + (int64_t)(k - 1) * sa.ldh;
  double cn = alpha * alpha;
  if (nepi == NEPI_FINISH) {
    for (int i = 0; i < k; i++) {
      Hc[i] = sa.K[i + (int64_t)(k - 1) * sa.ldk] + sc->C[i] + sc->C2[i];
      cn += Hc[i] * Hc[i];
    }
  } else if (nepi == NEPI_CGS2) {
    for (int i = 0; i < k; i++) {
      Hc[i] = sc->S[i] + sc->C[i];
      cn += Hc[i] * Hc[i];
    }
  } else {  // MGS: the inner products are already in H
    for (int i = 0; i < k; i++) cn += Hc[i] * Hc[i];
  }
  Hc[k] = alpha;
  if (alpha <= 1e-13 * sqrt(cn)) set_status(sc, KC_ERR_BREAKDOWN);
  if (sa.flags & SF_GIVENS) givens_column(sc, sa.H, sa.ldh, k - 1, sa.R, sa.ldr);
}

// K3': x^T x (and x^T y) with a last-CTA epilogue (norms, MGS inner products).
template <typename TV, int NRHS>
__global__ void __launch_bounds__(RED_THREADS)
k_norm(const TV* __restrict__ x, const TV* __restrict__ y, int64_t m,
       double* __restrict__ partials, unsigned int* __restrict__ counter,
       Scalars* __restrict__ sc, int nepi, StepArgs sa) {
  using TA = typename Acc<TV>::T;
  constexpr int R = Grp<TV>::R;
  if (sc->stop) return;
  TA a0 = 0, a1 = 0;
  const int64_t ngroups = m / R;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    TV xv[R], yv[R];
    ldv_cg(x, g, xv);
    if (NRHS == 2) ldv_cg(y, g, yv);
#pragma unroll
    for (int r = 0; r < R; r++) {
      a0 += (TA)xv[r] * (TA)xv[r];
      if (NRHS == 2) a1 += (TA)xv[r] * (TA)yv[r];
    }
  }
  if (blockIdx.x == gridDim.x - 1)
    for (int64_t row = ngroups * R + threadIdx.x; row < m; row += blockDim.x) {
      TA xs = (TA)x[row];
      a0 += xs * xs;
      if (NRHS == 2) a1 += xs * (TA)y[row];
    }
  __shared__ double red[2][RED_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double d0 = (double)warp_sum(a0), d1 = NRHS == 2 ? (double)warp_sum(a1) : 0.0;
  if (lane == 0) { red[0][warp] = d0; red[1][warp] = d1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) { s0 += red[0][i]; s1 += red[1][i]; }
    partials[(int64_t)blockIdx.x * PSTRIDE] = s0;
    partials[(int64_t)blockIdx.x * PSTRIDE + 1] = s1;
  }
  if (!last_cta(counter)) return;
  __shared__ double tot[2];
  sum_partials(partials, gridDim.x, 2, tot);
  __syncthreads();
  if (threadIdx.x != 0) return;
  norm_epilogue(tot[0], tot[1], sc, nepi, sa);
}

// qcol = x * inv_alpha (converted to the basis type)
template <typename TQ, typename TV>
__global__ void __launch_bounds__(UPD_THREADS)
k_scale_to(const TV* __restrict__ x, TQ* __restrict__ qcol, int64_t m,
           const Scalars* __restrict__ sc) {
  using TA = typename Acc<TV>::T;
  if (sc->stop) return;
  const TA inva = (TA)sc->inv_alpha;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    TA q = (TA)__ldcg(x + r) * inva;
    st1(qcol, r, q);
  }
}

// v <- v - h q (MGS rank-1 projection; h read from the device scalars)
template <typename TQ, typename TV>
__global__ void __launch_bounds__(UPD_THREADS)
k_axpy_h(const TQ* __restrict__ q, TV* __restrict__ v, int64_t m,
         const Scalars* __restrict__ sc) {
  using TA = typename Acc<TV>::T;
  if (sc->stop) return;
  const TA h = (TA)sc->h;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x)
    v[r] = (TV)((TA)v[r] - h * (TA)ld1(q, r));
}

// ----------------------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------------------
static int grid_for(const kc_ctx* ctx, int64_t work_items, int per_block, int max_per_sm) {
  int64_t b = (work_items + per_block - 1) / per_block;
  int64_t cap = (int64_t)ctx->num_sms * max_per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// The grid of a grid-stride kernel capped at one full wave: `want` CTAs, at most the SM
// count times the CTAs of `kern` that fit on an SM at `threads` per CTA (looked up once
// per call site into `cache`).  A grid of 1216 CTAs that fit six to an SM would otherwise
// run as one full and one third-full wave (the finish's k_gemv_sub: 1.04 -> 0.99 ms; the
// stencil measured no change and the update, two full waves, was slower as one wave).
template <typename K>
static int one_wave(const kc_ctx* ctx, K kern, int threads, int want, std::atomic<int>& cache) {
  int occ = cache.load(std::memory_order_relaxed);
  if (occ == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0) != cudaSuccess ||
        occ < 1)
      occ = 1;
    cache.store(occ, std::memory_order_relaxed);
  }
  const int64_t cap = (int64_t)occ * ctx->num_sms;
  return want < cap ? want : (int)cap;
}

static int reduce_grid_for(const kc_ctx* ctx, int64_t ngroups) {
  // at least ~4 groups per lane before splitting across more CTAs
  int64_t b = (ngroups + 32 * 4 - 1) / (32 * 4);
  if (b > ctx->reduce_grid) b = ctx->reduce_grid;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace kc

#include "kc_reduce_tma.cuh"
#include "kc_reduce_tc.cuh"

namespace kc {

kc_status launch_spmv(kc_ctx* ctx, const kc_csr* A, const void* x, void* y, int vec_dtype) {
  ctx->dots_pending = 0;                        // a new matvec: earlier SpMV sums are stale
  int grid = grid_for(ctx, A->m, 256, 8);
  if ((A->val_dtype == KC_F64) != (vec_dtype == KC_F64))
    return fail(ctx, KC_ERR_INVALID_ARG, "spmv: matrix value type %d does not match vector type %d",
                A->val_dtype, vec_dtype);
  timing_begin(ctx, KID_SPMV);
  if (is_stencil(A)) {
    const int nx = A->grid[0], ny = A->grid[1], nz = A->grid[2];
    if (vec_dtype == KC_F64) {
      Stencil7<double> c;
      for (int i = 0; i < 7; i++) c.c[i] = A->stencil[i];
      KC_CUDA(ctx, launch_pdl(ctx->stream, k_stencil7<double>, grid, 256, 0, (const double*)x,
                              (double*)y, nx, ny, nz, c, (const Scalars*)ctx->scal,
                              (double*)nullptr));
    } else {
      Stencil7<float> c;
      for (int i = 0; i < 7; i++) c.c[i] = (float)A->stencil[i];
      KC_CUDA(ctx, launch_pdl(ctx->stream, k_stencil7<float>, grid, 256, 0, (const float*)x,
                              (float*)y, nx, ny, nz, c, (const Scalars*)ctx->scal,
                              (double*)nullptr));
    }
  } else if (A->val_dtype == KC_F64 && vec_dtype == KC_F64)
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_spmv<double, double>, grid, 256, 0, A->row_ptr,
                            A->col_idx, (const double*)A->val, (const double*)x, (double*)y,
                            A->m, (const Scalars*)ctx->scal, (double*)nullptr));
  else if (A->val_dtype == KC_F32 && vec_dtype == KC_F32)
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_spmv<float, float>, grid, 256, 0, A->row_ptr,
                            A->col_idx, (const float*)A->val, (const float*)x, (float*)y, A->m,
                            (const Scalars*)ctx->scal, (double*)nullptr));
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_spmv_dots(kc_ctx* ctx, const kc_csr* A, const void* x, void* y, int vec_dtype) {
  ctx->dots_pending = 0;
  if (vec_dtype != KC_F64 || A->val_dtype != KC_F64) return launch_spmv(ctx, A, x, y, vec_dtype);
  int grid = grid_for(ctx, A->m, 256, 8);               // <= 8 * num_sms (the dots buffer)
  timing_begin(ctx, KID_SPMV);
  if (is_stencil(A)) {
    Stencil7<double> c;
    for (int i = 0; i < 7; i++) c.c[i] = A->stencil[i];
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_stencil7<double, true>, grid, 256, 0,
                            (const double*)x, (double*)y, A->grid[0], A->grid[1], A->grid[2],
                            c, (const Scalars*)ctx->scal, ctx->dots));
  } else {
    static std::atomic<int> occ{0};
    grid = one_wave(ctx, k_spmv<double, double, true>, 256, grid, occ);
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_spmv<double, double, true>, grid, 256, 0,
                            A->row_ptr, A->col_idx, (const double*)A->val, (const double*)x,
                            (double*)y, A->m, (const Scalars*)ctx->scal, ctx->dots));
  }
  KC_LAUNCHED(ctx);
  ctx->dots_pending = grid;
  ctx->dots_x = x;
  ctx->dots_y = y;
  return KC_OK;
}

template <typename TQ, typename TV, int NRHS>
static kc_status reduce_dispatch(kc_ctx* ctx, int grid, const TQ* Q, int64_t ldq, int k,
                                 const TV* x, const TV* y, int64_t m, int epi,
                                 const StepArgs& sa) {
  const int ntask = k + 1;
  // Few tasks: one warp per task and as many CTAs per SM as fit, so that every SM streams
  // many row ranges at once (16 warps sharing one row range left most of them idle with one
  // memory round trip per iteration: 159 us for w and v of an FP32 basis at m = 16 M, 63 us
  // this way); measured faster up to 10 tasks, while from 13 to 16 the 2 x 16-warp layout
  // is ahead.  17-32 and 33-48 tasks: two or three slots per warp in ceil(ntask / slots)
  // warps, so that no warp carries more columns than the others (17 tasks on 16 warps ran
  // at half pace).  FP32 / BF16 vectors with at most RED_RSUB_TASKS tasks: CTAs of
  // RED_WARPS / ntask row sub-blocks of ntask warps, so that each SM holds as many warps
  // with loads in flight while the partials (and the last CTA's sums over them) stay few.
  int nw = RED_WARPS, rsub = 1;
  // FP32 / BF16 vectors from RED_RSUB_TASKS + 1 to 48 tasks: three slots per warp in CTAs
  // of ceil(ntask / 3) warps, as many per SM as fit.  Every layout holds about 32 warps per
  // SM (64 registers), so three slots keep the most basis loads in flight (one slot per
  // warp left the FP32 reduction at 0.62-0.72 of HBM at k = 10-25, m = 16 M).
  const bool split = sizeof(TV) == 4 && ntask <= RED_RSUB_TASKS;
  const bool three = sizeof(TV) == 4 && !split && ntask <= 3 * RED_WARPS;
  const int slots = split ? 1 : (three ? 3 : (ntask <= 10 ? 1 : (ntask <= RED_WARPS ? 0 : (ntask <= 2 * RED_WARPS ? 2 : (ntask <= 3 * RED_WARPS ? 3 : 0)))));
  if (slots) {
    nw = (ntask + slots - 1) / slots;
    if (split) rsub = RED_WARPS / ntask;
    const int nwc = nw * rsub;                    // warps per CTA
    static int occ[4][RED_WARPS + 1];             // resident CTAs per SM, by slots and warps
    int& o = occ[slots][nwc];
    if (o == 0) {
      int n = 0;
      const cudaError_t e =
          slots == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_reduce<TQ, TV, 1, NRHS>, 32 * nwc, 0)
          : slots == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_reduce<TQ, TV, 2, NRHS>, 32 * nwc, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_reduce<TQ, TV, 3, NRHS>, 32 * nwc, 0);
      if (e != cudaSuccess || n < 1) n = 1;
      o = n;
    }
    const int cps = o < PARTIAL_CTAS_PER_SM ? o : PARTIAL_CTAS_PER_SM;
    const int64_t ngroups = m / Grp<TV>::R;
    int64_t b = (ngroups + 32 * 4 * rsub - 1) / (32 * 4 * rsub);   // >= 4 groups per lane
    const int64_t cap = (int64_t)ctx->num_sms * cps;
    if (b > cap) b = cap;
    grid = (int)(b < 1 ? 1 : b);
  }
  cudaError_t le = cudaSuccess;
  auto args = [&](auto kern) {
    le = launch_pdl(ctx->stream, kern, grid, 32 * nw * rsub, 0, Q, ldq, k, x, y, m,
                    ctx->partials, ctx->counters, ctx->scal, epi, sa, rsub,
                    group_counters(ctx));
  };
  if (three) args(k_reduce<TQ, TV, 3, NRHS>);
  else if (ntask <= RED_WARPS) args(k_reduce<TQ, TV, 1, NRHS>);
  else if (ntask <= 2 * RED_WARPS) args(k_reduce<TQ, TV, 2, NRHS>);
  else if (ntask <= 3 * RED_WARPS) args(k_reduce<TQ, TV, 3, NRHS>);
  else if (ntask <= 4 * RED_WARPS) args(k_reduce<TQ, TV, 4, NRHS>);
  else args(k_reduce<TQ, TV, 8, NRHS>);
  KC_CUDA(ctx, le);
  return KC_OK;
}

// Task layout of the offload reduction for ntask equal tasks (the DCGS2 step: k + 2; the
// finish's one-vector reductions: k + 1, which share the entry of ntask - 2):
// Task layout: nsplit subsets of nt tasks (ceil(ntask / 48) <= nsplit <= ceil(ntask /
// 32)), CTAs of nw <= 16 warps with tpw slots, chosen once per k and size class to
// maximise resident warps x used slots.  Three slots (one row group per iteration,
// which fits 64 registers) keep 33-48 tasks in one subset, so that w and v are read
// once per row block.  Below 33 tasks their small CTAs pay off only on long vectors:
// at m = 16 M, 8 warps x 3 slots beat 12 x 2 for 21-24 tasks (753-822 us against
// 833-872), while at m = 10^6 the larger CTAs won (83-86 us against 90-97).  (Three
// subsets and more, or more subsets than needed, measured slower.)  Sweeps of every
// layout at each k (m = 16 M and 10^6) found three ranges where the score misjudges,
// taken from the measurements instead: 33-36 tasks run fastest as two subsets of two
// slots (5% at both sizes), and up to 16 tasks as one subset of two slots on long
// vectors (up to 14%) but of one slot on short ones.
// With `split_rows` (the two-vector kernel only), up to F64X_RSUB_TASKS tasks on long
// vectors run as one slot per warp in CTAs of rsub row sub-blocks (about eight warps).
static void f64x_layout(kc_ctx* ctx, int ntask, int big, bool split_rows, int& nsplit,
                        int& nt, int& tpw, int& nw, int& occ, int& rsub) {
  {
      int* pick = ctx->red_pick[split_rows ? 1 : 0][big][ntask - 1];
      if (pick[0] == 0) {
        auto occ_of = [&](int tp, int nww) {
          int& o = ctx->red_occ[tp - 1][nww];
          if (o == 0) {
            int n = 0;
            cudaError_t e =
                tp == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_reduce_f64x<1, 2>, 32 * nww, 0)
                : tp == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_reduce_f64x<2, 2>, 32 * nww, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_reduce_f64x<3, 1>, 32 * nww, 0);
            if (e != cudaSuccess || n < 1) n = 1;
            o = n > PARTIAL_CTAS_PER_SM ? PARTIAL_CTAS_PER_SM : n;
          }
          return o;
        };
        auto take = [&](int ns, int tp) {
          const int ntt = (ntask + ns - 1) / ns;
          const int nww = (ntt + tp - 1) / tp;
          pick[0] = ns; pick[1] = ntt; pick[2] = tp; pick[3] = nww; pick[4] = occ_of(tp, nww);
          pick[5] = 1;
        };
        if (split_rows && big && ntask <= F64X_RSUB_TASKS) {
          const int rs = F64X_RSUB_WARPS / ntask > 1 ? F64X_RSUB_WARPS / ntask : 1;
          pick[0] = 1; pick[1] = ntask; pick[2] = 1; pick[3] = ntask * rs;
          pick[4] = occ_of(1, ntask * rs); pick[5] = rs;
        } else if (ntask >= 33 && ntask <= 36) {
          take(2, 2);
        } else if (ntask <= 16) {
          take(1, big && ntask >= 5 ? 2 : 1);
        } else {
          double best = -1.0;
          const int s0 = (ntask + 31) / 32;
          const int tpmax = (ntask > 32 || (big && ntask > 20)) ? 3 : 2;
          for (int ns = (ntask + 47) / 48; ns <= s0; ns++)
            for (int tp = 1; tp <= tpmax; tp++) {
              const int ntt = (ntask + ns - 1) / ns;
              const int nww = (ntt + tp - 1) / tp;
              if (nww > 16) continue;
              const int o = occ_of(tp, nww);
              const int warps = o * nww < 32 ? o * nww : 32;
              const double score = warps * (double)ntask / ((double)ns * nww * tp) /
                                   (1.0 + 0.03 * (ns - s0));
              if (score > best) {
                best = score;
                take(ns, tp);
              }
            }
        }
      }
      nsplit = pick[0]; nt = pick[1]; tpw = pick[2]; nw = pick[3]; occ = pick[4];
      rsub = pick[5];
    }
}

static kc_status launch_spmv_reduce_small(kc_ctx* ctx, const kc_csr* A, const double* Q,
                                          int64_t ldq, int k, const double* w, double* v,
                                          const StepArgs& sa) {
  ctx->dots_pending = 0;
  // one wave, the same grid for both operator forms (so that a stencil run and the run on
  // its CSR matrix sum in the same order and agree bit for bit); <= 8 CTAs per SM, the
  // partials rows
  static std::atomic<int> occ[2][FUSE_KMAX + 1];
  Stencil7<double> c = {};
  if (is_stencil(A))
    for (int i = 0; i < 7; i++) c.c[i] = A->stencil[i];
  cudaError_t le = cudaSuccess;
  auto go = [&](auto ks, auto kcsr, std::atomic<int>& os, std::atomic<int>& oc) {
    int grid = grid_for(ctx, A->m, 256, 8);
    grid = one_wave(ctx, ks, 256, grid, os);
    grid = one_wave(ctx, kcsr, 256, grid, oc);
    if (is_stencil(A))
      le = launch_pdl(ctx->stream, ks, grid, 256, 0, (const int32_t*)nullptr,
                      (const int32_t*)nullptr, (const double*)nullptr, A->grid[0], A->grid[1],
                      A->grid[2], c, Q, ldq, w, v, A->m, ctx->partials, ctx->counters,
                      ctx->scal, sa);
    else
      le = launch_pdl(ctx->stream, kcsr, grid, 256, 0, A->row_ptr, A->col_idx,
                      (const double*)A->val, 0, 0, 0, c, Q, ldq, w, v, A->m, ctx->partials,
                      ctx->counters, ctx->scal, sa);
  };
  timing_begin(ctx, KID_SPMV_REDUCE);
  switch (k) {
    case 0: go(k_spmv_reduce_small<true, 0>, k_spmv_reduce_small<false, 0>, occ[0][0], occ[1][0]); break;
    case 1: go(k_spmv_reduce_small<true, 1>, k_spmv_reduce_small<false, 1>, occ[0][1], occ[1][1]); break;
    case 2: go(k_spmv_reduce_small<true, 2>, k_spmv_reduce_small<false, 2>, occ[0][2], occ[1][2]); break;
    case 3: go(k_spmv_reduce_small<true, 3>, k_spmv_reduce_small<false, 3>, occ[0][3], occ[1][3]); break;
    default: go(k_spmv_reduce_small<true, 4>, k_spmv_reduce_small<false, 4>, occ[0][4], occ[1][4]); break;
  }
  KC_CUDA(ctx, le);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_matvec_reduce(kc_ctx* ctx, const kc_csr* A, const void* Q, int64_t ldq,
                               int q_dtype, int k, const void* w, void* v, int64_t m, int vec,
                               const StepArgs& sa) {
  if (vec == KC_F64 && q_dtype == KC_F64 && A->val_dtype == KC_F64 && ctx->fp64_mode == 1 &&
      k <= FUSE_KMAX && (ctx->staged & 8) && !(ctx->staged & 2))
    return launch_spmv_reduce_small(ctx, A, (const double*)Q, ldq, k, (const double*)w,
                                    (double*)v, sa);
  KC_TRY((vec == KC_F64 ? launch_spmv_dots : launch_spmv)(ctx, A, w, v, vec));
  return launch_reduce(ctx, Q, ldq, q_dtype, k, w, v, m, vec, EPI_DCGS2, sa);
}

kc_status launch_reduce(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k,
                        const void* x, const void* y, int64_t m, int vec_dtype, int epilogue,
                        const StepArgs& sa) {
  if (k + 1 > NMAX) return fail(ctx, KC_ERR_INVALID_ARG, "reduce: k = %d too large", k);
  const int R = vec_dtype == KC_F64 ? 2 : 4;
  const int grid = reduce_grid_for(ctx, m / R);
  const bool two = y != nullptr;
  const bool ok = (q_dtype == KC_F64 && vec_dtype == KC_F64) ||
                  (q_dtype != KC_F64 && vec_dtype == KC_F32);
  if (!ok)
    return fail(ctx, KC_ERR_INVALID_ARG, "reduce: unsupported basis/vector types %d/%d", q_dtype, vec_dtype);
  // beta and s from the step's SpMV (launch_spmv_dots), taken only by the offload kernel
  const int ndots = (ctx->dots_pending > 0 && ctx->dots_x == x && ctx->dots_y == y &&
                     epilogue == EPI_DCGS2) ? ctx->dots_pending : 0;
  ctx->dots_pending = 0;
  timing_begin(ctx, KID_REDUCE);
  if (q_dtype == KC_F64 && vec_dtype == KC_F64 && two && epilogue == EPI_DCGS2 &&
      ctx->fp64_mode == 2 && reduce_tcx_supported(k, m, Q, ldq, x, y)) {
    kc_status st = launch_reduce_tcx(ctx, (const double*)Q, ldq, k, (const double*)x,
                                     (const double*)y, m, sa);
    if (st != KC_OK) return st;
  } else if (q_dtype == KC_F64 && vec_dtype == KC_F64 && two && epilogue == EPI_DCGS2 &&
      (ctx->staged & 2) && reduce_tma_supported(k, m)) {
    kc_status st = launch_reduce_tma(ctx, (const double*)Q, ldq, k, (const double*)x,
                                     (const double*)y, m, ctx->fp64_mode >= 1, sa);
    if (st != KC_OK) return st;
  } else if (q_dtype == KC_F64 && vec_dtype == KC_F64 && two &&
             (epilogue == EPI_DCGS2 || epilogue == EPI_PARTIAL) && ctx->fp64_mode >= 1) {
    // with beta and s from the SpMV the step's tasks are its k columns only
    const int ntask = ndots ? k : k + 2;
    int nsplit, nt, tpw, nw, occ, rsub;
    const bool big = m >= ((int64_t)1 << 22);
    // (one task on short vectors: a two-warp CTA as for two tasks, one warp idle)
    f64x_layout(ctx, ntask < 1 ? 1 : (ntask < 2 && !big ? 2 : ntask), big, true, nsplit, nt,
                tpw, nw, occ, rsub);
    int64_t gcap = (m / 2 + 32 * 4 - 1) / (32 * 4);            // row blocks: >= 4 groups/lane
    int64_t nr = ((int64_t)ctx->num_sms * occ + nsplit - 1) / nsplit;
    if (nr > gcap) nr = gcap < 1 ? 1 : gcap;
    if (ntask == 0) {                        // k = 0: the epilogue alone, on the SpMV's sums
      nr = 1;                                // (eight warps to share their loads)
      nsplit = 1;
      nt = 0;
      nw = 8;
      tpw = 1;
      rsub = 1;
    }
    const int g = (int)(nr * nsplit);
    cudaError_t le = cudaSuccess;
    auto go = [&](auto kern) {
      le = launch_pdl(ctx->stream, kern, g, 32 * nw, 0, (const double*)Q, ldq, k,
                      (const double*)x, (const double*)y, m, ctx->partials, ctx->counters,
                      ctx->scal, sa, nsplit, nt, epilogue,
                      (const double*)(ndots ? ctx->dots : nullptr), ndots, rsub,
                      group_counters(ctx));
    };
    if (tpw == 1) go(k_reduce_f64x<1, 2>);
    else if (tpw == 2) go(k_reduce_f64x<2, 2>);
    else go(k_reduce_f64x<3, 1>);
    KC_CUDA(ctx, le);
  } else if (q_dtype == KC_F64 && vec_dtype == KC_F64 && !two && k >= 1 &&
             (epilogue == EPI_STORE_C || epilogue == EPI_STORE_C1 || epilogue == EPI_STORE_C2 ||
              epilogue == EPI_PARTIAL) &&
             ctx->fp64_mode >= 1) {
    // one vector (the CGS2 finish): the offload layout for k + 1 FP64 tasks
    int nsplit, nt, tpw, nw, occ, rsub;
    f64x_layout(ctx, k + 1, m >= ((int64_t)1 << 22), false, nsplit, nt, tpw, nw, occ, rsub);
    int64_t gcap = (m / 2 + 32 * 4 - 1) / (32 * 4);
    int64_t nr = ((int64_t)ctx->num_sms * occ + nsplit - 1) / nsplit;
    if (nr > gcap) nr = gcap < 1 ? 1 : gcap;
    const int g = (int)(nr * nsplit);
    auto go = [&](auto kern) {
      kern<<<g, 32 * nw, 0, ctx->stream>>>((const double*)Q, ldq, k, (const double*)x, m,
                                           ctx->partials, ctx->counters, ctx->scal, sa, nsplit,
                                           nt, epilogue);
    };
    // the finish's first projection in float-float (the second one corrects it)
    const bool off = epilogue == EPI_STORE_C1 && !(ctx->staged & 4);
    if (off) {
      if (tpw == 1) go(k_reduce1_f64<1, 2, true>);
      else if (tpw == 2) go(k_reduce1_f64<2, 2, true>);
      else go(k_reduce1_f64<3, 2, true>);
    } else {
      if (tpw == 1) go(k_reduce1_f64<1, 2, false>);
      else if (tpw == 2) go(k_reduce1_f64<2, 2, false>);
      else go(k_reduce1_f64<3, 2, false>);
    }
  } else if (q_dtype == KC_F64 && vec_dtype == KC_F64) {
    if (two) KC_TRY((reduce_dispatch<double, double, 2>(ctx, grid, (const double*)Q, ldq, k, (const double*)x, (const double*)y, m, epilogue, sa)));
    else KC_TRY((reduce_dispatch<double, double, 1>(ctx, grid, (const double*)Q, ldq, k, (const double*)x, nullptr, m, epilogue, sa)));
  } else if (q_dtype == KC_F32 && vec_dtype == KC_F32) {
    if (two) KC_TRY((reduce_dispatch<float, float, 2>(ctx, grid, (const float*)Q, ldq, k, (const float*)x, (const float*)y, m, epilogue, sa)));
    else KC_TRY((reduce_dispatch<float, float, 1>(ctx, grid, (const float*)Q, ldq, k, (const float*)x, nullptr, m, epilogue, sa)));
  } else {
    if (two) KC_TRY((reduce_dispatch<__nv_bfloat16, float, 2>(ctx, grid, (const __nv_bfloat16*)Q, ldq, k, (const float*)x, (const float*)y, m, epilogue, sa)));
    else KC_TRY((reduce_dispatch<__nv_bfloat16, float, 1>(ctx, grid, (const __nv_bfloat16*)Q, ldq, k, (const float*)x, nullptr, m, epilogue, sa)));
  }
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_dcgs2_update(kc_ctx* ctx, void* Q, int64_t ldq, int q_dtype, int k, void* w,
                              const void* v, int64_t m, int vec_dtype) {
  if (q_dtype == KC_F64 && (ctx->staged & 1))
    return launch_update_staged(ctx, (double*)Q, ldq, k, (double*)w, (const double*)v, m);
  const int R = vec_dtype == KC_F64 ? 2 : 4;
  const int grid = grid_for(ctx, m / R, UPD_THREADS, 8);
  timing_begin(ctx, KID_UPDATE);
  // (two waves of 4 CTAs per SM: one wave of CTAs with twice the rows measured 3.6% slower)
  if (q_dtype == KC_F64 && ctx->fp64_mode >= 1)
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_dcgs2_update_f64x, grid, UPD_THREADS, 0, (double*)Q,
                            ldq, k, (double*)w, (const double*)v, m,
                            (const Scalars*)ctx->scal, !(ctx->staged & 4)));
  else if (q_dtype == KC_F64)
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_dcgs2_update<double, double>, grid, UPD_THREADS, 0,
                            (double*)Q, ldq, k, (double*)w, (const double*)v, m,
                            (const Scalars*)ctx->scal));
  else if (q_dtype == KC_F32)
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_dcgs2_update<float, float>, grid, UPD_THREADS, 0,
                            (float*)Q, ldq, k, (float*)w, (const float*)v, m,
                            (const Scalars*)ctx->scal));
  else
    KC_CUDA(ctx, launch_pdl(ctx->stream, k_dcgs2_update<__nv_bfloat16, float>, grid,
                            UPD_THREADS, 0, (__nv_bfloat16*)Q, ldq, k, (float*)w,
                            (const float*)v, m, (const Scalars*)ctx->scal));
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_proj_reduce(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k, void* w,
                             int64_t m, int vec_dtype, const StepArgs& sa) {
  const bool fused = q_dtype == KC_F64 && vec_dtype == KC_F64 && ctx->fp64_mode >= 1 &&
                     !(ctx->staged & 4) && k >= 1 && k <= PR_MAXK && (ldq & 1) == 0 &&
                     ((uintptr_t)Q & 15) == 0 && m >= PR_TR;
  if (!fused) {                                 // the two passes apart
    KC_TRY(launch_gemv_sub(ctx, Q, ldq, q_dtype, k, w, m, vec_dtype, 0));
    return launch_reduce(ctx, Q, ldq, q_dtype, k, w, nullptr, m, vec_dtype, EPI_STORE_C2, sa);
  }
  static std::atomic<unsigned long long> attr{0};
  const int smem = 2 * k * PR_LD * (int)sizeof(double);
  KC_TRY(smem_attr_once(ctx, attr, k_proj_reduce, 2 * PR_MAXK * PR_LD * (int)sizeof(double),
                        "proj_reduce"));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_proj_reduce, PR_THREADS, smem) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  if (per_sm > PARTIAL_CTAS_PER_SM) per_sm = PARTIAL_CTAS_PER_SM;
  int64_t grid = (int64_t)ctx->num_sms * per_sm, ntiles = m / PR_TR;
  if (grid > ntiles) grid = ntiles;
  timing_begin(ctx, KID_FIN_REDUCE);
  k_proj_reduce<<<(int)grid, PR_THREADS, smem, ctx->stream>>>((const double*)Q, ldq, k,
      (double*)w, m, ctx->partials, ctx->counters, ctx->scal, sa);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_gemv_sub(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k, void* x,
                          int64_t m, int vec_dtype, int which) {
  const int R = vec_dtype == KC_F64 ? 2 : 4;
  int grid = grid_for(ctx, m / R, UPD_THREADS, 8);
  timing_begin(ctx, KID_GEMV_SUB);
  static std::atomic<int> occ{0};
  if (q_dtype == KC_F64) grid = one_wave(ctx, k_gemv_sub<double, double>, UPD_THREADS, grid, occ);
  if (q_dtype == KC_F64)
    k_gemv_sub<double, double><<<grid, UPD_THREADS, 0, ctx->stream>>>((const double*)Q, ldq, k, (double*)x, m, ctx->scal, which, ctx->fp64_mode >= 1 && which != 2 && !(ctx->staged & 4));
  else if (q_dtype == KC_F32)
    k_gemv_sub<float, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const float*)Q, ldq, k, (float*)x, m, ctx->scal, which, 0);
  else
    k_gemv_sub<__nv_bfloat16, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const __nv_bfloat16*)Q, ldq, k, (float*)x, m, ctx->scal, which, 0);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_fallback_norm(kc_ctx* ctx, const void* Q, int64_t ldq, int q_dtype, int k,
                               const void* w, int64_t m, const StepArgs& sa) {
  const int grid = grid_for(ctx, m / 4, UPD_THREADS, 2);
  timing_begin(ctx, KID_NORM);
  if (q_dtype == KC_F32)
    k_fallback_norm<float, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const float*)Q, ldq, k, (const float*)w, m, ctx->partials, ctx->counters + 2, ctx->scal, sa);
  else if (q_dtype == KC_BF16)
    k_fallback_norm<__nv_bfloat16, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const __nv_bfloat16*)Q, ldq, k, (const float*)w, m, ctx->partials, ctx->counters + 2, ctx->scal, sa);
  else
    k_fallback_norm<double, double><<<grid, UPD_THREADS, 0, ctx->stream>>>((const double*)Q, ldq, k, (const double*)w, m, ctx->partials, ctx->counters + 2, ctx->scal, sa);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_norm(kc_ctx* ctx, const void* x, const void* y, int64_t m, int vec_dtype,
                      int nepi, const StepArgs& sa) {
  const int R = vec_dtype == KC_F64 ? 2 : 4;
  const int grid = grid_for(ctx, m / R, RED_THREADS * 4, 2);
  timing_begin(ctx, KID_NORM);
  if (vec_dtype == KC_F64) {
    if (y) k_norm<double, 2><<<grid, RED_THREADS, 0, ctx->stream>>>((const double*)x, (const double*)y, m, ctx->partials, ctx->counters + 1, ctx->scal, nepi, sa);
    else k_norm<double, 1><<<grid, RED_THREADS, 0, ctx->stream>>>((const double*)x, nullptr, m, ctx->partials, ctx->counters + 1, ctx->scal, nepi, sa);
  } else {
    if (y) k_norm<float, 2><<<grid, RED_THREADS, 0, ctx->stream>>>((const float*)x, (const float*)y, m, ctx->partials, ctx->counters + 1, ctx->scal, nepi, sa);
    else k_norm<float, 1><<<grid, RED_THREADS, 0, ctx->stream>>>((const float*)x, nullptr, m, ctx->partials, ctx->counters + 1, ctx->scal, nepi, sa);
  }
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_scale_to(kc_ctx* ctx, const void* x, void* qcol, int q_dtype, int64_t m,
                          int vec_dtype) {
  const int grid = grid_for(ctx, m, UPD_THREADS, 8);
  timing_begin(ctx, KID_SCALE);
  if (q_dtype == KC_F64 && vec_dtype == KC_F64)
    k_scale_to<double, double><<<grid, UPD_THREADS, 0, ctx->stream>>>((const double*)x, (double*)qcol, m, ctx->scal);
  else if (q_dtype == KC_F32)
    k_scale_to<float, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const float*)x, (float*)qcol, m, ctx->scal);
  else
    k_scale_to<__nv_bfloat16, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const float*)x, (__nv_bfloat16*)qcol, m, ctx->scal);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_axpy_h(kc_ctx* ctx, const void* q, int q_dtype, void* v, int64_t m,
                        int vec_dtype) {
  const int grid = grid_for(ctx, m, UPD_THREADS, 8);
  timing_begin(ctx, KID_AXPY);
  if (q_dtype == KC_F64)
    k_axpy_h<double, double><<<grid, UPD_THREADS, 0, ctx->stream>>>((const double*)q, (double*)v, m, ctx->scal);
  else if (q_dtype == KC_F32)
    k_axpy_h<float, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const float*)q, (float*)v, m, ctx->scal);
  else
    k_axpy_h<__nv_bfloat16, float><<<grid, UPD_THREADS, 0, ctx->stream>>>((const __nv_bfloat16*)q, (float*)v, m, ctx->scal);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

}  // namespace kc

// ----------------------------------------------------------------------------------------
// Row-partitioned DCGS2 (Section 5's distributed layout): each rank owns a block of rows of
// Q, w, v and A; its reduction stores its partial sums (EPI_PARTIAL), the caller sums them
// over the ranks (the one global reduction of the step), and the kernels below continue
// from those sums.  The scalar step runs redundantly on every rank on identical sums, so
// H and K stay replicated.
// ----------------------------------------------------------------------------------------
namespace kc {

__global__ void __launch_bounds__(RED_THREADS)
k_scalar_from_totals(const double* __restrict__ totals, int k, Scalars* __restrict__ sc,
                     StepArgs sa) {
  __shared__ double tot[PSTRIDE];
  if (sc->stop) return;
  for (int i = threadIdx.x; i < 2 * (k + 1); i += blockDim.x) tot[i] = __ldcg(totals + i);
  __syncthreads();
  epilogue_from_tot(tot, k, 2, sc, EPI_DCGS2, sa);
}

// totals = [c_0 .. c_{k-1}, x^T x]: the coefficients of a finish projection and the
// squared norm of the vector they came from (which 0: C, 1: C2)
__global__ void k_store_totals(const double* __restrict__ totals, int k, int which,
                               Scalars* __restrict__ sc) {
  double* dst = which == 0 ? sc->C : sc->C2;
  for (int i = threadIdx.x; i < k; i += blockDim.x) dst[i] = __ldcg(totals + i);
  if (threadIdx.x == 0) {
    sc->norm_sq = __ldcg(totals + k);
    if (!isfinite(sc->norm_sq)) set_status(sc, KC_ERR_NONFINITE);
  }
}

// totals[0] = ||u||^2 over all ranks: the finish's H column, alpha and 1/alpha
__global__ void k_finish_from_norm(const double* __restrict__ totals, Scalars* __restrict__ sc,
                                   StepArgs sa) {
  if (threadIdx.x == 0) norm_epilogue(__ldcg(totals), 0.0, sc, NEPI_FINISH, sa);
}

kc_status launch_scalar_from_totals(kc_ctx* ctx, const double* totals, int k,
                                    const StepArgs& sa) {
  if (k + 1 > NMAX) return fail(ctx, KC_ERR_INVALID_ARG, "scalar step: k = %d too large", k);
  timing_begin(ctx, KID_SMALL);
  k_scalar_from_totals<<<1, RED_THREADS, 0, ctx->stream>>>(totals, k, ctx->scal, sa);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_store_totals(kc_ctx* ctx, const double* totals, int k, int which) {
  timing_begin(ctx, KID_SMALL);
  k_store_totals<<<1, 128, 0, ctx->stream>>>(totals, k, which, ctx->scal);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

kc_status launch_finish_from_norm(kc_ctx* ctx, const double* totals, const StepArgs& sa) {
  timing_begin(ctx, KID_SMALL);
  k_finish_from_norm<<<1, 32, 0, ctx->stream>>>(totals, ctx->scal, sa);
  KC_LAUNCHED(ctx);
  return KC_OK;
}

}  // namespace kc

// ----------------------------------------------------------------------------------------
// One DCGS2 step without any allocation, for callers that cannot call cudaMalloc: code
// running inside a CUDA stream-ordered allocator callback, plugins whose host process owns
// the device memory budget, and environments where a context (kc_create) is not
// available.  The fused reduction's scratch (per-CTA partial sums, the last-CTA ticket
// and the step scalars) lives in the file-scope array below instead of context workspace.
// ----------------------------------------------------------------------------------------
namespace kc {

constexpr int NOALLOC_MAX_GRID = 152;   // reduction CTAs, and rows of partials below
struct NoAllocScratch {
  Scalars sc;
  unsigned int counter[4];
  double partials[NOALLOC_MAX_GRID * PSTRIDE];
};

// About 325 KB; every GPU that loads libkrylov holds it until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device addresses of g_noalloc_scratch, looked up once per device (host code may not
// use the symbol itself: on the host it only names a stand-in, not device memory).
constexpr int NOALLOC_MAX_DEVICES = 64;
static NoAllocScratch* g_noalloc_ptr[NOALLOC_MAX_DEVICES];

static kc_status noalloc_setup(NoAllocScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return KC_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KC_ERR_CUDA;
    g_noalloc_ptr[dev] = (NoAllocScratch*)p;
  }
  *out = g_noalloc_ptr[dev];
  return KC_OK;
}

}  // namespace kc

extern "C" kc_status dcgs2_arnoldi_step_noalloc(const kc_csr* A, kc_arnoldi* st,
                                                void* cuda_stream) {
  using namespace kc;
  if (validate_csr_entries(nullptr, A) != KC_OK || validate_state(nullptr, A, st) != KC_OK)
    return KC_ERR_INVALID_ARG;
  if (st->q_dtype != KC_F64 || A->val_dtype != KC_F64) return KC_ERR_INVALID_ARG;
  const int k = st->k;
  if (k + 2 > st->ncap || st->finished) return KC_ERR_INVALID_ARG;
  if (k + 1 > NMAX) return KC_ERR_INVALID_ARG;          // partials rows hold 2*NMAX+4 values
  NoAllocScratch* scr = nullptr;
  kc_status s = noalloc_setup(&scr);
  if (s != KC_OK) return s;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int64_t m = A->m;
  // what must start at zero: the ticket counters, the stop flag and the status word
  if (cudaMemsetAsync(scr->counter, 0, sizeof(scr->counter), stream) != cudaSuccess ||
      cudaMemsetAsync(&scr->sc.stop, 0, sizeof(int), stream) != cudaSuccess ||
      cudaMemsetAsync(&scr->sc.status, 0, sizeof(int), stream) != cudaSuccess)
    return KC_ERR_CUDA;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return KC_ERR_CUDA;
  int64_t gs = (m + 255) / 256;
  const int gspmv = (int)(gs < 1 ? 1 : (gs > 8 * (int64_t)sms ? 8 * (int64_t)sms : gs));
  k_spmv<double, double><<<gspmv, 256, 0, stream>>>(A->row_ptr, A->col_idx,
      (const double*)A->val, (const double*)st->w, (double*)st->v, m, &scr->sc);
  StepArgs sa = {};
  sa.H = st->H;
  sa.ldh = st->ldh;
  sa.K = st->K;
  sa.ldk = st->ncap;
  sa.k = k;
  sa.pyth_tol = 0.0;
  int64_t gr = (m / 2 + 32 * 4 - 1) / (32 * 4);
  const int maxg = sms < NOALLOC_MAX_GRID ? sms : NOALLOC_MAX_GRID;
  const int grid = (int)(gr < 1 ? 1 : (gr > maxg ? maxg : gr));
  const double* Q = (const double*)st->Q;
  const double* w = (const double*)st->w;
  const double* v = (const double*)st->v;
  const int ntask = k + 1;
  auto go = [&](auto kern) {
    kern<<<grid, RED_THREADS, 0, stream>>>(Q, st->ldq, k, w, v, m, scr->partials, scr->counter,
                                           &scr->sc, (int)EPI_DCGS2, sa, 1,
                                           (unsigned int*)nullptr);
  };
  if (ntask <= RED_WARPS) go(k_reduce<double, double, 1, 2>);
  else if (ntask <= 2 * RED_WARPS) go(k_reduce<double, double, 2, 2>);
  else if (ntask <= 4 * RED_WARPS) go(k_reduce<double, double, 4, 2>);
  else go(k_reduce<double, double, 8, 2>);
  int64_t gu = (m / 2 + UPD_THREADS - 1) / UPD_THREADS;
  const int gupd = (int)(gu < 1 ? 1 : (gu > 8 * (int64_t)sms ? 8 * (int64_t)sms : gu));
  k_dcgs2_update<double, double><<<gupd, UPD_THREADS, 0, stream>>>(
      (double*)st->Q, st->ldq, k, (double*)st->w, (const double*)st->v, m, &scr->sc);
  if (cudaGetLastError() != cudaSuccess) return KC_ERR_CUDA;
  st->k = k + 1;
  return KC_OK;
}

extern "C" kc_status dcgs2_noalloc_read_status(int* status, void* cuda_stream) {
  using namespace kc;
  if (!status) return KC_ERR_INVALID_ARG;
  NoAllocScratch* scr = nullptr;
  kc_status s = noalloc_setup(&scr);
  if (s != KC_OK) return s;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int v = KC_OK;
  if (cudaMemcpyAsync(&v, &scr->sc.status, sizeof(int), cudaMemcpyDeviceToHost, stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return KC_ERR_CUDA;
  *status = v;
  return KC_OK;
}
