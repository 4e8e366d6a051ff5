// Restarted FP64 DCGS2-GMRES(n) for small problems in ONE launch per solve.
//
// At m = 10^4 (the 2D convection-diffusion problem of the GMRES benchmark) a DCGS2 step of
// the multi-kernel path is three launches whose cost is latency, not bytes: the fused
// reduction alone takes 12-30 us of partial sums, last-CTA ticket and serial scalar work
// for 2.5 MB of basis.  Here one persistent kernel runs the whole solve; its CTAs own
// contiguous row blocks of Q, v, w and x and run every phase in place:
//   per Arnoldi step (Algorithm 4): v = A w on the CTA's rows; the partial sums of
//   [Q_k, w]^T [w, v]; one exchange; every CTA adds the partials of all CTAs in the same
//   rank order, so every CTA holds bitwise the same C, S, beta, s and takes the same
//   decisions; alpha by Pythagoras, T by Stephen's trick; the row-local update of q_k and
//   w; CTA 0 alone forms the lagged H and K columns and rotates the finalised column
//   (Givens, stop test); a barrier makes w (read across row blocks by the next matvec) and
//   CTA 0's stop flag visible;
//   per cycle: the CGS2 finish of the last column (two projections and a norm), the
//   triangular solve y = R^{-1} g in CTA 0 (column-parallel back substitution), x += Q y,
//   and the FP64 residual b - A x with its norm for the restart test.
// Two ways to exchange, one kernel body (a policy template):
//   cluster: one thread-block cluster of 16 CTAs (8 where 16 cannot be scheduled); the
//     partials and CTA 0's published state are read from the other CTAs' shared memory
//     (distributed shared memory) after a hardware cluster barrier;
//   grid: one CTA per SM on the whole GPU, launched cooperatively (all CTAs resident); the
//     partials go through global memory and the barrier is a counter and generation word
//     in global memory whose spin is bounded (about a second), after which the kernel
//     sets an error word, every CTA leaves the solve, and the call reports KC_ERR_TIMEOUT.
// A CTA keeps its rows of the basis, of v and of w in shared memory where they fit (w is
// also written to global memory for the other CTAs' matvecs) and CTA 0 keeps H, K, R
// there, so the step's dependent chains run at shared-memory latency; otherwise the same
// code addresses them in global memory.  The partial-sum buffers alternate between
// reductions, so one barrier per reduction is enough: a CTA writes a buffer again only
// after the next reduction's barrier, which every CTA reaches after it has read that
// buffer.  Vectors other CTAs write (w, x) are read through L2 (ld.global.cg), never from a
// stale L1 line; in the cluster form a last barrier keeps every CTA (and its shared memory)
// alive until all remote reads are done.
#include "kc_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace kc {

constexpr int GC_THREADS = 1024;       // one thread per row at config 1 (625 rows per CTA)
constexpr int GC_WARPS = GC_THREADS / 32;
constexpr int GC_PART = 2 * NMAX + 2;
constexpr int GC_DYN_SMEM_MAX = 200 * 1024;   // dynamic shared memory the kernel may use
constexpr long long GRID_WAIT_LIMIT = 2000000000LL;   // cycles (about 1 s) per barrier
// rows up to which the default takes the grid form: GMRES(30) to 1e-10 on 2D problems took
// 113.8 vs 176.7 ms (m = 65,536), 763 vs 945 ms (m = 262,144) against the multi-kernel
// path, and 9.24 vs 7.50 s at m = 1,048,576, where the basis streams from HBM
constexpr int64_t GMRES_GRID_MAX_ROWS = 393216;

// CTA 0's state that every CTA reads after a barrier
struct GcPub {
  int stop, ncols;
  double est;
  double y[NMAX];
};

// grid barrier: arrivals, generation, error word (zeroed before the launch)
struct GridBar {
  unsigned int count, gen;
  int err, pad;
};

struct GcArgs {
  // operator: CSR (stencil == 0) or the 7-point stencil
  const int32_t* rp;
  const int32_t* ci;
  const double* val;
  int nx, ny, nz, stencil;
  double c7[7];
  const double* b;
  double* x;
  double* Q;        // global basis (used when the rows do not fit in shared memory)
  int64_t ldq;
  double* w;
  double* v;
  double* H;        // (n+1) x n, ld n+1   (global copies, used when not in shared memory)
  double* K;        // (n+1) x n, ld n+1
  double* R;        // n x n, ld n
  int n;
  int maxit;
  int64_t m;
  int rc;           // rows per CTA, at most (the shared-memory row capacity)
  int smem_q;       // the CTA's rows of Q, v and w live in shared memory
  int smem_h;       // CTA 0 keeps H, K, R in shared memory
  double rtol;
  double* out;      // matvecs, cycles, est, rn, bnorm, result, last status
  // grid form only
  double* gpart;    // [2][grid][GC_PART] partial sums
  GcPub* pub;       // CTA 0's published state
  GridBar* bar;
  int bar_extra;    // arrivals expected beyond the CTAs (test hook: > 0 makes a wait run out)
  int skip0;        // CTA 0 owns no rows (grid form: its serial work overlaps the others')
};

__device__ __forceinline__ double gc_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (A y)_r with y read through L2 (its entries outside this CTA's rows are written by others)
__device__ __forceinline__ double gc_apply_row(const GcArgs& a, const double* y, int64_t r) {
  double s = 0.0;
  if (a.stencil) {
    const int64_t pl = (int64_t)a.nx * a.ny;
    const int64_t t = r / a.nx;
    const int ix = (int)(r - t * a.nx), iy = (int)(t % a.ny), iz = (int)(t / a.ny);
    if (iz > 0) s += a.c7[5] * __ldcg(y + r - pl);
    if (iy > 0) s += a.c7[3] * __ldcg(y + r - a.nx);
    if (ix > 0) s += a.c7[1] * __ldcg(y + r - 1);
    s += a.c7[0] * __ldcg(y + r);
    if (ix < a.nx - 1) s += a.c7[2] * __ldcg(y + r + 1);
    if (iy < a.ny - 1) s += a.c7[4] * __ldcg(y + r + a.nx);
    if (iz < a.nz - 1) s += a.c7[6] * __ldcg(y + r + pl);
    return s;
  }
  for (int j = a.rp[r]; j < a.rp[r + 1]; j++) s += a.val[j] * __ldcg(y + a.ci[j]);
  return s;
}

// this thread's partial of a scalar sum -> part[0] of the CTA (fixed order)
__device__ void gc_block_sum(double val, double* part, double* scratch) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  val = gc_warp_sum(val);
  if (lane == 0) scratch[warp] = val;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < GC_WARPS; i++) s += scratch[i];
    part[0] = s;
  }
}

__device__ __forceinline__ void gc_set_status(int* st, int v) {
  if (*st == KC_OK) *st = v;
}

// ---- exchange policies ---------------------------------------------------------------------

struct ClusterComm {
  cg::cluster_group cl;
  int rank, nb;
  GcPub* pub_w;          // where CTA 0 writes its state (its shared memory)
  const GcPub* pub_r;    // where every CTA reads it (CTA 0's shared memory, mapped)
  __device__ ClusterComm(const GcArgs&, GcPub* s_pub) : cl(cg::this_cluster()) {
    rank = (int)cl.block_rank();
    nb = (int)cl.num_blocks();
    pub_w = s_pub;
    pub_r = cl.map_shared_rank(s_pub, 0);
  }
  __device__ bool sync() {
    __threadfence();
    cl.sync();
    return true;
  }
  // every CTA: tot[i] = sum over ranks (in rank order) of their `mine`[i]
  __device__ bool sum(double* mine, int, double* tot, int nval) {
    sync();
    for (int i = threadIdx.x; i < nval; i += blockDim.x) {
      double s = 0.0;
#pragma unroll 16
      for (int c = 0; c < nb; c++) s += cl.map_shared_rank(mine, c)[i];
      tot[i] = s;
    }
    __syncthreads();
    return true;
  }
  __device__ int ld(const int* p) const { return *(volatile const int*)p; }
  __device__ double ld(const double* p) const { return *(volatile const double*)p; }
  __device__ void finish() { cl.sync(); }   // no CTA exits while its shared memory may be read
};

struct GridComm {
  int rank, nb;
  GridBar* bar;
  double* gpart;
  GcPub* pub_w;
  const GcPub* pub_r;
  unsigned int arrivals;
  __device__ GridComm(const GcArgs& a, GcPub*) {
    rank = (int)blockIdx.x;
    nb = (int)gridDim.x;
    arrivals = (unsigned int)(nb + a.bar_extra);
    bar = a.bar;
    gpart = a.gpart;
    pub_w = a.pub;
    pub_r = a.pub;
  }
  // bounded barrier over the grid: false once any CTA has given up waiting.  Every thread
  // fences its global writes before the CTA's arrival.
  __device__ bool sync() {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int g = *(volatile unsigned int*)&bar->gen;
      if (atomicAdd(&bar->count, 1u) == arrivals - 1u) {
        atomicExch(&bar->count, 0u);
        __threadfence();
        atomicAdd(&bar->gen, 1u);
      } else {
        const long long t0 = clock64();
        while (*(volatile unsigned int*)&bar->gen == g) {
          if (clock64() - t0 > GRID_WAIT_LIMIT) {
            atomicExch(&bar->err, 1);
            break;
          }
        }
      }
      __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&bar->err == 0;
  }
  __device__ bool sum(double* mine, int buf, double* tot, int nval) {
    double* my = gpart + ((int64_t)buf * nb + rank) * GC_PART;
    __syncthreads();                         // every warp's partials are in `mine`
    for (int i = threadIdx.x; i < nval; i += blockDim.x) my[i] = mine[i];
    if (!sync()) return false;
    // one warp per value: lanes add ranks lane, lane + 32, ... then a fixed shuffle tree,
    // so the totals are bitwise the same in every CTA
    const double* base = gpart + (int64_t)buf * nb * GC_PART;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < nval; i += (int)(blockDim.x >> 5)) {
      double s = 0.0;
#pragma unroll 8
      for (int c = lane; c < nb; c += 32) s += __ldcg(base + (int64_t)c * GC_PART + i);
      s = gc_warp_sum(s);
      if (lane == 0) tot[i] = s;
    }
    __syncthreads();
    return true;
  }
  __device__ int ld(const int* p) const { return __ldcg(p); }
  __device__ double ld(const double* p) const { return __ldcg(p); }
  __device__ void finish() {}
};

// ---- the solve -----------------------------------------------------------------------------

template <class Comm>
__global__ void __launch_bounds__(GC_THREADS, 1) k_gmres_fused(const GcArgs a) {
  extern __shared__ __align__(16) double gc_dyn[];
  __shared__ double part[2][GC_PART];
  __shared__ double tot[GC_PART];
  __shared__ double sC[NMAX], sC2[NMAX], sT[NMAX + 1], sy[NMAX];
  __shared__ double s_g[NMAX + 1], s_gc[NMAX], s_gs[NMAX];   // CTA 0: Givens state
  __shared__ double scratch[GC_WARPS];
  __shared__ double s_alpha, s_inv_alpha;
  __shared__ int s_status;                                   // CTA 0: first failure of a cycle
  __shared__ GcPub s_pub;                                    // cluster form: CTA 0's state
  Comm comm(a, &s_pub);
  const int rank = comm.rank, nb = comm.nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // row block of this CTA: the CTAs that own rows split them evenly (with skip0, CTA 0
  // owns none and its H, K, Givens work runs while the others compute)
  const int nrb = a.skip0 ? nb - 1 : nb, rr = a.skip0 ? rank - 1 : rank;
  const int64_t r0 = rr < 0 ? 0 : a.m * rr / nrb, r1 = rr < 0 ? 0 : a.m * (rr + 1) / nrb;
  const int nrow = (int)(r1 - r0);
  const int n = a.n, ldh = n + 1, ldk = n + 1, ldr = n;
  // this CTA's rows of the basis (column j at Qb + j * qs, row r at index r - r0), of v
  // and of w, and CTA 0's H, K, R: in shared memory where they fit, else in global memory.
  // w is also kept in global memory (wg), where the other CTAs' matvecs read it.
  double* const dyn = gc_dyn;
  double* const Qb = a.smem_q ? dyn : a.Q + r0;
  const int64_t qs = a.smem_q ? (int64_t)a.rc : a.ldq;
  double* const vb = a.smem_q ? dyn + (int64_t)(n + 1) * a.rc : a.v + r0;
  double* const wg = a.w + r0;
  double* const wb = a.smem_q ? vb + a.rc : wg;
  double* const hb = a.smem_q ? wb + a.rc : dyn;
  double* const Hm = a.smem_h ? hb : a.H;
  double* const Km = a.smem_h ? hb + (n + 1) * n : a.K;
  double* const Rm = a.smem_h ? hb + 2 * (n + 1) * n : a.R;
  GcPub* const pw = comm.pub_w;
  const GcPub* const pr = comm.pub_r;
  int pb = 0;                             // partial-sum buffer of the next reduction
  int matvecs = 0, cycles = 0, last_status = KC_OK, result = KC_ERR_NOT_CONVERGED;
  double rn = 0.0, est = 0.0, bnorm = 0.0, target = 0.0;
  // H below its subdiagonal is never written but is read by the K-column product
  // (T - H(0:k, 0:k-1) C / alpha over the full block): zero it (the global copy is zeroed by the host)
  if (rank == 0 && a.smem_h)
    for (int i = tid; i < (n + 1) * n; i += GC_THREADS) Hm[i] = 0.0;

  // ||b|| and the absolute tolerance
  {
    double acc = 0.0;
    for (int64_t r = r0 + tid; r < r1; r += GC_THREADS) acc += a.b[r] * a.b[r];
    gc_block_sum(acc, part[pb], scratch);
    if (!comm.sum(part[pb], pb, tot, 1)) goto failed;
    pb ^= 1;
  }
  bnorm = sqrt(tot[0]);
  if (!(bnorm > 0.0)) {
    for (int64_t r = r0 + tid; r < r1; r += GC_THREADS) a.x[r] = 0.0;
    result = KC_OK;
    goto done;
  }
  target = a.rtol * bnorm;

  for (;;) {
    // ---- FP64 residual w = r = b - A x and its norm (x is written by every CTA) ----
    if (!comm.sync()) goto failed;
    {
      double acc = 0.0;
      for (int i = tid; i < nrow; i += GC_THREADS) {
        const double rr = a.b[r0 + i] - gc_apply_row(a, a.x, r0 + i);
        wb[i] = rr;
        if (a.smem_q) wg[i] = rr;
        acc += rr * rr;
      }
      gc_block_sum(acc, part[pb], scratch);
      if (!comm.sum(part[pb], pb, tot, 1)) goto failed;
      pb ^= 1;
    }
    rn = sqrt(tot[0]);
    if (rn <= target) { result = KC_OK; break; }
    if (matvecs >= a.maxit) break;

    // ---- one GMRES(n) cycle ----
    if (rank == 0 && tid == 0) {
      pw->stop = 0;
      pw->ncols = 0;
      pw->est = 0.0;
      s_status = KC_OK;
    }
    bool stopped = false;
    for (int k = 0; k < n; k++) {
      // v = A w on this CTA's rows (w of the neighbouring rows comes from other CTAs)
      for (int i = tid; i < nrow; i += GC_THREADS) vb[i] = gc_apply_row(a, a.w, r0 + i);
      __syncthreads();
      // partial sums: task t < k gives (q_t^T w, q_t^T v), task k (w^T w, w^T v)
      for (int t = warp; t <= k; t += GC_WARPS) {
        const double* q = t < k ? Qb + (int64_t)t * qs : wb;
        double s0 = 0.0, s1 = 0.0;
        for (int i = lane; i < nrow; i += 32) {
          const double qi = q[i];
          s0 += qi * wb[i];
          s1 += qi * vb[i];
        }
        s0 = gc_warp_sum(s0);
        s1 = gc_warp_sum(s1);
        if (lane == 0) {
          part[pb][2 * t] = s0;
          part[pb][2 * t + 1] = s1;
        }
      }
      if (!comm.sum(part[pb], pb, tot, 2 * k + 2)) goto failed;
      pb ^= 1;
      // scalar step (every CTA): Pythagoras, T (eq. 30)
      if (warp == 0) {
        double cc = 0.0, cs = 0.0;
        for (int i = lane; i < k; i += 32) {
          cc += tot[2 * i] * tot[2 * i];
          cs += tot[2 * i] * tot[2 * i + 1];
        }
        cc = gc_warp_sum(cc);
        cs = gc_warp_sum(cs);
        if (lane == 0) {
          const double beta = tot[2 * k], s = tot[2 * k + 1];
          double a2 = beta - cc;
          if (!isfinite(a2) || !isfinite(s)) {
            if (rank == 0) gc_set_status(&s_status, KC_ERR_NONFINITE);
          } else if (!(a2 > 0.0)) {
            if (rank == 0) gc_set_status(&s_status, KC_ERR_PYTHAGORAS_NEG);
            a2 = fmax(a2, 1e-300);
          }
          const double alpha = sqrt(a2), ia = 1.0 / alpha;
          s_alpha = alpha;
          s_inv_alpha = ia;
          sT[k] = (s - cs) * ia * ia;
        }
      }
      __syncthreads();
      const double alpha = s_alpha, inv_alpha = s_inv_alpha;
      for (int i = tid; i < k; i += GC_THREADS) {
        sC[i] = tot[2 * i];
        sT[i] = tot[2 * i + 1] * inv_alpha;
      }
      __syncthreads();
      // update of this CTA's rows: q_k = (w - Q C)/alpha, w <- v/alpha - Q T - q_k T_k
      for (int i = tid; i < nrow; i += GC_THREADS) {
        double qc = 0.0, qt = 0.0;
        for (int j = 0; j < k; j++) {
          const double qj = Qb[(int64_t)j * qs + i];
          qc += qj * sC[j];
          qt += qj * sT[j];
        }
        const double q = (wb[i] - qc) * inv_alpha;
        Qb[(int64_t)k * qs + i] = q;
        const double wn = vb[i] * inv_alpha - qt - q * sT[k];
        wb[i] = wn;
        if (a.smem_q) wg[i] = wn;
      }
      // CTA 0: H(0:k, k-1) = K(0:k, k-1) + C, H(k, k-1) = alpha;
      // K(0:k, k) = T - H(0:k, 0:k-1) C / alpha; Givens of column k-1
      if (rank == 0) {
        if (k >= 1) {
          for (int i = tid; i < k; i += GC_THREADS)
            Hm[i + (int64_t)(k - 1) * ldh] = Km[i + (int64_t)(k - 1) * ldk] + sC[i];
          if (tid == 0) Hm[k + (int64_t)(k - 1) * ldh] = alpha;
          __syncthreads();
          if (warp == 0) {
            double cn = 0.0;
            for (int i = lane; i <= k; i += 32) {
              const double h = Hm[i + (int64_t)(k - 1) * ldh];
              cn += h * h;
            }
            cn = gc_warp_sum(cn);
            if (lane == 0 && alpha <= 1e-13 * sqrt(cn)) gc_set_status(&s_status, KC_ERR_BREAKDOWN);
          }
          if (tid == 32) {                  // Givens rotation of the finalised column k-1
            const double e = givens_rotate(s_gc, s_gs, s_g, Hm, ldh, k - 1, Rm, ldr);
            pw->est = e;
            pw->ncols = k;
            if (!(e > target)) pw->stop = 1;
          }
        } else if (tid == 0) {
          s_g[0] = alpha;
        }
        for (int i = tid; i <= k; i += GC_THREADS) {
          double hc = 0.0;
          for (int j = 0; j < k; j++) hc += Hm[i + (int64_t)j * ldh] * sC[j];
          Km[i + (int64_t)k * ldk] = sT[i] - hc * inv_alpha;
        }
      }
      // w and CTA 0's stop flag become visible to every CTA
      if (!comm.sync()) goto failed;
      if (comm.ld(&pr->stop)) { stopped = true; break; }
    }
    if (!stopped) {
      // CGS2 finish of the last column: C1 = Q^T w, w -= Q C1, C2 = Q^T w, w -= Q C2,
      // alpha = ||w||; H(:, n-1) = K(:, n-1) + C1 + C2, H(n, n-1) = alpha
      for (int pass = 0; pass < 3; pass++) {
        const int ntask = pass < 2 ? n : 0;      // pass 2: the norm alone
        for (int t = warp; t <= ntask; t += GC_WARPS) {
          const double* q = t < ntask ? Qb + (int64_t)t * qs : wb;
          double s0 = 0.0;
          for (int i = lane; i < nrow; i += 32) s0 += q[i] * wb[i];
          s0 = gc_warp_sum(s0);
          if (lane == 0) part[pb][t] = s0;
        }
        if (!comm.sum(part[pb], pb, tot, ntask + 1)) goto failed;
        pb ^= 1;
        if (pass == 2) break;
        double* cdst = pass == 0 ? sC : sC2;
        for (int i = tid; i < n; i += GC_THREADS) cdst[i] = tot[i];
        __syncthreads();
        for (int i = tid; i < nrow; i += GC_THREADS) {
          double qc = 0.0;
          for (int j = 0; j < n; j++) qc += Qb[(int64_t)j * qs + i] * cdst[j];
          wb[i] -= qc;
        }
        __syncthreads();
      }
      const double alpha = sqrt(tot[0]);
      if (rank == 0) {
        for (int i = tid; i < n; i += GC_THREADS)
          Hm[i + (int64_t)(n - 1) * ldh] = Km[i + (int64_t)(n - 1) * ldk] + sC[i] + sC2[i];
        if (tid == 0) Hm[n + (int64_t)(n - 1) * ldh] = alpha;
        __syncthreads();
        if (warp == 0) {
          double cn = 0.0;
          for (int i = lane; i <= n; i += 32) {
            const double h = Hm[i + (int64_t)(n - 1) * ldh];
            cn += h * h;
          }
          cn = gc_warp_sum(cn);
          if (lane == 0 && alpha <= 1e-13 * sqrt(cn)) gc_set_status(&s_status, KC_ERR_BREAKDOWN);
        }
        if (tid == 32) {
          const double e = givens_rotate(s_gc, s_gs, s_g, Hm, ldh, n - 1, Rm, ldr);
          pw->est = e;
          pw->ncols = n;
          if (!(e > target)) pw->stop = 1;
        }
      }
    }
    // y = R^{-1} g in CTA 0 (column-oriented back substitution), published with the
    // column count; then x += Q y everywhere
    if (rank == 0) {
      __syncthreads();
      const int nc = pw->ncols;
      for (int i = tid; i < nc; i += GC_THREADS) sy[i] = s_g[i];
      for (int j = nc - 1; j >= 0; j--) {
        __syncthreads();
        if (tid == 0) sy[j] = sy[j] / Rm[j + (int64_t)j * ldr];
        __syncthreads();
        const double yj = sy[j];
        for (int i = tid; i < j; i += GC_THREADS) sy[i] -= Rm[i + (int64_t)j * ldr] * yj;
      }
      __syncthreads();
      for (int i = tid; i < nc; i += GC_THREADS) pw->y[i] = sy[i];
    }
    if (!comm.sync()) goto failed;
    {
      const int nc = comm.ld(&pr->ncols);   // columns finalised in this cycle
      double* yl = sT;                      // local copy of y (T is not needed any more)
      for (int i = tid; i < nc; i += GC_THREADS) yl[i] = comm.ld(&pr->y[i]);
      __syncthreads();
      for (int i = tid; i < nrow; i += GC_THREADS) {
        double s = 0.0;
        for (int j = 0; j < nc; j++) s += Qb[(int64_t)j * qs + i] * yl[j];
        a.x[r0 + i] += s;
      }
      const int stop_flag = comm.ld(&pr->stop);
      matvecs += (stop_flag && nc < n) ? nc + 1 : n;
      cycles++;
      est = comm.ld(&pr->est);
      if (rank == 0 && s_status != KC_OK && s_status != KC_ERR_BREAKDOWN) last_status = s_status;
    }
  }
  goto done;
failed:
  result = KC_ERR_TIMEOUT;
done:
  comm.finish();
  if (rank == 0 && tid == 0) {
    a.out[0] = matvecs;
    a.out[1] = cycles;
    a.out[2] = est;
    a.out[3] = rn;
    a.out[4] = bnorm;
    a.out[5] = result;
    a.out[6] = last_status;
  }
}

// ---- launch --------------------------------------------------------------------------------

// cluster size the device can schedule for the kernel with `smem` bytes of dynamic shared
// memory (16, else 8; 0 if neither)
static int gmres_cluster_size(int smem) {
  for (int cs = 16; cs >= 8; cs /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(GC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_gmres_fused<ClusterComm>, &cfg) ==
            cudaSuccess &&
        nclusters >= 1)
      return cs;
    cudaGetLastError();
  }
  return 0;
}

static void gmres_fused_setup(kc_ctx* ctx) {
  static std::atomic<unsigned long long> attr_done{0};
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (!(attr_done.load(std::memory_order_acquire) & bit)) {
    cudaFuncSetAttribute(k_gmres_fused<ClusterComm>,
                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_gmres_fused<ClusterComm>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, GC_DYN_SMEM_MAX);
    cudaFuncSetAttribute(k_gmres_fused<GridComm>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, GC_DYN_SMEM_MAX);
    cudaGetLastError();
    attr_done.fetch_or(bit, std::memory_order_release);
  }
  if (ctx->gmres_cluster == 0) {
    const int probed = gmres_cluster_size(GC_DYN_SMEM_MAX);
    ctx->gmres_cluster = probed > 0 ? probed : -1;
  }
}

// shared-memory bytes of a CTA's rows of Q (n+1 columns), v and w
static int64_t gmres_fused_row_bytes(int64_t m, int n, int ctas) {
  return (int64_t)(n + 3) * ((m + ctas - 1) / ctas) * 8;
}

bool gmres_grid_preferred(kc_ctx* ctx, int64_t m, int n) {
  gmres_fused_setup(ctx);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gmres_fused<GridComm>, GC_THREADS,
                                                    GC_DYN_SMEM_MAX) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  (void)n;
  return occ >= 1 && m <= GMRES_GRID_MAX_ROWS;
}

size_t gmres_grid_workspace(const kc_ctx* ctx) {
  return (size_t)2 * ctx->num_sms * GC_PART * sizeof(double) + sizeof(GcPub) + sizeof(GridBar);
}

kc_status gmres_fused_solve(kc_ctx* ctx, int grid_form, const kc_csr* A, const double* b,
                            double* x, double* Q, int64_t ldq, double* w, double* v, double* H,
                            double* K, double* R, int n, int maxit, double rtol,
                            void* grid_ws, double* out_dev, double* out_host) {
  gmres_fused_setup(ctx);
  int ctas;
  if (grid_form) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gmres_fused<GridComm>,
                                                      GC_THREADS, GC_DYN_SMEM_MAX) !=
            cudaSuccess ||
        occ < 1)
      return fail(ctx, KC_ERR_CUDA, "gmres: the grid-wide kernel cannot be resident");
    ctas = ctx->num_sms;
  } else {
    if (ctx->gmres_cluster < 0)
      return fail(ctx, KC_ERR_CUDA, "gmres: no thread-block cluster can be scheduled");
    ctas = ctx->gmres_cluster;
  }
  GcArgs a = {};
  if (is_stencil(A)) {
    a.stencil = 1;
    a.nx = A->grid[0];
    a.ny = A->grid[1];
    a.nz = A->grid[2];
    for (int i = 0; i < 7; i++) a.c7[i] = A->stencil[i];
  } else {
    a.rp = A->row_ptr;
    a.ci = A->col_idx;
    a.val = (const double*)A->val;
  }
  a.b = b; a.x = x; a.Q = Q; a.ldq = ldq; a.w = w; a.v = v; a.H = H; a.K = K; a.R = R;
  a.n = n; a.maxit = maxit; a.m = A->m; a.rtol = rtol; a.out = out_dev;
  // shared-memory residency: rows of Q, v and w per CTA, then CTA 0's H, K, R
  a.skip0 = grid_form && ctas >= 2 ? 1 : 0;
  const int row_ctas = ctas - a.skip0;
  const int64_t bq = gmres_fused_row_bytes(A->m, n, row_ctas);
  const int64_t bh = (int64_t)(2 * (n + 1) * n + n * n) * 8;
  a.rc = (int)((A->m + row_ctas - 1) / row_ctas);
  a.smem_q = bq <= GC_DYN_SMEM_MAX;
  a.smem_h = (a.smem_q ? bq : 0) + bh <= GC_DYN_SMEM_MAX;
  const int64_t dyn = (a.smem_q ? bq : 0) + (a.smem_h ? bh : 0);
  a.bar_extra = ctx->barrier_test ? 1 : 0;
  ctx->barrier_test = 0;
  timing_begin(ctx, KID_OTHER);
  if (grid_form) {
    char* g = (char*)grid_ws;
    a.gpart = (double*)g;
    a.pub = (GcPub*)(g + (size_t)2 * ctas * GC_PART * sizeof(double));
    a.bar = (GridBar*)((char*)a.pub + sizeof(GcPub));
    KC_CUDA(ctx, cudaMemsetAsync(a.bar, 0, sizeof(GridBar), ctx->stream));
    void* args[] = {(void*)&a};
    KC_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_gmres_fused<GridComm>, dim3(ctas),
                                             dim3(GC_THREADS), args, (size_t)dyn, ctx->stream));
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas, 1, 1);
    cfg.blockDim = dim3(GC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)dyn;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    KC_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_gmres_fused<ClusterComm>, a));
  }
  KC_LAUNCHED(ctx);
  KC_CUDA(ctx, cudaMemcpyAsync(out_host, out_dev, 7 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return KC_OK;
}

}  // namespace kc
