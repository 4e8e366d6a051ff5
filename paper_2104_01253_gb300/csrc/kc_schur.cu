// Krylov-Schur eigenvalues (Stewart's restart) on DCGS2-Arnoldi, all on the GPU.
//
// The small dense step runs in one CTA in FP64 shared memory:
//   1. Householder reduction of B = H(0:n, 0:n) to Hessenberg form (B is full after a
//      restart), accumulating Z;
//   2. Francis double-shift QR iterations (implicit bulge chasing) to real Schur form,
//      with deflation on negligible subdiagonals and exceptional shifts every tenth
//      iteration; 2x2 blocks with real eigenvalues are split by one rotation;
//   3. reordering: adjacent diagonal blocks are swapped until the wanted Ritz values
//      (largest real part) lead.  A swap solves the Sylvester equation
//      T11 X - X T22 = T12 and applies the orthogonal factor of [-X; I];
//   4. Ritz residuals |b^T Z y| / ||y|| (eq. "ArnoldiRes", b = last row of H) from
//      eigenvectors y of the leading block by (complex) back substitution.
// The host then truncates Q <- Q Z(:, 0:p), keeps q_n, sets H = [T_pp; b^T Z(:, 0:p)],
// projects A q_p once against Q_{p+1} and resumes DCGS2 steps.
#include "kc_internal.cuh"

namespace kc {

constexpr int KS_MAX = 64;          // largest ncv supported by the dense step
constexpr int KS_THREADS = 64;

struct KsOut {
  int p;                            // kept columns
  int nconv;
  int status;                       // 0 ok, 1 QR did not converge, 2 swap failed
  int nblocks;
  double eig_re[KS_MAX], eig_im[KS_MAX], resid[KS_MAX];   // wanted, sorted, first p
  double btil[KS_MAX];              // b^T Z
};

struct Ks {
  double* T;      // smem, row-major [n][ld]
  double* Z;
  int n, ld;
  __device__ double& t(int i, int j) { return T[i * ld + j]; }
  __device__ double& z(int i, int j) { return Z[i * ld + j]; }
};

// Householder reflector for a (len <= 4): P = I - beta v v^T with P a = alpha e1.
__device__ void house(const double* a, int len, double* v, double* beta) {
  double nrm = 0.0;
  for (int i = 0; i < len; i++) nrm += a[i] * a[i];
  nrm = sqrt(nrm);
  if (nrm == 0.0) {
    for (int i = 0; i < len; i++) v[i] = 0.0;
    v[0] = 1.0;
    *beta = 0.0;
    return;
  }
  const double alpha = a[0] >= 0.0 ? -nrm : nrm;
  for (int i = 0; i < len; i++) v[i] = a[i];
  v[0] -= alpha;
  double vv = 0.0;
  for (int i = 0; i < len; i++) vv += v[i] * v[i];
  *beta = vv > 0.0 ? 2.0 / vv : 0.0;
}

// rows r0..r0+len-1, columns c0..c1-1: T <- P T   (all threads)
__device__ void left_reflect(Ks& K, int r0, int len, const double* v, double beta, int c0, int c1) {
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < len; i++) s += v[i] * K.t(r0 + i, c);
    s *= beta;
    for (int i = 0; i < len; i++) K.t(r0 + i, c) -= s * v[i];
  }
}

// columns c0..c0+len-1, rows r0..r1-1: M <- M P   (M = T or Z; all threads)
__device__ void right_reflect(double* M, int ld, int c0, int len, const double* v, double beta,
                              int r0, int r1) {
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < len; i++) s += M[r * ld + c0 + i] * v[i];
    s *= beta;
    for (int i = 0; i < len; i++) M[r * ld + c0 + i] -= s * v[i];
  }
}

// rows/cols j, j+1: T <- G^T T G, Z <- Z G with G = [c -s; s c]   (all threads)
__device__ void rotate(Ks& K, int j, double c, double s) {
  const int n = K.n;
  for (int col = threadIdx.x; col < n; col += blockDim.x) {
    double a = K.t(j, col), b = K.t(j + 1, col);
    K.t(j, col) = c * a + s * b;
    K.t(j + 1, col) = -s * a + c * b;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double a = K.t(r, j), b = K.t(r, j + 1);
    K.t(r, j) = c * a + s * b;
    K.t(r, j + 1) = -s * a + c * b;
    a = K.z(r, j);
    b = K.z(r, j + 1);
    K.z(r, j) = c * a + s * b;
    K.z(r, j + 1) = -s * a + c * b;
  }
  __syncthreads();
}

__device__ void hessenberg(Ks& K, double* sv) {
  const int n = K.n;
  for (int j = 0; j + 2 < n; j++) {
    const int len = n - j - 1;
    // Householder on T(j+1:n, j): computed in a length-n scratch (sv), beta in sv[KS_MAX]
    if (threadIdx.x == 0) {
      double nrm = 0.0;
      for (int i = 0; i < len; i++) nrm += K.t(j + 1 + i, j) * K.t(j + 1 + i, j);
      nrm = sqrt(nrm);
      const double a0 = K.t(j + 1, j);
      const double alpha = a0 >= 0.0 ? -nrm : nrm;
      for (int i = 0; i < len; i++) sv[i] = K.t(j + 1 + i, j);
      sv[0] -= alpha;
      double vv = 0.0;
      for (int i = 0; i < len; i++) vv += sv[i] * sv[i];
      sv[KS_MAX] = (nrm == 0.0 || vv == 0.0) ? 0.0 : 2.0 / vv;
    }
    __syncthreads();
    const double beta = sv[KS_MAX];
    if (beta != 0.0) {
      left_reflect(K, j + 1, len, sv, beta, j, n);
      __syncthreads();
      right_reflect(K.T, K.ld, j + 1, len, sv, beta, 0, n);
      right_reflect(K.Z, K.ld, j + 1, len, sv, beta, 0, n);
      __syncthreads();
    }
    for (int i = j + 2 + threadIdx.x; i < n; i += blockDim.x) K.t(i, j) = 0.0;
    __syncthreads();
  }
}

// Francis double-shift QR to real Schur form.  Returns false if it does not converge.
__device__ bool francis(Ks& K, double* sv) {
  const int n = K.n;
  const double eps = 2.220446049250313e-16;
  double tnorm = 0.0;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) tnorm = fmax(tnorm, fabs(K.t(i, j)));
  __shared__ int s_hi, s_l, s_iter, s_total, s_done;
  if (threadIdx.x == 0) { s_hi = n - 1; s_iter = 0; s_total = 0; s_done = 0; }
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) {
      int hi = s_hi;
      while (hi >= 0) {
        int l = hi;
        while (l > 0) {
          double s = fabs(K.t(l - 1, l - 1)) + fabs(K.t(l, l));
          if (s == 0.0) s = tnorm;
          if (fabs(K.t(l, l - 1)) < eps * s) { K.t(l, l - 1) = 0.0; break; }
          l--;
        }
        if (l >= hi - 1) {               // 1x1 or 2x2 block converged
          hi = l - 1;
          s_iter = 0;
          continue;
        }
        s_l = l;
        break;
      }
      s_hi = hi;
      if (hi < 0) s_done = 1;
      else if (++s_total > 40 * n) s_done = 2;
      s_iter++;
    }
    __syncthreads();
    if (s_done) break;
    const int hi = s_hi, l = s_l;
    // shifts: the eigenvalues of the trailing 2x2 block, or an exceptional pair
    __shared__ double xyz[4];
    if (threadIdx.x == 0) {
      double tr, det;
      if (s_iter % 11 == 10) {
        const double s = fabs(K.t(hi, hi - 1)) + fabs(K.t(hi - 1, hi - 2));
        tr = 1.5 * s;
        det = s * s;
      } else {
        tr = K.t(hi - 1, hi - 1) + K.t(hi, hi);
        det = K.t(hi - 1, hi - 1) * K.t(hi, hi) - K.t(hi - 1, hi) * K.t(hi, hi - 1);
      }
      const double a = K.t(l, l), b = K.t(l, l + 1), c = K.t(l + 1, l);
      xyz[0] = a * a + b * c - tr * a + det;
      xyz[1] = c * (a + K.t(l + 1, l + 1) - tr);
      xyz[2] = c * K.t(l + 2, l + 1);
    }
    __syncthreads();
    for (int k = l; k <= hi - 1; k++) {
      const int len = (k <= hi - 2) ? 3 : 2;
      __shared__ double v[4], beta;
      if (threadIdx.x == 0) house(xyz, len, v, &beta);
      __syncthreads();
      const int q = k > l ? k - 1 : l;
      left_reflect(K, k, len, v, beta, q, n);
      __syncthreads();
      const int r = (k + 3 < hi) ? k + 3 : hi;
      right_reflect(K.T, K.ld, k, len, v, beta, 0, r + 1);
      right_reflect(K.Z, K.ld, k, len, v, beta, 0, n);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (k > l) {
          K.t(k + 1, k - 1) = 0.0;
          if (len == 3) K.t(k + 2, k - 1) = 0.0;
        }
        if (k < hi - 1) {
          xyz[0] = K.t(k + 1, k);
          xyz[1] = K.t(k + 2, k);
          xyz[2] = (k < hi - 2) ? K.t(k + 3, k) : 0.0;
        }
      }
      __syncthreads();
    }
  }
  return s_done == 1;
}

// eigenvalues of [a b; c d]: returns true if complex (re +- i im)
__device__ bool eig2(double a, double b, double c, double d, double* re1, double* im1,
                     double* re2) {
  const double p = 0.5 * (a - d);
  const double disc = p * p + b * c;
  if (disc >= 0.0) {
    const double sq = sqrt(disc);
    const double z = p + (p >= 0.0 ? sq : -sq);
    *re1 = d + z;
    *re2 = (z != 0.0) ? d - b * c / z : d;
    *im1 = 0.0;
    return false;
  }
  *re1 = 0.5 * (a + d);
  *re2 = *re1;
  *im1 = sqrt(-disc);
  return true;
}

// Split every 2x2 diagonal block that has real eigenvalues into two 1x1 blocks.
__device__ void split_real_pairs(Ks& K) {
  const int n = K.n;
  for (int j = 0; j + 1 < n; j++) {
    __shared__ int s_do;
    __shared__ double cs, sn;
    if (threadIdx.x == 0) {
      s_do = 0;
      if (K.t(j + 1, j) != 0.0) {
        const double a = K.t(j, j), b = K.t(j, j + 1), c = K.t(j + 1, j), d = K.t(j + 1, j + 1);
        double r1, i1, r2;
        if (!eig2(a, b, c, d, &r1, &i1, &r2)) {
          // eigenvector for r1: (b, r1 - a) or (r1 - d, c), the better conditioned one
          double u0 = b, u1 = r1 - a;
          double w0 = r1 - d, w1 = c;
          if (u0 * u0 + u1 * u1 < w0 * w0 + w1 * w1) { u0 = w0; u1 = w1; }
          const double nn = hypot(u0, u1);
          cs = u0 / nn;
          sn = u1 / nn;
          s_do = 1;
        }
      }
    }
    __syncthreads();
    if (s_do) {
      rotate(K, j, cs, sn);
      if (threadIdx.x == 0) K.t(j + 1, j) = 0.0;
      __syncthreads();
    }
  }
}

// Swap the adjacent diagonal blocks at j1 (size n1) and j1+n1 (size n2).
__device__ bool swap_blocks(Ks& K, int j1, int n1, int n2) {
  const int n = K.n, nb = n1 + n2;
  __shared__ double Qh[4][4];
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_ok = 1;
    // Sylvester T11 X - X T22 = T12 as a (n1*n2) linear system, x = vec(X) column-major
    const int N = n1 * n2;
    double M[4][5];
    for (int r = 0; r < N; r++)
      for (int c = 0; c <= N; c++) M[r][c] = 0.0;
    for (int jj = 0; jj < n2; jj++)
      for (int ii = 0; ii < n1; ii++) {
        const int row = ii + jj * n1;
        for (int kk = 0; kk < n1; kk++) M[row][kk + jj * n1] += K.t(j1 + ii, j1 + kk);
        for (int kk = 0; kk < n2; kk++) M[row][ii + kk * n1] -= K.t(j1 + n1 + kk, j1 + n1 + jj);
        M[row][N] = K.t(j1 + ii, j1 + n1 + jj);
      }
    double scale = 0.0;
    for (int r = 0; r < N; r++)
      for (int c = 0; c < N; c++) scale = fmax(scale, fabs(M[r][c]));
    for (int c = 0; c < N; c++) {           // Gaussian elimination, partial pivoting
      int piv = c;
      for (int r = c + 1; r < N; r++)
        if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
      if (fabs(M[piv][c]) <= 1e-300 + 1e-15 * scale) { M[piv][c] = 1e-15 * scale + 1e-300; }
      if (piv != c)
        for (int k = 0; k <= N; k++) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
      for (int r = c + 1; r < N; r++) {
        const double f = M[r][c] / M[c][c];
        for (int k = c; k <= N; k++) M[r][k] -= f * M[c][k];
      }
    }
    double X[4];
    for (int r = N - 1; r >= 0; r--) {
      double s = M[r][N];
      for (int k = r + 1; k < N; k++) s -= M[r][k] * X[k];
      X[r] = s / M[r][r];
    }
    // W = [-X; I] (nb x n2); Householder QR, accumulate Qh = H1 H2 (nb x nb)
    double W[4][2];
    for (int jj = 0; jj < n2; jj++) {
      for (int ii = 0; ii < n1; ii++) W[ii][jj] = -X[ii + jj * n1];
      for (int kk = 0; kk < n2; kk++) W[n1 + kk][jj] = (kk == jj) ? 1.0 : 0.0;
    }
    for (int r = 0; r < 4; r++)
      for (int c = 0; c < 4; c++) Qh[r][c] = (r == c) ? 1.0 : 0.0;
    for (int jj = 0; jj < n2; jj++) {
      double a[4], v[4], beta;
      const int len = nb - jj;
      for (int i = 0; i < len; i++) a[i] = W[jj + i][jj];
      house(a, len, v, &beta);
      for (int c = jj; c < n2; c++) {           // W <- H W
        double s = 0.0;
        for (int i = 0; i < len; i++) s += v[i] * W[jj + i][c];
        s *= beta;
        for (int i = 0; i < len; i++) W[jj + i][c] -= s * v[i];
      }
      for (int r = 0; r < nb; r++) {            // Qh <- Qh H
        double s = 0.0;
        for (int i = 0; i < len; i++) s += Qh[r][jj + i] * v[i];
        s *= beta;
        for (int i = 0; i < len; i++) Qh[r][jj + i] -= s * v[i];
      }
    }
  }
  __syncthreads();
  // T(j1:j1+nb, j1:n) <- Qh^T T(...);  T(0:j1+nb, j1:j1+nb) <- T Qh;  Z <- Z Qh
  for (int c = j1 + threadIdx.x; c < n; c += blockDim.x) {
    double old[4], nw[4];
    for (int i = 0; i < nb; i++) old[i] = K.t(j1 + i, c);
    for (int i = 0; i < nb; i++) {
      double s = 0.0;
      for (int l = 0; l < nb; l++) s += Qh[l][i] * old[l];
      nw[i] = s;
    }
    for (int i = 0; i < nb; i++) K.t(j1 + i, c) = nw[i];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double old[4], nw[4];
    if (r < j1 + nb) {
      for (int i = 0; i < nb; i++) old[i] = K.t(r, j1 + i);
      for (int i = 0; i < nb; i++) {
        double s = 0.0;
        for (int l = 0; l < nb; l++) s += old[l] * Qh[l][i];
        nw[i] = s;
      }
      for (int i = 0; i < nb; i++) K.t(r, j1 + i) = nw[i];
    }
    for (int i = 0; i < nb; i++) old[i] = K.z(r, j1 + i);
    for (int i = 0; i < nb; i++) {
      double s = 0.0;
      for (int l = 0; l < nb; l++) s += old[l] * Qh[l][i];
      nw[i] = s;
    }
    for (int i = 0; i < nb; i++) K.z(r, j1 + i) = nw[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double blk = 0.0, low = 0.0;
    for (int i = 0; i < nb; i++)
      for (int j = 0; j < nb; j++) blk = fmax(blk, fabs(K.t(j1 + i, j1 + j)));
    for (int i = n2; i < nb; i++)
      for (int j = 0; j < n2; j++) {
        low = fmax(low, fabs(K.t(j1 + i, j1 + j)));
        K.t(j1 + i, j1 + j) = 0.0;
      }
    if (low > 1e-10 * blk) s_ok = 0;
    // the moved 1x1 blocks have no subdiagonal coupling
    if (n2 == 1 && nb > 1) { /* new leading block is 1x1 */ }
    for (int i = 0; i + 1 < nb; i++) {
      const bool leading2 = (n2 == 2 && i == 0), trailing2 = (n1 == 2 && i == n2);
      if (!leading2 && !trailing2) K.t(j1 + i + 1, j1 + i) = 0.0;
    }
  }
  __syncthreads();
  return s_ok;
}

// block structure: start of each block and its size
__device__ int blocks_of(Ks& K, int* bstart, int* bsize) {
  int nb = 0;
  for (int j = 0; j < K.n;) {
    const int sz = (j + 1 < K.n && K.t(j + 1, j) != 0.0) ? 2 : 1;
    bstart[nb] = j;
    bsize[nb] = sz;
    nb++;
    j += sz;
  }
  return nb;
}

__device__ void block_eigs(Ks& K, int j, int sz, double* re, double* im) {
  if (sz == 1) { re[0] = K.t(j, j); im[0] = 0.0; re[1] = 0.0; im[1] = 0.0; return; }
  double r1, i1, r2;
  eig2(K.t(j, j), K.t(j, j + 1), K.t(j + 1, j), K.t(j + 1, j + 1), &r1, &i1, &r2);
  re[0] = r1; im[0] = i1; re[1] = r1; im[1] = -i1;
}

__device__ bool key_before(double ra, double ia, int xa, double rb, double ib, int xb) {
  if (ra != rb) return ra > rb;
  if (ia != ib) return ia > ib;
  return xa < xb;
}

__global__ void __launch_bounds__(KS_THREADS)
k_ks_schur(const double* __restrict__ H, int ldh, int n, int nkeep, int nev, double tol,
           double* __restrict__ Tout, double* __restrict__ Zout, KsOut* __restrict__ out) {
  extern __shared__ double smem[];
  Ks K;
  K.n = n;
  K.ld = n;
  K.T = smem;
  K.Z = smem + n * n;
  double* sv = smem + 2 * n * n;              // KS_MAX + 1 scratch
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    K.T[idx] = H[i + (int64_t)j * ldh];
    K.Z[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  hessenberg(K, sv);
  const bool ok = francis(K, sv);
  if (!ok) {
    if (threadIdx.x == 0) { out->status = 1; out->p = 0; out->nconv = 0; }
    return;
  }
  split_real_pairs(K);

  // wanted set: the nkeep eigenvalues of largest real part (+1 to keep a pair together)
  __shared__ int bstart[KS_MAX], bsize[KS_MAX], bwant[KS_MAX], s_nb, s_p, s_fail;
  if (threadIdx.x == 0) {
    const int nb = blocks_of(K, bstart, bsize);
    double er[KS_MAX], ei[KS_MAX];
    int eb[KS_MAX], ne = 0;
    for (int b = 0; b < nb; b++) {
      double re[2], im[2];
      block_eigs(K, bstart[b], bsize[b], re, im);
      for (int e = 0; e < bsize[b]; e++) { er[ne] = re[e]; ei[ne] = im[e]; eb[ne] = b; ne++; }
      bwant[b] = 0;
    }
    // selection by repeated minimum search (n <= 64)
    int chosen[KS_MAX];
    for (int e = 0; e < ne; e++) chosen[e] = 0;
    int p = 0, lastc = -1;
    while (p < nkeep && p < ne) {
      int best = -1;
      for (int e = 0; e < ne; e++)
        if (!chosen[e] && (best < 0 || key_before(er[e], ei[e], e, er[best], ei[best], best)))
          best = e;
      chosen[best] = 1;
      lastc = best;
      p++;
    }
    if (lastc >= 0 && ei[lastc] != 0.0) {     // complete a split conjugate pair
      for (int e = 0; e < ne; e++)
        if (!chosen[e] && eb[e] == eb[lastc]) { chosen[e] = 1; p++; }
    }
    for (int e = 0; e < ne; e++)
      if (chosen[e]) bwant[eb[e]] = 1;
    s_nb = nb;
    s_p = p;
    s_fail = 0;
  }
  __syncthreads();
  // bubble the wanted blocks to the front
  for (int guard = 0; guard < 4 * KS_MAX * KS_MAX; guard++) {
    __shared__ int s_swap;
    if (threadIdx.x == 0) {
      s_swap = -1;
      for (int b = 0; b + 1 < s_nb; b++)
        if (!bwant[b] && bwant[b + 1]) { s_swap = b; break; }
    }
    __syncthreads();
    const int b = s_swap;
    if (b < 0) break;
    const bool good = swap_blocks(K, bstart[b], bsize[b], bsize[b + 1]);
    if (threadIdx.x == 0) {
      if (!good) s_fail = 1;
      const int s1 = bsize[b], s2 = bsize[b + 1];
      bsize[b] = s2;
      bsize[b + 1] = s1;
      bstart[b + 1] = bstart[b] + s2;
      const int w = bwant[b];
      bwant[b] = bwant[b + 1];
      bwant[b + 1] = w;
    }
    __syncthreads();
  }
  // b~ = b^T Z, b = H(n, 0:n)
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += H[n + (int64_t)i * ldh] * K.z(i, j);
    out->btil[j] = s;
  }
  __syncthreads();
  // Ritz values of the leading p x p block and their residuals |b~^T y| / ||y||
  if (threadIdx.x == 0) {
    const int p = s_p;
    int nbp = 0;
    int bs[KS_MAX], bz[KS_MAX];
    for (int j = 0; j < p;) {
      const int sz = (j + 1 < p && K.t(j + 1, j) != 0.0) ? 2 : 1;
      bs[nbp] = j; bz[nbp] = sz; nbp++; j += sz;
    }
    double er[KS_MAX], ei[KS_MAX], rs[KS_MAX];
    int ne = 0;
    for (int bb = 0; bb < nbp; bb++) {
      double re[2], im[2];
      block_eigs(K, bs[bb], bz[bb], re, im);
      // eigenvector for re[0] + i im[0] (complex back substitution), support 0..j_end
      const int j = bs[bb];
      const double lr = re[0], li = im[0];
      double yr[KS_MAX], yi[KS_MAX];
      int top;
      if (bz[bb] == 1) {
        yr[j] = 1.0; yi[j] = 0.0; top = j;
      } else {
        // (b, lambda - a) for the block [a b; c d]
        yr[j] = K.t(j, j + 1); yi[j] = 0.0;
        yr[j + 1] = lr - K.t(j, j); yi[j + 1] = li;
        top = j + 1;
      }
      int i = j - 1;
      while (i >= 0) {
        const bool two = (i >= 1 && K.t(i, i - 1) != 0.0);
        if (!two) {
          double sr = 0.0, si = 0.0;
          for (int l = i + 1; l <= top; l++) { sr += K.t(i, l) * yr[l]; si += K.t(i, l) * yi[l]; }
          // (T_ii - lambda) y_i = -s
          double dr = K.t(i, i) - lr, di = -li;
          if (fabs(dr) + fabs(di) < 1e-14 * (fabs(lr) + fabs(li) + 1e-300)) dr = 1e-14 * (fabs(lr) + 1.0);
          const double den = dr * dr + di * di;
          yr[i] = (-sr * dr - si * di) / den;
          yi[i] = (-si * dr + sr * di) / den;
          i -= 1;
        } else {
          // rows i-1, i with the 2x2 block; complex 2x2 solve by Cramer's rule
          double s1r = 0.0, s1i = 0.0, s2r = 0.0, s2i = 0.0;
          for (int l = i + 1; l <= top; l++) {
            s1r += K.t(i - 1, l) * yr[l]; s1i += K.t(i - 1, l) * yi[l];
            s2r += K.t(i, l) * yr[l]; s2i += K.t(i, l) * yi[l];
          }
          const double ar = K.t(i - 1, i - 1) - lr, ai = -li, b2 = K.t(i - 1, i);
          const double c2 = K.t(i, i - 1), dr = K.t(i, i) - lr, di = -li;
          // det = (a)(d) - b c
          const double detr = ar * dr - ai * di - b2 * c2, deti = ar * di + ai * dr;
          const double den = detr * detr + deti * deti + 1e-300;
          // x1 = (-s1 d + b s2)/det, x2 = (-a s2 + c s1)/det
          const double n1r = -(s1r * dr - s1i * di) + b2 * s2r, n1i = -(s1r * di + s1i * dr) + b2 * s2i;
          const double n2r = -(ar * s2r - ai * s2i) + c2 * s1r, n2i = -(ar * s2i + ai * s2r) + c2 * s1i;
          yr[i - 1] = (n1r * detr + n1i * deti) / den; yi[i - 1] = (n1i * detr - n1r * deti) / den;
          yr[i] = (n2r * detr + n2i * deti) / den; yi[i] = (n2i * detr - n2r * deti) / den;
          i -= 2;
        }
      }
      double nr2 = 0.0, pr = 0.0, pi = 0.0;
      for (int l = 0; l <= top; l++) {
        nr2 += yr[l] * yr[l] + yi[l] * yi[l];
        pr += out->btil[l] * yr[l];
        pi += out->btil[l] * yi[l];
      }
      const double res = sqrt(pr * pr + pi * pi) / sqrt(nr2);
      for (int e = 0; e < bz[bb]; e++) { er[ne] = re[e]; ei[ne] = im[e]; rs[ne] = res; ne++; }
    }
    // sort the p Ritz values (largest real part first, then larger imaginary part)
    int used[KS_MAX];
    for (int e = 0; e < ne; e++) used[e] = 0;
    int nconv = 0;
    for (int o = 0; o < ne; o++) {
      int best = -1;
      for (int e = 0; e < ne; e++)
        if (!used[e] && (best < 0 || key_before(er[e], ei[e], e, er[best], ei[best], best))) best = e;
      used[best] = 1;
      out->eig_re[o] = er[best];
      out->eig_im[o] = ei[best];
      out->resid[o] = rs[best];
      if (o < nev && rs[best] <= tol * hypot(er[best], ei[best])) nconv++;
    }
    out->p = p;
    out->nconv = nconv;
    out->status = s_fail ? 2 : 0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    Tout[i + (int64_t)j * n] = K.T[idx];
    Zout[i + (int64_t)j * n] = K.Z[idx];
  }
}

// Qnew(:, j) = Q(:, 0:n) Z(:, j) for j < p; Qnew(:, p) = Q(:, n)
__global__ void __launch_bounds__(256) k_ks_truncate(const double* __restrict__ Q, int64_t ldq,
                                                     int n, int p, const double* __restrict__ Z,
                                                     double* __restrict__ Qn, int64_t m) {
  __shared__ double zs[KS_MAX * KS_MAX];
  for (int idx = threadIdx.x; idx < n * p; idx += blockDim.x) zs[idx] = Z[idx];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    double qrow[KS_MAX];
    for (int i = 0; i < n; i++) qrow[i] = Q[r + (int64_t)i * ldq];
    for (int j = 0; j < p; j++) {
      double s = 0.0;
      for (int i = 0; i < n; i++) s += qrow[i] * zs[i + j * n];
      Qn[r + (int64_t)j * ldq] = s;
    }
    Qn[r + (int64_t)p * ldq] = Q[r + (int64_t)n * ldq];
  }
}

// H <- [T_pp; b~_p] (zero elsewhere), K(0:p+1, p) = S (the restart projection)
__global__ void k_ks_newH(double* __restrict__ H, int ldh, double* __restrict__ Kc, int ldk,
                          int ncols, const double* __restrict__ T, int n, int p,
                          const KsOut* __restrict__ out) {
  for (int idx = threadIdx.x; idx < ldh * ncols; idx += blockDim.x) {
    const int i = idx % ldh, j = idx / ldh;
    double v = 0.0;
    if (j < p && i < p) v = T[i + (int64_t)j * n];
    else if (j < p && i == p) v = out->btil[j];
    H[idx] = v;
    Kc[(int64_t)i + (int64_t)j * ldk] = 0.0;
  }
}

__global__ void k_ks_setK(double* __restrict__ Kc, int ldk, int p, const Scalars* __restrict__ sc) {
  for (int i = threadIdx.x; i <= p; i += blockDim.x) Kc[i + (int64_t)p * ldk] = sc->S[i];
}

}  // namespace kc

using namespace kc;

extern "C" kc_status krylov_schur_eigs(kc_ctx* ctx, const kc_csr* A, const double* v0,
                                       const kc_ks_opts* opts, double* eig_re, double* eig_im,
                                       double* resid, int* nconv, int* restarts, int* matvecs) {
  if (!ctx) return KC_ERR_INVALID_ARG;
  kc_status s = validate_csr(ctx, A);
  if (s != KC_OK) return s;
  if (!v0 || !opts || !eig_re || !eig_im || !resid)
    return fail(ctx, KC_ERR_INVALID_ARG, "NULL argument");
  if (A->val_dtype != KC_F64) return fail(ctx, KC_ERR_INVALID_ARG, "A must have FP64 values");
  const int n = opts->ncv, nkeep = opts->nkeep, nev = opts->nev;
  if (n < 3 || n > KS_MAX || nkeep < 1 || nkeep + 2 > n || nev < 1 || nev > nkeep)
    return fail(ctx, KC_ERR_INVALID_ARG,
                "need 1 <= nev <= nkeep, nkeep + 2 <= ncv <= %d", KS_MAX);
  if ((uintptr_t)v0 & 15) return fail(ctx, KC_ERR_INVALID_ARG, "v0 must be 16-byte aligned");
  const int64_t m = A->m;
  if (m <= n) return fail(ctx, KC_ERR_INVALID_ARG, "matrix too small for ncv = %d", n);
  const int64_t ldq = (m + 31) / 32 * 32;
  const int ncap = n + 1;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t off = 0;
  const size_t oQ0 = off; off = al(off + (size_t)ncap * ldq * 8);
  const size_t oQ1 = off; off = al(off + (size_t)ncap * ldq * 8);
  const size_t ow = off; off = al(off + (size_t)ldq * 8);
  const size_t ov = off; off = al(off + (size_t)ldq * 8);
  const size_t oH = off; off = al(off + (size_t)ncap * n * 8);
  const size_t oK = off; off = al(off + (size_t)ncap * n * 8);
  const size_t oT = off; off = al(off + (size_t)n * n * 8);
  const size_t oZ = off; off = al(off + (size_t)n * n * 8);
  const size_t oO = off; off = al(off + sizeof(KsOut));
  if ((s = ensure_workspace(ctx, off)) != KC_OK) return s;
  char* ws = (char*)ctx->ws;
  double* Qa = (double*)(ws + oQ0);
  double* Qb = (double*)(ws + oQ1);
  double* w = (double*)(ws + ow);
  double* v = (double*)(ws + ov);
  double* H = (double*)(ws + oH);
  double* Kc = (double*)(ws + oK);
  double* T = (double*)(ws + oT);
  double* Z = (double*)(ws + oZ);
  KsOut* out = (KsOut*)(ws + oO);
  KsOut hout;
  const size_t smem = (size_t)(2 * n * n + KS_MAX + 8) * sizeof(double);
  KC_CUDA(ctx, cudaFuncSetAttribute(k_ks_schur, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  KC_CUDA(ctx, cudaMemsetAsync(H, 0, (size_t)ncap * n * 8, ctx->stream));
  KC_CUDA(ctx, cudaMemsetAsync(Kc, 0, (size_t)ncap * n * 8, ctx->stream));
  KC_CUDA(ctx, cudaMemcpyAsync(w, v0, m * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  StepArgs sa = {};
  sa.H = H;
  sa.ldh = ncap;
  sa.K = Kc;
  sa.ldk = ncap;
  sa.pyth_tol = 0.0;
  int mv = 0, rs = 0, k0 = 0;
  kc_status result = KC_ERR_NOT_CONVERGED;
  for (;;) {
    // expand k0 .. n-1 with DCGS2 steps, then the CGS2 finish (column n)
    for (int k = k0; k < n; k++) {
      sa.k = k;
      if ((s = launch_matvec_reduce(ctx, A, Qa, ldq, KC_F64, k, w, v, m, KC_F64, sa)) != KC_OK)
        return s;
      if ((s = launch_dcgs2_update(ctx, Qa, ldq, KC_F64, k, w, v, m, KC_F64)) != KC_OK) return s;
      mv++;
    }
    sa.k = n;
    if ((s = launch_reduce(ctx, Qa, ldq, KC_F64, n, w, nullptr, m, KC_F64, EPI_STORE_C1, sa)) != KC_OK) return s;
    if ((s = launch_proj_reduce(ctx, Qa, ldq, KC_F64, n, w, m, KC_F64, sa)) != KC_OK) return s;
    if ((s = launch_gemv_sub(ctx, Qa, ldq, KC_F64, n, w, m, KC_F64, 1)) != KC_OK) return s;
    if ((s = launch_norm(ctx, w, nullptr, m, KC_F64, NEPI_FINISH, sa)) != KC_OK) return s;
    if ((s = launch_scale_to(ctx, w, Qa + (size_t)n * ldq, KC_F64, m, KC_F64)) != KC_OK) return s;
    // dense Schur step on the GPU
    timing_begin(ctx, KID_SMALL);
    k_ks_schur<<<1, KS_THREADS, smem, ctx->stream>>>(H, ncap, n, nkeep, nev, opts->tol, T, Z, out);
    KC_LAUNCHED(ctx);
    KC_CUDA(ctx, cudaMemcpyAsync(&hout, out, sizeof(KsOut), cudaMemcpyDeviceToHost, ctx->stream));
    KC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hout.status == 1) return fail(ctx, KC_ERR_NOT_CONVERGED, "Schur QR iteration did not converge");
    if (hout.status == 2) return fail(ctx, KC_ERR_NOT_CONVERGED, "Schur reordering was unstable");
    if (hout.nconv >= nev) { result = KC_OK; break; }
    if (rs >= opts->maxrestarts) break;
    // truncate to p columns plus q_n, then one projection of A q_p
    const int p = hout.p;
    timing_begin(ctx, KID_OTHER);
    {
      int64_t b = (m + 255) / 256, cap = (int64_t)ctx->num_sms * 8;
      k_ks_truncate<<<(int)(b > cap ? cap : b), 256, 0, ctx->stream>>>(Qa, ldq, n, p, Z, Qb, m);
    }
    KC_LAUNCHED(ctx);
    double* t = Qa; Qa = Qb; Qb = t;
    timing_begin(ctx, KID_SMALL);
    k_ks_newH<<<1, 256, 0, ctx->stream>>>(H, ncap, Kc, ncap, n, T, n, p, out);
    KC_LAUNCHED(ctx);
    if ((s = launch_spmv(ctx, A, Qa + (size_t)p * ldq, w, KC_F64)) != KC_OK) return s;
    sa.k = p + 1;
    if ((s = launch_reduce(ctx, Qa, ldq, KC_F64, p + 1, w, nullptr, m, KC_F64, EPI_STORE_S, sa)) != KC_OK) return s;
    if ((s = launch_gemv_sub(ctx, Qa, ldq, KC_F64, p + 1, w, m, KC_F64, 2)) != KC_OK) return s;
    timing_begin(ctx, KID_SMALL);
    k_ks_setK<<<1, 128, 0, ctx->stream>>>(Kc, ncap, p, ctx->scal);
    KC_LAUNCHED(ctx);
    mv++;
    k0 = p + 1;
    rs++;
  }
  for (int i = 0; i < nev; i++) {
    eig_re[i] = hout.eig_re[i];
    eig_im[i] = hout.eig_im[i];
    resid[i] = hout.resid[i];
  }
  if (nconv) *nconv = hout.nconv;
  if (restarts) *restarts = rs;
  if (matvecs) *matvecs = mv;
  if (result != KC_OK)
    fail(ctx, result, "krylov_schur_eigs: %d of %d converged after %d restarts", hout.nconv, nev, rs);
  return result;
}
