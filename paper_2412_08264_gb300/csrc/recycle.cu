// Recycle-space refresh (Section 3): Ritz, harmonic Ritz and Ritz generalized singular vectors.
//
// For every listed pair with W = [U^(i-1), V^(i-1)] (t = s + k columns):
//   1. G = W^T W; W~ = W D P R^{-1} from the pivoted Cholesky factor of the column-scaled Gram,
//      leaving out columns within a relative threshold of the span of those kept (an
//      orthonormal basis of the numerical range of W).  W~ is
//      formed explicitly: projecting W^T H W with the coefficients instead would square their
//      conditioning in the projected matrices.
//   2. HW~ = H W~ (t' Hessian actions at the current point: the outer form, eq. (3.3)).
//   3. T = W~^T H W~; for Ritz-GSV also J~ = J W~ (eq. (3.4)), for harmonic Ritz (HW~)^T HW~.
//   4. Small FP64 problem on one CTA per pair:
//        Ritz (eq. (3.1))      eigh(T), select smallest / largest / both;
//        harmonic (eq. (3.2))  (HW~)^T HW~ rho = theta T rho via Cholesky of T;
//        RGSV (Thm 3.1, eq. (3.4))  mu, V_H = singular values and right singular vectors of J~ T^{-1}
//        (Householder QR of J~ T^{-1}, then one-sided Jacobi on its triangular factor: the squared
//        matrix is never formed), X = T^{-1} V_H D_H, D_H = diag(1 / sqrt(1 + mu^2)); Z = W~ V_H diag(mu).
//   5. U~ = W~ Y, C~ = HW~ Y (no new Hessian actions), then C~ = C R by CholeskyQR (twice),
//      U = U~ R^{-1}, so that C = H U and C^T C = I (Section 2.2.2); Z^T C for the estimate.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "device.cuh"

namespace bl {

// ---------------------------------------------------------------------------------------------
// Small dense FP64 linear algebra, one CTA per pair.

// Parallel cyclic Jacobi (round-robin pairing) on symmetric n x n A (ld n), eigenvectors in V.
// On return A's diagonal holds the eigenvalues; w (ascending) and V's columns are sorted.
__device__ void dev_jacobi(double* A, double* V, int n, double* w, double* cs, int* perm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  __syncthreads();
  if (n <= 1) {
    if (tid == 0 && n == 1) { w[0] = A[0]; perm[0] = 0; }
    __syncthreads();
    return;
  }
  const int m = n + (n & 1);
  __shared__ double offs, dias;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (tid == 0) { offs = 0.0; dias = 0.0; }
    __syncthreads();
    double lo = 0.0, ld = 0.0;
    for (int idx = tid; idx < n * n; idx += nt) {
      const int i = idx / n, j = idx - (idx / n) * n;
      if (i == j) ld += A[idx] * A[idx];
      else lo += A[idx] * A[idx];
    }
    lo = warp_sum(lo);
    ld = warp_sum(ld);
    if ((tid & 31) == 0) { atomicAdd(&offs, lo); atomicAdd(&dias, ld); }
    __syncthreads();
    // converged when the off-diagonal mass is below (1e-12)^2 of the diagonal's: a few ulps of
    // FP64 per entry for t <= 96 (a stricter bound is never reached through rounding)
    const bool done = !(offs > 1e-24 * dias) || offs == 0.0;
    __syncthreads();
    if (done) break;
    for (int rnd = 0; rnd < m - 1; ++rnd) {
      // rotation parameters for the m/2 disjoint pairs of this round
      for (int i = tid; i < m / 2; i += nt) {
        int p, q;
        if (i == 0) { p = rnd; q = m - 1; }
        else { p = (rnd + i) % (m - 1); q = (rnd - i + m - 1) % (m - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * n + q];
          if (fabs(apq) > 1e-300) {
            const double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[4 * i] = c; cs[4 * i + 1] = s; cs[4 * i + 2] = p; cs[4 * i + 3] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = tid; idx < (m / 2) * n; idx += nt) {
        const int i = idx / n, j = idx - (idx / n) * n;
        const int p = (int)cs[4 * i + 2], q = (int)cs[4 * i + 3];
        if (q >= n) continue;
        const double c = cs[4 * i], s = cs[4 * i + 1];
        const double ap = A[p * n + j], aq = A[q * n + j];
        A[p * n + j] = c * ap - s * aq;
        A[q * n + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J.  Consecutive threads take consecutive rotation pairs of one
      // row j, so a warp touches one row at scattered columns (a column walk with stride n
      // would put every lane of the warp in the same shared-memory bank).
      const int hp = m / 2;
      for (int idx = tid; idx < hp * n; idx += nt) {
        const int j = idx / hp, i = idx - (idx / hp) * hp;
        const int p = (int)cs[4 * i + 2], q = (int)cs[4 * i + 3];
        if (q >= n) continue;
        const double c = cs[4 * i], s = cs[4 * i + 1];
        const double ap = A[j * n + p], aq = A[j * n + q];
        A[j * n + p] = c * ap - s * aq;
        A[j * n + q] = s * ap + c * aq;
        const double vp = V[j * n + p], vq = V[j * n + q];
        V[j * n + p] = c * vp - s * vq;
        V[j * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // sort ascending (ties by index)
  if (tid == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = 1; i < n; ++i) {
      const int pi = perm[i];
      const double v = A[pi * n + pi];
      int j = i - 1;
      while (j >= 0 && A[perm[j] * n + perm[j]] > v) { perm[j + 1] = perm[j]; --j; }
      perm[j + 1] = pi;
    }
    for (int i = 0; i < n; ++i) w[i] = A[perm[i] * n + perm[i]];
  }
  __syncthreads();
}

// In-place lower Cholesky of SPD n x n A (ld lda); returns false (in every thread) if not SPD.
__device__ bool dev_cholesky(double* A, int n, int lda) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j * lda + j];
      for (int k = 0; k < j; ++k) d -= A[j * lda + k] * A[j * lda + k];
      if (!(d > 0.0)) { ok = 0; d = 1.0; }
      A[j * lda + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double v = A[i * lda + j];
      for (int k = 0; k < j; ++k) v -= A[i * lda + k] * A[j * lda + k];
      A[i * lda + j] = v / A[j * lda + j];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - (idx / n) * n;
    if (j > i) A[i * lda + j] = 0.0;
  }
  __syncthreads();
  return ok != 0;
}

// Solve L L^T X = B in place (L lower, ld lda; B n x nrhs, ld ldb), one thread per column.
__device__ void dev_chol_solve(const double* L, int n, int lda, double* B, int nrhs, int ldb) {
  for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double v = B[i * ldb + c];
      for (int k = 0; k < i; ++k) v -= L[i * lda + k] * B[k * ldb + c];
      B[i * ldb + c] = v / L[i * lda + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = B[i * ldb + c];
      for (int k = i + 1; k < n; ++k) v -= L[k * lda + i] * B[k * ldb + c];
      B[i * ldb + c] = v / L[i * lda + i];
    }
  }
  __syncthreads();
}

// Indices selected from ascending values: smallest s, largest s, or both halves (Table 1).
__device__ __forceinline__ int sel_index(int n, int s, int which, int j) {
  if (which == BL_SIZE_SMALL) return j;
  if (which == BL_SIZE_LARGE) return n - s + j;
  const int lo = s - s / 2;
  return j < lo ? j : n - (s - j);
}

struct DenseArgs {
  int TM, p;
  double* G;     // K x TM x TM: W^T W   -> scratch
  double* T;     // K x TM x TM: W~^T H W~
  double* GH;    // K x TM x TM: (HW~)^T HW~
  const double* J;  // K x jcols x p: J W~ ([k][col][m])
  int jcols;
  double* Y;     // K x TM x TM: coefficient outputs
  double* Y2;    // K x TM x TM
  double* scratch;  // K x 4 x TM x TM
  int* tk;       // reduced basis size per pair (in/out)
  int* snew;     // selected size per pair (out)
  const int* mask;
  int kind, size, side, s;
  double drop;   // relative pivot threshold of the orthonormalisation
};

// 1. G (t x t) -> B1 (t x t'): orthonormal-basis coefficients.  Pivoted Cholesky of the
// column-scaled Gram D G D = P R^T R P^T, stopped when the largest remaining pivot falls below
// `drop` (the columns left out lie within sqrt(drop) of the span of those kept); then
// B1 = D P R^{-1}, so W~ = W B1 has W~^T W~ = I over the kept columns and spans them.
__global__ void k_dense_orth(DenseArgs a, const int* tcols) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = blockIdx.x;
  if (!a.mask[k]) return;
  const int t = tcols[k], TM = a.TM;
  double* As = reinterpret_cast<double*>(smem_raw);   // t x t scaled Gram, updated in place
  double* Rs = As + TM * TM;                          // factor rows; row j indexed by original column
  double* dsc = Rs + TM * TM;
  double* dres = dsc + TM;                            // remaining pivots
  int* piv = reinterpret_cast<int*>(dres + TM);
  __shared__ int s_stop, s_tk;
  const double* G = a.G + (size_t)k * TM * TM;
  for (int i = threadIdx.x; i < t; i += blockDim.x) {
    const double d = G[i * TM + i];
    dsc[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    piv[i] = i;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
    const int i = idx / t, j = idx - (idx / t) * t;
    As[idx] = 0.5 * (G[i * TM + j] + G[j * TM + i]) * dsc[i] * dsc[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < t; i += blockDim.x) dres[i] = As[i * t + i];
  if (threadIdx.x == 0) s_tk = t;
  __syncthreads();
  for (int j = 0; j < t; ++j) {
    if (threadIdx.x == 0) {
      int p = j;
      for (int i = j + 1; i < t; ++i)
        if (dres[piv[i]] > dres[piv[p]]) p = i;
      s_stop = !(dres[piv[p]] > a.drop);   // unit diagonal: the threshold is relative
      if (!s_stop) {
        const int tmp = piv[j];
        piv[j] = piv[p];
        piv[p] = tmp;
      } else {
        s_tk = j;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int pj = piv[j];
    const double rjj = sqrt(dres[pj]);
    // row j of R over the remaining columns, from the updated Schur complement.  Entries are kept
    // under the original column index: later pivot swaps reorder positions, not columns.
    for (int i = j + threadIdx.x; i < t; i += blockDim.x) {
      const int pi = piv[i];
      Rs[j * TM + pi] = (i == j) ? rjj : As[pj * t + pi] / rjj;
    }
    __syncthreads();
    // trailing update A[pi][pl] -= R[j][pi] R[j][pl] over the columns still to be pivoted
    const int m = t - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int pi = piv[j + 1 + idx / m], pl = piv[j + 1 + idx % m];
      As[pi * t + pl] -= Rs[j * TM + pi] * Rs[j * TM + pl];
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < t; i += blockDim.x) dres[piv[i]] = As[piv[i] * t + piv[i]];
    __syncthreads();
  }
  const int tk = s_tk;
  if (threadIdx.x == 0) a.tk[k] = tk;
  // B1 = D P R^{-1}: column c solves R x = e_c (upper triangular), row piv[i] of B1 gets x_i
  double* Y = a.Y + (size_t)k * TM * TM;   // t x t'
  for (int idx = threadIdx.x; idx < t * tk; idx += blockDim.x) Y[(idx / tk) * TM + idx % tk] = 0.0;
  __syncthreads();
  // in pivoted order R_pos[i][l] = Rs[i][piv[l]] (upper triangular over the kept columns)
  for (int c = threadIdx.x; c < tk; c += blockDim.x) {
    double x[kMaxTM];
    for (int i = c + 1; i < tk; ++i) x[i] = 0.0;
    for (int i = c; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) v -= Rs[i * TM + piv[l]] * x[l];
      x[i] = v / Rs[i * TM + piv[i]];
    }
    for (int i = 0; i <= c; ++i) Y[piv[i] * TM + c] = dsc[piv[i]] * x[i];
  }
}

// 2. selection: Y (t' x s) recycle coefficients, Y2 (t' x s) NSC coefficients
__global__ void k_dense_select(DenseArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = blockIdx.x;
  if (!a.mask[k]) return;
  const int TM = a.TM, t = a.tk[k];
  double* As = reinterpret_cast<double*>(smem_raw);
  double* Vs = As + TM * TM;
  double* w = Vs + TM * TM;
  double* cs = w + TM;
  int* perm = reinterpret_cast<int*>(cs + 2 * TM + 4);
  double* T = a.T + (size_t)k * TM * TM;
  double* Y = a.Y + (size_t)k * TM * TM;
  double* Y2 = a.Y2 + (size_t)k * TM * TM;
  double* S1 = a.scratch + (size_t)k * 4 * TM * TM;   // t x t scratch
  double* S2 = S1 + TM * TM;
  __shared__ int s_sel;
  if (threadIdx.x == 0) {
    int s = min(a.s, t);
    if (a.kind == BL_RECYCLE_RGSV) s = min(s, a.p);
    s_sel = s;
    a.snew[k] = s;
  }
  // symmetrise T
  for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
    const int i = idx / t, j = idx - (idx / t) * t;
    S1[i * TM + j] = 0.5 * (T[i * TM + j] + T[j * TM + i]);
  }
  __syncthreads();
  const int s = s_sel;
  if (s == 0) return;
  if (a.kind == BL_RECYCLE_RITZ) {
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) As[idx] = S1[(idx / t) * TM + idx % t];
    __syncthreads();
    dev_jacobi(As, Vs, t, w, cs, perm);
    for (int idx = threadIdx.x; idx < t * s; idx += blockDim.x) {
      const int i = idx / s, j = idx - (idx / s) * s;
      Y[i * TM + j] = Vs[i * t + perm[sel_index(t, s, a.size, j)]];
    }
    return;
  }
  // Cholesky of T in S1 (lower)
  const bool ok = dev_cholesky(S1, t, TM);
  if (!ok) {
    if (threadIdx.x == 0) a.snew[k] = -1;   // not SPD: reported as breakdown by the host
    return;
  }
  if (a.kind == BL_RECYCLE_HRITZ) {
    // M = L^{-1} GH L^{-T}: solve with columns, then rows
    const double* GH = a.GH + (size_t)k * TM * TM;
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
      const int i = idx / t, j = idx - (idx / t) * t;
      S2[i * TM + j] = 0.5 * (GH[i * TM + j] + GH[j * TM + i]);
    }
    __syncthreads();
    // forward solve L X = GH (columns), then L M^T = X^T
    for (int pass = 0; pass < 2; ++pass) {
      for (int c = threadIdx.x; c < t; c += blockDim.x)
        for (int i = 0; i < t; ++i) {
          double v = S2[i * TM + c];
          for (int kk = 0; kk < i; ++kk) v -= S1[i * TM + kk] * S2[kk * TM + c];
          S2[i * TM + c] = v / S1[i * TM + i];
        }
      __syncthreads();
      // transpose S2 in place
      for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
        const int i = idx / t, j = idx - (idx / t) * t;
        if (i < j) { const double x = S2[i * TM + j]; S2[i * TM + j] = S2[j * TM + i]; S2[j * TM + i] = x; }
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
      const int i = idx / t, j = idx - (idx / t) * t;
      As[idx] = 0.5 * (S2[i * TM + j] + S2[j * TM + i]);
    }
    __syncthreads();
    dev_jacobi(As, Vs, t, w, cs, perm);
    // rho = L^{-T} y for the selected eigenvectors
    for (int idx = threadIdx.x; idx < t * s; idx += blockDim.x) {
      const int i = idx / s, j = idx - (idx / s) * s;
      Y[i * TM + j] = Vs[i * t + perm[sel_index(t, s, a.size, j)]];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < s; c += blockDim.x)
      for (int i = t - 1; i >= 0; --i) {
        double v = Y[i * TM + c];
        for (int kk = i + 1; kk < t; ++kk) v -= S1[kk * TM + i] * Y[kk * TM + c];
        Y[i * TM + c] = v / S1[i * TM + i];
      }
    return;
  }
  // RGSV (Theorem 3.1): the singular values mu and right singular vectors V_H of B = J~ T^{-1},
  // computed without forming B^T B (which would square the conditioning and lose the small mu):
  //   B^T = T^{-1} J~^T by two triangular solves with the Cholesky factor (in place in J's storage);
  //   p >= t: B P = Q R by Householder QR with column pivoting (largest remaining column first, Q
  //     not kept), then one-sided Jacobi on the columns of M = R^T: M W = [mu_1 u_1, ...] with
  //     R = W diag(mu) U^T, so V_H = P U, u_l = (column l of M W) / mu_l.  The pivoted factor's rows
  //     are graded, which is what makes Jacobi on R^T converge in a few sweeps (Drmac and Veselic's
  //     preconditioned one-sided Jacobi) where Jacobi on R itself first spends ~10 sweeps sorting;
  //   p < t (rank <= p, the other t - p values are mu = 0): Householder QR without pivoting, then
  //     one-sided Jacobi on the columns of R (p long) accumulating V_H: R V_H = [mu_1 q_1, ...].
  double* Bt = const_cast<double*>(a.J) + (size_t)k * a.jcols * a.p;   // t x p, row j = column j of B
  const int p = a.p;
  dev_chol_solve(S1, t, TM, Bt, p, p);            // rows of Bt: T^{-1} J~^T
  const bool tall = p >= t;
  const int r = min(p, t);                        // rows of R
  // tall: Rb holds M = R^T column-major (column i = row i of R, t long, at Rb[i * t]);
  // otherwise Rb holds R column-major (column l, r long, at Rb[l * r])
  double* Rb = As;
  double* Vh = Vs;                                // V_H, column-major: column l at Vh[l * t]
  double* nrm = cs + TM;                          // squared norms of the unreduced parts of the columns
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double s_alpha, s_beta;
  __shared__ int s_piv;
  for (int idx = threadIdx.x; idx < r * t; idx += blockDim.x) Rb[idx] = 0.0;
  for (int l = threadIdx.x; l < t; l += blockDim.x) perm[l] = l;   // P: column l of B P is column perm[l] of B
  if (tall)
    for (int l = wid; l < t; l += nw) {
      const double* y = Bt + (size_t)l * p;
      double ss = 0.0;
      for (int m = lane; m < p; m += 32) ss += y[m] * y[m];
      ss = warp_sum(ss);
      if (lane == 0) nrm[l] = ss;
    }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tall) {
      // pivot: the remaining column with the largest unreduced norm (ties to the lowest index)
      if (threadIdx.x == 0) {
        int best = j;
        for (int l = j + 1; l < t; ++l)
          if (nrm[l] > nrm[best]) best = l;
        s_piv = best;
      }
      __syncthreads();
      const int q = s_piv;
      if (q != j) {
        double* xj = Bt + (size_t)j * p;
        double* xq = Bt + (size_t)q * p;
        for (int m = threadIdx.x; m < p; m += blockDim.x) { const double u = xj[m]; xj[m] = xq[m]; xq[m] = u; }
        for (int i = threadIdx.x; i < j; i += blockDim.x) {   // rows 0..j-1 of R already hold these columns
          const double u = Rb[i * t + j]; Rb[i * t + j] = Rb[i * t + q]; Rb[i * t + q] = u;
        }
        if (threadIdx.x == 0) {
          const double u = nrm[j]; nrm[j] = nrm[q]; nrm[q] = u;
          const int pi = perm[j]; perm[j] = perm[q]; perm[q] = pi;
        }
      }
      __syncthreads();
    }
    double* x = Bt + (size_t)j * p;               // column j of B (P)
    if (wid == 0) {
      double ss = 0.0;
      for (int m = j + lane; m < p; m += 32) ss += x[m] * x[m];
      ss = warp_sum(ss);
      if (lane == 0) {
        const double sg = sqrt(ss), x0 = x[j];
        const double al = x0 >= 0.0 ? -sg : sg;   // R[j][j]
        s_alpha = al;
        s_beta = sg > 0.0 ? 1.0 / (sg * (sg + fabs(x0))) : 0.0;   // 2 / v^T v with v = x - al e_j
        x[j] = x0 - al;
      }
    }
    __syncthreads();
    const double be = s_beta;
    if (threadIdx.x == 0) Rb[tall ? j * t + j : j * r + j] = s_alpha;
    // apply (I - be v v^T) to the columns l > j; warp per column; the unreduced norm is recomputed
    for (int l = j + 1 + wid; l < t; l += nw) {
      double* y = Bt + (size_t)l * p;
      double d = 0.0;
      for (int m = j + lane; m < p; m += 32) d += x[m] * y[m];
      d = warp_sum(d) * be;
      double ss = 0.0;
      for (int m = j + lane; m < p; m += 32) {
        const double v = y[m] - d * x[m];
        y[m] = v;
        if (m > j) ss += v * v;
      }
      ss = warp_sum(ss);
      __syncwarp();
      if (lane == 0) {
        nrm[l] = ss;
        if (tall) Rb[j * t + l] = y[j];
        else Rb[l * r + j] = y[j];
      }
    }
    __syncthreads();
  }
  // one-sided Jacobi (round-robin pairs; one warp per pair) on the n columns (each len long) of Rb,
  // rotating V_H alongside unless tall: until every pair is orthogonal to 1e-12 relative, at most
  // 30 sweeps (pairs still rotating then sit at the rounding floor of columns whose norms differ by
  // many orders)
  const int n = tall ? r : t, len = tall ? t : r;
  if (!tall)
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) Vh[idx] = (idx / t == idx % t) ? 1.0 : 0.0;
  __shared__ int s_rot;
  const int mm = n + (n & 1);
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < mm - 1; ++rnd) {
      for (int i = wid; i < mm / 2; i += nw) {
        int pp, qq;
        if (i == 0) { pp = rnd; qq = mm - 1; }
        else { pp = (rnd + i) % (mm - 1); qq = (rnd - i + mm - 1) % (mm - 1); }
        if (pp > qq) { const int tt = pp; pp = qq; qq = tt; }
        if (qq >= n) continue;
        double* cp = Rb + pp * len;
        double* cq = Rb + qq * len;
        double al = 0.0, bb = 0.0, ga = 0.0;
        for (int m = lane; m < len; m += 32) {
          al += cp[m] * cp[m];
          bb += cq[m] * cq[m];
          ga += cp[m] * cq[m];
        }
        al = warp_sum(al);
        bb = warp_sum(bb);
        ga = warp_sum(ga);
        if (!(fabs(ga) > 1e-12 * sqrt(al * bb)) || ga == 0.0) continue;
        const double ze = (bb - al) / (2.0 * ga);
        const double tn = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1.0 + ze * ze));
        const double c = 1.0 / sqrt(1.0 + tn * tn), sn = c * tn;
        for (int m = lane; m < len; m += 32) {
          const double u = cp[m], v = cq[m];
          cp[m] = c * u - sn * v;
          cq[m] = sn * u + c * v;
        }
        if (!tall) {
          double* vp = Vh + pp * t;
          double* vq = Vh + qq * t;
          for (int m = lane; m < t; m += 32) {
            const double u = vp[m], v = vq[m];
            vp[m] = c * u - sn * v;
            vq[m] = sn * u + c * v;
          }
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  // mu_l = ||column l of Rb||; tall: V_H column l = P (column l / mu_l) (e_{P l} for mu_l = 0, which
  // needs J~ rank-deficient with p >= t)
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double ss = 0.0;
    for (int m = 0; m < len; ++m) ss += Rb[l * len + m] * Rb[l * len + m];
    cs[l] = sqrt(ss);
  }
  __syncthreads();
  if (tall)
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
      const int l = idx / t, m = idx - (idx / t) * t;
      const double mu = cs[l];
      Vh[l * t + perm[m]] = mu > 0.0 ? Rb[l * t + m] / mu : (m == l ? 1.0 : 0.0);
    }
  __syncthreads();
  // sorted ascending (ties by index) into w / perm
  if (threadIdx.x == 0) {
    for (int i = 0; i < t; ++i) perm[i] = i;
    for (int i = 1; i < t; ++i) {
      const int pi = perm[i];
      const double v = cs[pi];
      int j = i - 1;
      while (j >= 0 && cs[perm[j]] > v) { perm[j + 1] = perm[j]; --j; }
      perm[j + 1] = pi;
    }
    for (int i = 0; i < t; ++i) w[i] = cs[perm[i]];
  }
  __syncthreads();
  // V_H,sel into Y2 (scaled by mu below), X_sel = T^{-1} V_H,sel D_H into Y
  for (int idx = threadIdx.x; idx < t * s; idx += blockDim.x) {
    const int i = idx / s, j = idx - (idx / s) * s;
    const int e = sel_index(t, s, a.size, j);
    const double vh = Vh[perm[e] * t + i];
    Y2[i * TM + j] = vh;
    Y[i * TM + j] = vh;
  }
  __syncthreads();
  dev_chol_solve(S1, t, TM, Y, s, TM);         // Y = T^{-1} V_H,sel
  for (int idx = threadIdx.x; idx < t * s; idx += blockDim.x) {
    const int i = idx / s, j = idx - (idx / s) * s;
    const int e = sel_index(t, s, a.size, j);
    const double mu = w[e];
    const double dh = 1.0 / sqrt(1.0 + mu * mu);
    const double x = Y[i * TM + j] * dh;
    const double vh = Y2[i * TM + j];
    if (a.side == BL_SIDE_RIGHT) Y[i * TM + j] = x;
    else if (a.side == BL_SIDE_LEFT) Y[i * TM + j] = vh;
    else Y[i * TM + j] = 0.5 * (vh + x);
    Y2[i * TM + j] = vh * mu;
  }
}

// 3. CholeskyQR step: S = C~^T C~ (s x s) -> Rinv (upper inverse of the Cholesky factor R^T = L)
__global__ void k_dense_cholinv(DenseArgs a, const int* scols, double* G, double* Rinv) {
  const int k = blockIdx.x;
  if (!a.mask[k]) return;
  const int TM = a.TM, s = scols[k];
  if (s <= 0) return;
  double* S = G + (size_t)k * TM * TM;
  double* R = Rinv + (size_t)k * TM * TM;
  for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int i = idx / s, j = idx - (idx / s) * s;
    if (i < j) { const double v = 0.5 * (S[i * TM + j] + S[j * TM + i]); S[i * TM + j] = v; S[j * TM + i] = v; }
  }
  __syncthreads();
  if (!dev_cholesky(S, s, TM)) {
    if (threadIdx.x == 0) a.snew[k] = -1;
    return;
  }
  // C = C~ L^{-T}: Rinv = L^{-T} (upper); column c of L^{-T} solves L^T x = e_c
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    for (int i = s - 1; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int kk = i + 1; kk < s; ++kk) v -= S[kk * TM + i] * R[kk * TM + c];
      R[i * TM + c] = v / S[i * TM + i];
    }
  }
}

__global__ void k_copy_ztc(const int* mask, const int* scols, const double* G, int TM, int SMAX, double* ztc,
                           int K) {
  const int k = blockIdx.x;
  if (!mask[k]) return;
  const int s = scols[k];
  for (int idx = threadIdx.x; idx < SMAX * SMAX; idx += blockDim.x) {
    const int i = idx / SMAX, j = idx - (idx / SMAX) * SMAX;
    ztc[(size_t)k * SMAX * SMAX + idx] = (i < s && j < s) ? G[(size_t)k * TM * TM + i * TM + j] : 0.0;
  }
}

// Inner refresh: H^(i-1) [U, V_m] from the last CG solve's record (no Hessian actions).  With
// C = H U, P H p_j = (r_j - r_{j+1}) / alpha_j and p_j = r_j + beta_{j-1} p_{j-1}:
//   H V_m = V_{m+1} T_m + C B_m,  T_m (m+1 x m) tridiagonal:
//     T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T[j+1][j] = -nu_{j+1} / (nu_j alpha_j),
//     T[j-1][j] = -nu_j / (nu_{j-1} alpha_{j-1});   B[:, j] = (C^T H p_j - beta_{j-1} C^T H p_{j-1}) / nu_j,
//   nu_j = ||r_j|| = sqrt(rho_j), beta_{j-1} = rho_j / rho_{j-1}.
// Writes M (s + m + 1 x s + m, ld TM) with H [U, V_m] = [C, V_{m+1}] M.
__global__ void k_lanczos_rel(const int* mask, const int* s_old, const int* tcols, const double* lz_alpha,
                              const double* lz_rho, const double* lz_c, int KMAX, int SMAX, int TM, double* M) {
  const int k = blockIdx.x;
  if (!mask[k]) return;
  const int s = s_old[k], t = tcols[k];
  double* Mk = M + (size_t)k * TM * TM;
  const double* al = lz_alpha + (size_t)k * KMAX;
  const double* rh = lz_rho + (size_t)k * KMAX;
  const double* cc = lz_c + (size_t)k * KMAX * SMAX;
  for (int idx = threadIdx.x; idx < (t + 1) * t; idx += blockDim.x) {
    const int i = idx / t, j = idx - (idx / t) * t;
    double v = 0.0;
    if (j < s) {
      v = (i == j) ? 1.0 : 0.0;
    } else {
      const int jj = j - s;
      const double bprev = jj > 0 ? rh[jj] / rh[jj - 1] : 0.0;
      if (i < s) {
        double b = cc[(size_t)jj * SMAX + i];
        if (jj > 0) b -= bprev * cc[(size_t)(jj - 1) * SMAX + i];
        v = b / sqrt(rh[jj]);
      } else {
        const int r = i - s;
        if (r == jj) v = 1.0 / al[jj] + (jj > 0 ? bprev / al[jj - 1] : 0.0);
        else if (r == jj + 1) v = -sqrt(rh[jj + 1]) / (sqrt(rh[jj]) * al[jj]);
        else if (r == jj - 1) v = -sqrt(rh[jj]) / (sqrt(rh[jj - 1]) * al[jj - 1]);
      }
    }
    Mk[i * TM + j] = v;
  }
}

template <typename T>
static bl_status refresh_impl(bl_problem* P, const std::vector<int>& mask_host, const bl_recycle_opts* o) {
  const int K = P->K, TM = P->TM;
  const bool inner = o->variant == BL_REFRESH_INNER;
  // sprev: columns of the previous U in W = [U, V].  The inner form takes U only when the recorded
  // solve deflated with it (its C^T H p_j then complete the relation); after a solve without that
  // space, W is the Krylov basis alone, whose plain Lanczos relation is exact
  std::vector<int> msk(K, 0), tcols(K, 0), sprev(K, 0);
  bool any = false, cleared = false;
  for (int k = 0; k < K; ++k) {
    if (!mask_host[k]) continue;
    sprev[k] = (!inner || P->lz_u[k]) ? P->s_k[k] : 0;
    const int t = sprev[k] + P->kb_k[k];
    if (inner && t == 0 && P->s_k[k] && P->lz_k[k]) {
      // the recorded solve neither deflated with this pair's space nor took a step (a warm start
      // already below tolerance): nothing relates the space to the new Hessian, so this pair alone
      // loses it (its next solve is plain CG) and the record is consumed; reported as a breakdown
      P->s_k[k] = 0;
      P->hz_k[k] = 0;
      P->lz_k[k] = 0;
      cleared = true;
      continue;
    }
    // no basis yet: the recycle space stays empty (an inner refresh of a pair that holds a space
    // but has no record to relate it to is refused below)
    if (t == 0 && !(inner && P->s_k[k])) continue;
    msk[k] = 1;
    tcols[k] = t;
    any = true;
  }
  if (!any) {
    if (!cleared) return BL_OK;
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_s, P->s_k.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_hasz, P->hz_k.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));   // the host vectors are rewritten by later calls
    return fail(BL_EBREAKDOWN, "inner recycle refresh: a pair whose recorded solve took no step without its "
                               "recycle space was left with an empty space");
  }
  if (inner)
    for (int k = 0; k < K; ++k)
      if (msk[k] && (!P->lz_k[k] || tcols[k] == 0))
        return fail(BL_ESTATE, "inner refresh needs the last solve's Lanczos record (BL_STORE_LANCZOS)");
  int* d_mask = P->d_active + 2 * K;      // refresh mask
  int* d_t = P->d_cols;                   // t per pair
  int* d_tk = P->d_tk;                    // t' per pair
  int* d_sn = P->d_tk + K;                // selected s per pair
  BL_CUDA_TRY(cudaMemcpyAsync(d_mask, msk.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync(d_t, tcols.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  // 0. W = [U, V]
  for (int k = 0; k < K; ++k) {
    if (!msk[k]) continue;
    const auto& ph = P->ph[k];
    char* Wk = (char*)P->W + ph.off * TM * P->esz;
    if (sprev[k])
      BL_CUDA_TRY(cudaMemcpyAsync(Wk, (const char*)P->U + ph.off * P->SMAX * P->esz, (size_t)sprev[k] * ph.n * P->esz,
                                  cudaMemcpyDeviceToDevice, P->stream));
    if (P->kb_k[k])
      BL_CUDA_TRY(cudaMemcpyAsync(Wk + (size_t)sprev[k] * ph.n * P->esz, (const char*)P->V + ph.off * P->KMAX * P->esz,
                                  (size_t)P->kb_k[k] * ph.n * P->esz, cudaMemcpyDeviceToDevice, P->stream));
  }
  int tmax = 0;
  for (int k = 0; k < K; ++k) tmax = std::max(tmax, tcols[k]);
  const int smax = std::min(o->s, P->SMAX);
  if (inner) {
    // H^(i-1) W = [C, V_{m+1}] M from the record: X = [C, V_0 .. V_m] staged in Wt
    std::vector<int> xc(K, 0);
    for (int k = 0; k < K; ++k) {
      if (!msk[k]) continue;
      const auto& ph = P->ph[k];
      char* Xk = (char*)P->Wt + ph.off * TM * P->esz;
      xc[k] = tcols[k] + 1;
      if (sprev[k])
        BL_CUDA_TRY(cudaMemcpyAsync(Xk, (const char*)P->C + ph.off * P->SMAX * P->esz,
                                    (size_t)sprev[k] * ph.n * P->esz, cudaMemcpyDeviceToDevice, P->stream));
      BL_CUDA_TRY(cudaMemcpyAsync(Xk + (size_t)sprev[k] * ph.n * P->esz, (const char*)P->V + ph.off * P->KMAX * P->esz,
                                  (size_t)(P->kb_k[k] + 1) * ph.n * P->esz, cudaMemcpyDeviceToDevice, P->stream));
    }
    BL_CUDA_TRY(cudaMemcpyAsync(d_tk, xc.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    int* d_sprev = P->d_tk + 2 * K;
    BL_CUDA_TRY(cudaMemcpyAsync(d_sprev, sprev.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    {
      ProfScope ps(P, BL_KC_DENSE);
      k_lanczos_rel<<<K, 256, 0, P->stream>>>(d_mask, d_sprev, d_t, P->lz_alpha, P->lz_rho, P->lz_c, P->KMAX, P->SMAX,
                                              TM, P->dY2);
      BL_LAUNCH_CHECK(P);
    }
    bl_status sx = ts_gemm(P, P->Wt, TM, d_tk, tmax + 1, P->dY2, P->HWt, TM, d_t, tmax, nullptr, nullptr, 0, nullptr,
                           0, d_mask);
    if (sx != BL_OK) return sx;
  }
  DenseArgs da{};
  da.TM = TM;
  da.p = P->p;
  da.G = P->dG;
  da.T = P->dT;
  da.GH = P->dT + (size_t)K * TM * TM;
  da.J = P->dJ;
  da.jcols = tmax;
  da.Y = P->dY;
  da.Y2 = P->dY2;
  da.scratch = P->dY3;
  da.tk = d_tk;
  da.snew = d_sn;
  da.mask = d_mask;
  da.kind = o->kind;
  da.size = o->size;
  da.side = o->side;
  da.s = o->s;
  da.drop = P->prec == BL_FP32 ? 1e-6 : 1e-12;
  const size_t dsm = (2 * (size_t)TM * TM + 4 * TM + 8) * sizeof(double) + TM * sizeof(int) + 64;
  if (!P->capturing) {
    BL_CUDA_TRY(cudaFuncSetAttribute(k_dense_orth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    BL_CUDA_TRY(cudaFuncSetAttribute(k_dense_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
  }

  // 1. orthonormal basis W~ = W B1
  bl_status st = ts_gram(P, P->W, TM, d_t, tmax, P->W, TM, d_t, tmax, d_mask, P->dG);
  if (st != BL_OK) return st;
  {
    ProfScope ps(P, BL_KC_DENSE);
    k_dense_orth<<<K, 256, dsm, P->stream>>>(da, d_t);
    BL_LAUNCH_CHECK(P);
  }
  st = ts_gemm(P, P->W, TM, d_t, tmax, P->dY, P->Wt, TM, d_tk, tmax, nullptr, nullptr, 0, nullptr, 0, d_mask);
  if (st != BL_OK) return st;
  // 2. H W~: Hessian actions at the current point (outer), or H^(i-1) W B1 from the record (inner)
  if (inner) {
    st = ts_gemm(P, P->HWt, TM, d_t, tmax, P->dY, P->HWt, TM, d_tk, tmax, nullptr, nullptr, 0, nullptr, 0, d_mask);
    if (st != BL_OK) return st;
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_cols, d_tk, K * sizeof(int), cudaMemcpyDeviceToDevice, P->stream));
  } else {
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_cols, d_tk, K * sizeof(int), cudaMemcpyDeviceToDevice, P->stream));
    st = launch_hvp(P, P->Wt, P->HWt, TM, tmax, d_mask, nullptr, nullptr);
    if (st != BL_OK) return st;
  }
  // 3. projected matrices
  st = ts_gram(P, P->Wt, TM, d_tk, tmax, P->HWt, TM, d_tk, tmax, d_mask, P->dT);
  if (st != BL_OK) return st;
  if (o->kind == BL_RECYCLE_HRITZ) {
    st = ts_gram(P, P->HWt, TM, d_tk, tmax, P->HWt, TM, d_tk, tmax, d_mask, P->dT + (size_t)K * TM * TM);
    if (st != BL_OK) return st;
  }
  if (o->kind == BL_RECYCLE_RGSV) {
    st = launch_jw(P, P->Wt, TM, tmax, d_mask, P->dJ);
    if (st != BL_OK) return st;
  }
  // 4. selection
  {
    ProfScope ps(P, BL_KC_DENSE);
    // 16 warps: the Householder updates and the Jacobi rounds give a warp per column / per pair
    k_dense_select<<<K, 512, dsm, P->stream>>>(da);
    BL_LAUNCH_CHECK(P);
  }
  // 5. U~ = W~ Y and Z = W~ Y2 in one pass over W~, C~ = HW~ Y
  const bool rgsv = o->kind == BL_RECYCLE_RGSV;
  st = ts_gemm(P, P->Wt, TM, d_tk, tmax, P->dY, P->U, P->SMAX, d_sn, smax, rgsv ? P->dY2 : nullptr,
               rgsv ? P->Z : nullptr, P->SMAX, d_sn, smax, d_mask);
  if (st != BL_OK) return st;
  if (inner) {
    // C~ = H^(i) U~: the new system's operator (s Hessian actions)
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_cols, d_sn, K * sizeof(int), cudaMemcpyDeviceToDevice, P->stream));
    st = launch_hvp(P, P->U, P->C, P->SMAX, smax, d_mask, nullptr, nullptr);
  } else {
    st = ts_gemm(P, P->HWt, TM, d_tk, tmax, P->dY, P->C, P->SMAX, d_sn, smax, nullptr, nullptr, 0, nullptr, 0, d_mask);
  }
  if (st != BL_OK) return st;
  // CholeskyQR2 of C~, applied to U~ as well
  for (int rep = 0; rep < 2; ++rep) {
    st = ts_gram(P, P->C, P->SMAX, d_sn, smax, P->C, P->SMAX, d_sn, smax, d_mask, P->dG);
    if (st != BL_OK) return st;
    {
      ProfScope ps(P, BL_KC_DENSE);
      k_dense_cholinv<<<K, 128, 0, P->stream>>>(da, d_sn, P->dG, P->dY);
      BL_LAUNCH_CHECK(P);
    }
    st = ts_gemm(P, P->C, P->SMAX, d_sn, smax, P->dY, P->C, P->SMAX, d_sn, smax, nullptr, nullptr, 0, nullptr, 0,
                 d_mask);
    if (st != BL_OK) return st;
    st = ts_gemm(P, P->U, P->SMAX, d_sn, smax, P->dY, P->U, P->SMAX, d_sn, smax, nullptr, nullptr, 0, nullptr, 0,
                 d_mask);
    if (st != BL_OK) return st;
  }
  if (rgsv) {
    st = ts_gram(P, P->Z, P->SMAX, d_sn, smax, P->C, P->SMAX, d_sn, smax, d_mask, P->dG);
    if (st != BL_OK) return st;
    k_copy_ztc<<<K, 128, 0, P->stream>>>(d_mask, d_sn, P->dG, TM, P->SMAX, P->ztc, K);
    BL_LAUNCH_CHECK(P);
  }
  std::vector<int> sn(K, 0);
  BL_CUDA_TRY(cudaMemcpyAsync(sn.data(), d_sn, K * sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  bool broke = false;
  for (int k = 0; k < K; ++k) {
    if (!msk[k]) continue;
    if (sn[k] < 0) {
      broke = true;
      P->s_k[k] = 0;
      P->hz_k[k] = 0;
    } else {
      P->s_k[k] = sn[k];
      P->hz_k[k] = (o->kind == BL_RECYCLE_RGSV && sn[k] > 0) ? 1 : 0;
    }
    P->kb_k[k] = 0;   // the basis and its Lanczos record have been consumed
    P->lz_k[k] = 0;
  }
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_s, P->s_k.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_hasz, P->hz_k.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  if (broke) return fail(BL_EBREAKDOWN, "recycle refresh: projected Hessian not positive definite");
  if (cleared) {
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    return fail(BL_EBREAKDOWN, "inner recycle refresh: a pair whose recorded solve took no step without its "
                               "recycle space was left with an empty space");
  }
  return BL_OK;
}

bl_status run_ritz_update(bl_problem* P, const std::vector<int>& mask_host, const bl_recycle_opts* o) {
  const bl_status st = P->prec == BL_FP32 ? refresh_impl<float>(P, mask_host, o) : refresh_impl<double>(P, mask_host, o);
  const bl_status ke = check_kernel_error(P);
  return ke != BL_OK ? ke : st;
}

}  // namespace bl
