// Batched recycled conjugate gradient for H_k w_k = g_k (Section 2.2, stopping rules of Section 4).
//
// Augmented CG over the recycle space U_k with C_k = H_k U_k, C_k^T C_k = I:
//   init   r = g - H w0;  c0 = C^T r;  w += U c0;  r -= C c0;  p = r;  rho = r^T r;  z = 0
//   loop   q = H p;  c = C^T q;  alpha = rho / p^T q;  w += alpha p;  z -= alpha c;
//          r -= alpha (q - C c);  beta = rho' / rho;  p = r + beta p
//   end    w += U z
// which is CG on P H P (P = I - C C^T) with the recycle-space coefficients gathered in z, so that
// g - H (w + U z) = r and C^T r = 0 hold throughout (the augmentation of Algorithm 3 carried
// over to CG).  The hypergradient-error estimate of eq. (4.2), ||Z^T r||, is formed from the
// updated residual in the same pass that updates it.
//
// Recycled MINRES (Algorithm 3, for symmetric indefinite Hessians) shares the initial projection
// and runs Lanczos on P H P from v_1 = r_0 / beta_1, the QR factorisation of the tridiagonal by
// Givens rotations (c_k, s_k) and zeta_k = -s_k zeta_{k-1} (|zeta_k| is the residual norm).  The
// direction vt_k = (v_k - gamma_k vt_{k-2} - delta_k vt_{k-1}) / eps~_k updates w by
// c_k zeta_{k-1} vt_k; its recycle-space part bt_k = U beta~_k, with the s coefficients beta~_k
// following the same recurrence driven by C^T H v_k, is subtracted through z (the minus sign of the
// reading of Algorithm 3).  The explicit residual of Appendix A enters the hypergradient-error rule
// only through Z^T res, carried by the s-dimensional images of its recurrence, Z^T Hvt_k and
// Z^T C beta~_k.
//
// All pairs advance together: vectors are batched over pairs, every per-pair scalar (rho, alpha,
// beta, the s-vectors c, z, Z^T r) lives on the device in FP64, and each kernel skips the pairs
// whose `active` flag is cleared (converged, iteration cap or breakdown).  The Hessian action
// of the FoE regulariser computes p^T q, C^T q and Z^T q in its epilogue.
#include <cmath>

#include "common.cuh"
#include "device.cuh"

namespace bl {

struct KrylovArgs {
  const PairDev* pairs;
  const ChunkDev* chunks;
  SolveState* st;
  const int* s_k;     // effective recycle dimension (0 for plain CG)
  const int* hasz;    // NSC operator present and used
  int SMAX, KMAX;
  double* c;          // K x SMAX
  double* zc;         // K x SMAX
  double* e;          // K x SMAX
  double* ztr;        // K x SMAX
  const double* ztc;  // K x SMAX x SMAX, row i = Z_i^T C
  double* cpart;
  const double* tpart;
  int n_tiles, n_chunks;
  double *b1, *b2, *h1, *h2;   // MINRES: beta~_{k-1}, beta~_{k-2}, Z^T Hvt_{k-1}, Z^T Hvt_{k-2} (K x SMAX)
  // CG Lanczos record (BL_STORE_LANCZOS): alpha_j, rho_j (K x KMAX), C^T H p_j (K x KMAX x SMAX)
  int lanczos;
  double *lz_alpha, *lz_rho, *lz_c;
  unsigned long long* nbytes;   // algorithmic bytes of the vector passes (profiling), or null
};

// Per-chunk partial sums of up to 64 components, one warp total each, written to part[chunk][off + m].
template <int NT>
__device__ __forceinline__ void flush_components(const double* warp_vals, int cnt, double* dst) {
  if ((int)threadIdx.x < cnt) {
    double t = 0.0;
    for (int q2 = 0; q2 < NT / 32; ++q2) t += warp_vals[q2 * 65 + threadIdx.x];
    dst[threadIdx.x] = t;
  }
}

// r = g - q (warm) or r = g, w = 0 (cold); partials [0] ||g||^2, [1..s] C^T r.
template <typename T>
__global__ void k_init_r(KrylovArgs a, const T* g, const T* q, T* r, T* w, const T* C, int warm,
                         const int* mask) {
  __shared__ double red[8 * 65];
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!mask[ch.pair]) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  const int ncomp = 1 + a.SMAX;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* Cb = C + pr.off * a.SMAX;
  {
    Accum<T> acc;
    for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
      const long long gi = pr.off + ch.start + t;
      const T gv = g[gi];
      r[gi] = warm ? gv - q[gi] : gv;
      if (!warm) w[gi] = T(0);
      acc.add(gv * gv);
    }
    const double v = warp_total(acc);
    if (lane == 0) red[wid * 65] = v;
  }
  // each thread reads back only the r values it wrote
  for (int cc = 1; cc <= s; cc += 64) {
    const int cnt = min(64, s + 1 - cc);
    for (int m = 0; m < cnt; ++m) {
      const T* col = Cb + (long long)(cc - 1 + m) * pr.n;
      Accum<T> acc;
      for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
        const long long li = ch.start + t;
        acc.add(col[li] * r[pr.off + li]);
      }
      const double v = warp_total(acc);
      if (lane == 0) red[wid * 65 + 1 + m] = v;
    }
    __syncthreads();
    if (cc == 1) flush_components<kChunkThreads>(red, 1 + cnt, a.cpart + (size_t)blockIdx.x * ncomp);
    else flush_components<kChunkThreads>(red + 1, cnt, a.cpart + (size_t)blockIdx.x * ncomp + cc);
    __syncthreads();
  }
  if (s == 0) {
    __syncthreads();
    flush_components<kChunkThreads>(red, 1, a.cpart + (size_t)blockIdx.x * ncomp);
  }
}

// c0 = C^T r, ||g||^2 per pair
__global__ void k_scalar_init1(KrylovArgs a, const int* mask) {
  const int k = blockIdx.x;
  if (!mask[k]) return;
  const PairDev pr = a.pairs[k];
  const int s = a.s_k[k];
  const int ncomp = 1 + a.SMAX;
  for (int m = threadIdx.x; m <= s; m += blockDim.x) {
    double t = 0.0;
    for (int u = pr.cbeg; u < pr.cend; ++u) t += a.cpart[(size_t)u * ncomp + m];
    if (m == 0) a.st[k].gnorm2 = t;
    else a.c[k * a.SMAX + m - 1] = t;
  }
}

// w += U c0; r -= C c0; p = r; partials [0] rho, [1..nz] Z^T r
template <typename T>
__global__ void k_init2(KrylovArgs a, T* w, T* r, T* p, const T* U, const T* C, const T* Z, const int* mask) {
  __shared__ double red[8 * 65];
  __shared__ T cs[64];
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!mask[ch.pair]) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  const int nz = a.hasz[ch.pair] ? s : 0;
  const int ncomp = 1 + a.SMAX;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if ((int)threadIdx.x < s) cs[threadIdx.x] = (T)a.c[ch.pair * a.SMAX + threadIdx.x];
  __syncthreads();
  const T* Ub = U + pr.off * a.SMAX;
  const T* Cb = C + pr.off * a.SMAX;
  const T* Zb = Z + pr.off * a.SMAX;
  Accum<T> rho;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    T uc = 0, ccv = 0;
    for (int j = 0; j < s; ++j) {
      uc = fma(cs[j], Ub[(long long)j * pr.n + li], uc);
      ccv = fma(cs[j], Cb[(long long)j * pr.n + li], ccv);
    }
    const T rn = r[gi] - ccv;
    w[gi] = w[gi] + uc;
    r[gi] = rn;
    p[gi] = rn;
    rho.add(rn * rn);
  }
  {
    const double v = warp_total(rho);
    if (lane == 0) red[wid * 65] = v;
  }
  for (int m = 0; m < nz; ++m) {
    Accum<T> acc;
    for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
      const long long li = ch.start + t;
      acc.add(Zb[(long long)m * pr.n + li] * r[pr.off + li]);
    }
    const double v = warp_total(acc);
    if (lane == 0) red[wid * 65 + 1 + (m & 63)] = v;
    if ((m & 63) == 63 || m == nz - 1) {
      __syncthreads();
      const int base = (m & ~63);
      flush_components<kChunkThreads>(red + 1, m - base + 1, a.cpart + (size_t)blockIdx.x * ncomp + 1 + base);
      __syncthreads();
    }
  }
  __syncthreads();
  flush_components<kChunkThreads>(red, 1, a.cpart + (size_t)blockIdx.x * ncomp);
}

// rho, Z^T r, tolerance and the active flags
__global__ void k_scalar_init2(KrylovArgs a, const int* mask, int stop_nsc, double tol, int relative,
                               const double* nsc_scale, int maxit, int* flag) {
  __shared__ double sh[65];
  const int k = blockIdx.x;
  if (!mask[k]) return;
  const PairDev pr = a.pairs[k];
  const int s = a.s_k[k];
  const int nz = a.hasz[k] ? s : 0;
  const int ncomp = 1 + a.SMAX;
  for (int m = threadIdx.x; m <= nz; m += blockDim.x) {
    double t = 0.0;
    for (int u = pr.cbeg; u < pr.cend; ++u) t += a.cpart[(size_t)u * ncomp + m];
    if (m == 0) sh[64] = t;
    else a.ztr[k * a.SMAX + m - 1] = t;
  }
  for (int m = threadIdx.x; m < a.SMAX; m += blockDim.x) a.zc[k * a.SMAX + m] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    SolveState S = a.st[k];
    S.rho = sh[64];
    S.iters = 0;
    S.status = BL_OK;
    S.maxit = maxit;
    const bool nsc = stop_nsc && nz > 0;
    double est, scale;
    if (nsc) {
      double z2 = 0.0;
      for (int m = 0; m < nz; ++m) z2 += a.ztr[k * a.SMAX + m] * a.ztr[k * a.SMAX + m];
      est = sqrt(z2);
      scale = (relative && nsc_scale) ? nsc_scale[k] : 1.0;
    } else {
      est = sqrt(S.rho);
      scale = (relative || stop_nsc) ? sqrt(S.gnorm2) : 1.0;
    }
    S.tol = tol * scale;
    S.est = est;
    if (a.lanczos && a.KMAX > 0) a.lz_rho[(size_t)k * a.KMAX] = S.rho;
    S.active = (est >= S.tol && maxit > 0 && S.rho > 0.0) ? 1 : 0;
    if (!isfinite(S.rho)) {
      S.active = 0;
      S.status = BL_EBREAKDOWN;
    }
    a.st[k] = S;
    if (S.active) atomicAdd(flag, 1);
  }
}

// generic chunk dots for problems without the fused epilogue: [0] p^T q, [1..s] C^T q, [1+SMAX..] Z^T q
template <typename T>
__global__ void k_dots(KrylovArgs a, const T* p, const T* q, const T* C, const T* Z) {
  __shared__ double red[8 * 65];
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!a.st[ch.pair].active) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  const int nz = a.hasz[ch.pair] ? s : 0;
  const int ncomp = 1 + 2 * a.SMAX;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* Cb = C + pr.off * a.SMAX;
  const T* Zb = Z + pr.off * a.SMAX;
  const int total = 1 + s + nz;
  for (int base = 0; base < total; base += 64) {
    const int cnt = min(64, total - base);
    for (int m = 0; m < cnt; ++m) {
      const int comp = base + m;
      const T* src = comp == 0 ? p + pr.off
                               : (comp <= s ? Cb + (long long)(comp - 1) * pr.n : Zb + (long long)(comp - 1 - s) * pr.n);
      Accum<T> acc;
      for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
        const long long li = ch.start + t;
        acc.add(src[li] * q[pr.off + li]);
      }
      const double v = warp_total(acc);
      if (lane == 0) red[wid * 65 + m] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      double tt = 0.0;
      for (int q2 = 0; q2 < kChunkThreads / 32; ++q2) tt += red[q2 * 65 + threadIdx.x];
      const int comp = base + threadIdx.x;
      const int slot = comp <= s ? comp : comp - s + a.SMAX;
      a.cpart[(size_t)blockIdx.x * ncomp + slot] = tt;
    }
    __syncthreads();
  }
}

// The same partials for FP32 problems whose images are multiples of 4 pixels (16-byte aligned column
// starts): every thread keeps its four 128-bit blocks of q in registers (a chunk is 4,096 pixels =
// 1,024 blocks) and streams the matching blocks of the components, eight components per group with
// all their loads in flight, into compensated FP32 sums; one barrier per group combines the warps
// in FP64.  q is read once, and no warp idles while another finishes a component.
__global__ void __launch_bounds__(kChunkThreads) k_dots_v4(KrylovArgs a, const float* p, const float* q,
                                                           const float* C, const float* Z) {
  constexpr int NW = kChunkThreads / 32, GC = 8, PB = kChunk / 4 / kChunkThreads;
  static_assert(PB * 4 * kChunkThreads == kChunk, "a chunk is PB 128-bit blocks per thread");
  __shared__ double red[NW][GC];
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!a.st[ch.pair].active) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  const int nz = a.hasz[ch.pair] ? s : 0;
  const int ncomp = 1 + 2 * a.SMAX, nc = 1 + s + nz;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (a.nbytes && threadIdx.x == 0) atomicAdd(a.nbytes, (unsigned long long)ch.len * 4ull * (2 + s + nz));
  const int nv = ch.len >> 2;                                  // chunk lengths are multiples of 4
  const float4* q4 = reinterpret_cast<const float4*>(q + pr.off + ch.start);
  float4 qv[PB];
#pragma unroll
  for (int m = 0; m < PB; ++m) {
    const int i = threadIdx.x + m * kChunkThreads;
    qv[m] = i < nv ? q4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int g0 = 0; g0 < nc; g0 += GC) {
    Accum<float> acc[GC];
#pragma unroll
    for (int c = 0; c < GC; ++c) {
      const int comp = g0 + c;
      if (comp >= nc) break;
      const float* src = comp == 0 ? p + pr.off
                                   : (comp <= s ? C + pr.off * a.SMAX + (long long)(comp - 1) * pr.n
                                                : Z + pr.off * a.SMAX + (long long)(comp - 1 - s) * pr.n);
      const float4* s4 = reinterpret_cast<const float4*>(src + ch.start);
#pragma unroll
      for (int m = 0; m < PB; ++m) {
        const int i = threadIdx.x + m * kChunkThreads;
        if (i < nv) {
          const float4 u = s4[i];
          acc[c].add(u.x * qv[m].x);
          acc[c].add(u.y * qv[m].y);
          acc[c].add(u.z * qv[m].z);
          acc[c].add(u.w * qv[m].w);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < GC; ++c) {
      const double t = warp_total(acc[c]);
      if (lane == 0) red[wid][c] = t;
    }
    __syncthreads();
    if ((int)threadIdx.x < GC && g0 + (int)threadIdx.x < nc) {
      double tot = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) tot += red[w][threadIdx.x];
      const int comp = g0 + threadIdx.x;
      const int slot = comp <= s ? comp : comp - s + a.SMAX;
      a.cpart[(size_t)blockIdx.x * ncomp + slot] = tot;
    }
    __syncthreads();
  }
}

// alpha, c = C^T q, z -= alpha c; breakdown check
__global__ void k_scalar1(KrylovArgs a, int use_tiles) {
  __shared__ double sh[65];
  __shared__ double alpha_s;
  const int k = blockIdx.x;
  if (!a.st[k].active) return;
  const PairDev pr = a.pairs[k];
  const int s = a.s_k[k];
  const int ncomp = use_tiles ? 1 + 2 * a.SMAX : 1 + 2 * a.SMAX;
  const double* part = use_tiles ? a.tpart : a.cpart;
  const int beg = use_tiles ? pr.tbeg : pr.cbeg, end = use_tiles ? pr.tend : pr.cend;
  {
    // unit partials: a warp per value, its lanes over the pair's units
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int m = wid; m < 1 + s; m += nwarp) {
      double t = 0.0;
      for (int u = beg + lane; u < end; u += 32) t += part[(size_t)u * ncomp + m];
      t = warp_sum(t);
      if (lane == 0) sh[m] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SolveState S = a.st[k];
    S.pq = sh[0];
    if (!(S.pq > 0.0) || !isfinite(S.pq)) {
      S.active = 0;
      S.status = BL_EBREAKDOWN;
      alpha_s = 0.0;
    } else {
      S.alpha = S.rho / S.pq;
      alpha_s = S.alpha;
    }
    a.st[k] = S;
  }
  __syncthreads();
  const double al = alpha_s;
  const int it = a.st[k].iters;
  const bool rec = a.lanczos && it < a.KMAX;
  if (rec && threadIdx.x == 0) a.lz_alpha[(size_t)k * a.KMAX + it] = al;
  for (int m = threadIdx.x; m < s; m += blockDim.x) {
    a.c[k * a.SMAX + m] = sh[1 + m];
    a.zc[k * a.SMAX + m] -= al * sh[1 + m];
    if (rec) a.lz_c[((size_t)k * a.KMAX + it) * a.SMAX + m] = sh[1 + m];
  }
}

// w += alpha p; V[:, it] = r / ||r||; r -= alpha (q - C c); partials [0] rho' = r^T r and, for the
// NSC rule, [1..nz] Z^T r (read back from the r values this thread just wrote)
template <typename T>
__global__ void k_update(KrylovArgs a, T* w, T* r, const T* p, const T* q, const T* C, const T* Z, T* V,
                         int store, int nsc) {
  __shared__ double red[8 * 65];
  __shared__ T cs[64];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const SolveState S = a.st[ch.pair];
  if (!S.active) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  const int nz = (nsc && a.hasz[ch.pair]) ? s : 0;
  const int ncomp = 1 + a.SMAX;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if ((int)threadIdx.x < s) cs[threadIdx.x] = (T)a.c[ch.pair * a.SMAX + threadIdx.x];
  __syncthreads();
  const T* Cb = C + pr.off * a.SMAX;
  const T* Zb = Z + pr.off * a.SMAX;
  if (a.nbytes && threadIdx.x == 0) {
    const int stored = (store == 1 || (store == 2 && S.iters < a.KMAX)) ? 1 : 0;
    atomicAdd(a.nbytes, (unsigned long long)ch.len * sizeof(T) * (4 + s + nz + 2 + stored));
  }
  // store 1: ring of the most recent KMAX residuals; store 2: the first KMAX (Lanczos record)
  const bool st_now = store == 1 || (store == 2 && S.iters < a.KMAX);
  T* Vc = st_now ? V + pr.off * a.KMAX + (long long)(S.iters % a.KMAX) * pr.n : nullptr;
  const T inv_nr = (T)(1.0 / sqrt(S.rho));
  const T al = (T)S.alpha;
  Accum<T> rho;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    const T ro = r[gi];
    if (Vc) Vc[li] = ro * inv_nr;
    w[gi] = fma(al, p[gi], w[gi]);
    T ccv = 0;
    for (int j = 0; j < s; ++j) ccv = fma(cs[j], Cb[(long long)j * pr.n + li], ccv);
    const T rn = ro - al * (q[gi] - ccv);
    r[gi] = rn;
    rho.add(rn * rn);
  }
  {
    const double v = warp_total(rho);
    if (lane == 0) red[wid * 65] = v;
  }
  for (int m = 0; m < nz; ++m) {
    Accum<T> acc;
    for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
      const long long li = ch.start + t;
      acc.add(Zb[(long long)m * pr.n + li] * r[pr.off + li]);
    }
    const double v = warp_total(acc);
    if (lane == 0) red[wid * 65 + 1 + (m & 63)] = v;
    if ((m & 63) == 63 || m == nz - 1) {
      __syncthreads();
      const int base = (m & ~63);
      flush_components<kChunkThreads>(red + 1, m - base + 1, a.cpart + (size_t)blockIdx.x * ncomp + 1 + base);
      __syncthreads();
    }
  }
  __syncthreads();
  flush_components<kChunkThreads>(red, 1, a.cpart + (size_t)blockIdx.x * ncomp);
}

// The update pass for FP32 problems whose images are multiples of 4 pixels: each thread moves float4
// items (16-byte loads and stores), the C columns of an item loaded together before their products.
__global__ void k_update_v4(KrylovArgs a, float* w, float* r, const float* p, const float* q, const float* C,
                            const float* Z, float* V, int store, int nsc) {
  __shared__ double red[8 * 65];
  __shared__ float cs[64];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const SolveState S = a.st[ch.pair];
  if (!S.active) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  const int nz = (nsc && a.hasz[ch.pair]) ? s : 0;
  const int ncomp = 1 + a.SMAX;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if ((int)threadIdx.x < s) cs[threadIdx.x] = (float)a.c[ch.pair * a.SMAX + threadIdx.x];
  __syncthreads();
  const bool st_now = store == 1 || (store == 2 && S.iters < a.KMAX);
  if (a.nbytes && threadIdx.x == 0)
    atomicAdd(a.nbytes, (unsigned long long)ch.len * 4ull * (4 + s + nz + 2 + (st_now ? 1 : 0)));
  const long long g0 = pr.off + ch.start;
  const int nv = ch.len >> 2;
  float4* r4 = reinterpret_cast<float4*>(r + g0);
  float4* w4 = reinterpret_cast<float4*>(w + g0);
  const float4* p4 = reinterpret_cast<const float4*>(p + g0);
  const float4* q4 = reinterpret_cast<const float4*>(q + g0);
  const float* Cb = C + pr.off * a.SMAX + ch.start;
  float4* V4 = st_now ? reinterpret_cast<float4*>(V + pr.off * a.KMAX + (long long)(S.iters % a.KMAX) * pr.n +
                                                  ch.start)
                      : nullptr;
  const float inv_nr = (float)(1.0 / sqrt(S.rho));
  const float al = (float)S.alpha;
  Accum<float> rho;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const float4 ro = r4[i], pv = p4[i], qv = q4[i];
    float4 wv = w4[i];
    if (V4) V4[i] = make_float4(ro.x * inv_nr, ro.y * inv_nr, ro.z * inv_nr, ro.w * inv_nr);
    wv.x = fmaf(al, pv.x, wv.x);
    wv.y = fmaf(al, pv.y, wv.y);
    wv.z = fmaf(al, pv.z, wv.z);
    wv.w = fmaf(al, pv.w, wv.w);
    w4[i] = wv;
    float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int j = 0; j < s; ++j) {
      const float4 cv = reinterpret_cast<const float4*>(Cb + (long long)j * pr.n)[i];
      cc.x = fmaf(cs[j], cv.x, cc.x);
      cc.y = fmaf(cs[j], cv.y, cc.y);
      cc.z = fmaf(cs[j], cv.z, cc.z);
      cc.w = fmaf(cs[j], cv.w, cc.w);
    }
    const float4 rn = make_float4(ro.x - al * (qv.x - cc.x), ro.y - al * (qv.y - cc.y), ro.z - al * (qv.z - cc.z),
                                  ro.w - al * (qv.w - cc.w));
    r4[i] = rn;
    rho.add(rn.x * rn.x);
    rho.add(rn.y * rn.y);
    rho.add(rn.z * rn.z);
    rho.add(rn.w * rn.w);
  }
  {
    const double v = warp_total(rho);
    if (lane == 0) red[wid * 65] = v;
  }
  const float* Zb = Z + pr.off * a.SMAX + ch.start;
  for (int m = 0; m < nz; ++m) {
    Accum<float> acc;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      const float4 zv = reinterpret_cast<const float4*>(Zb + (long long)m * pr.n)[i];
      const float4 rv = r4[i];
      acc.add(zv.x * rv.x);
      acc.add(zv.y * rv.y);
      acc.add(zv.z * rv.z);
      acc.add(zv.w * rv.w);
    }
    const double v = warp_total(acc);
    if (lane == 0) red[wid * 65 + 1 + (m & 63)] = v;
    if ((m & 63) == 63 || m == nz - 1) {
      __syncthreads();
      const int base = (m & ~63);
      flush_components<kChunkThreads>(red + 1, m - base + 1, a.cpart + (size_t)blockIdx.x * ncomp + 1 + base);
      __syncthreads();
    }
  }
  __syncthreads();
  flush_components<kChunkThreads>(red, 1, a.cpart + (size_t)blockIdx.x * ncomp);
}

// rho', Z^T r, beta, stopping test
__global__ void k_scalar2(KrylovArgs a, int stop_nsc, int* flag) {
  __shared__ double sh[65];
  const int k = blockIdx.x;
  if (!a.st[k].active) return;
  const PairDev pr = a.pairs[k];
  const int s = a.s_k[k];
  const int nz = (stop_nsc && a.hasz[k]) ? s : 0;
  const int ncomp = 1 + a.SMAX;
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int m = wid; m <= nz; m += nwarp) {
      double t = 0.0;
      for (int u = pr.cbeg + lane; u < pr.cend; u += 32) t += a.cpart[(size_t)u * ncomp + m];
      t = warp_sum(t);
      if (lane == 0) sh[m] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SolveState S = a.st[k];
    const double rho_new = sh[0];
    S.rho_new = rho_new;
    S.beta = rho_new / S.rho;
    S.rho = rho_new;
    S.iters += 1;
    if (a.lanczos && S.iters < a.KMAX) a.lz_rho[(size_t)k * a.KMAX + S.iters] = rho_new;
    if (nz > 0) {
      double z2 = 0.0;
      for (int m = 0; m < nz; ++m) {
        a.ztr[k * a.SMAX + m] = sh[1 + m];
        z2 += sh[1 + m] * sh[1 + m];
      }
      S.est = sqrt(z2);
    } else {
      S.est = sqrt(rho_new);
    }
    if (!isfinite(rho_new)) {
      S.active = 0;
      S.status = BL_EBREAKDOWN;
    } else if (S.est < S.tol || rho_new == 0.0) {
      S.active = 0;
    } else if (S.iters >= S.maxit) {
      S.active = 0;
      S.status = BL_ENOCONV;
    }
    a.st[k] = S;
    if (S.active) atomicAdd(flag, 1);
  }
}

template <typename T>
__global__ void k_pupdate(KrylovArgs a, const T* r, T* p) {
  const ChunkDev ch = a.chunks[blockIdx.x];
  const SolveState S = a.st[ch.pair];
  if (!S.active) return;
  const PairDev pr = a.pairs[ch.pair];
  const T be = (T)S.beta;
  if (a.nbytes && threadIdx.x == 0) atomicAdd(a.nbytes, (unsigned long long)ch.len * sizeof(T) * 3);
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long gi = pr.off + ch.start + t;
    p[gi] = fma(be, p[gi], r[gi]);
  }
}

// Lanczos record: the residual after the last step, normalised, as basis vector `iters` (zero if the
// residual vanished), so that H V_m = V_{m+1} T_m + C B_m can be formed for m = min(iters, KMAX - 1)
template <typename T>
__global__ void k_store_last(KrylovArgs a, const T* r, T* V, const int* mask) {
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!mask[ch.pair]) return;
  const SolveState S = a.st[ch.pair];
  if (S.iters >= a.KMAX) return;
  const PairDev pr = a.pairs[ch.pair];
  T* Vc = V + pr.off * a.KMAX + (long long)S.iters * pr.n;
  const T sc = S.rho > 0.0 ? (T)(1.0 / sqrt(S.rho)) : T(0);
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) Vc[ch.start + t] = r[pr.off + ch.start + t] * sc;
}

// w += U z
template <typename T>
__global__ void k_finalize(KrylovArgs a, T* w, const T* U, const int* mask) {
  __shared__ T zs[64];
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!mask[ch.pair]) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  if (s == 0) return;
  if ((int)threadIdx.x < s) zs[threadIdx.x] = (T)a.zc[ch.pair * a.SMAX + threadIdx.x];
  __syncthreads();
  const T* Ub = U + pr.off * a.SMAX;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    T uz = 0;
    for (int j = 0; j < s; ++j) uz = fma(zs[j], Ub[(long long)j * pr.n + li], uz);
    w[gi] = w[gi] + uz;
  }
}


// ---------------------------------------------------------------------------------------------
// MINRES kernels

// beta_1 = ||r_0||, zeta_0 = beta_1, rotations (c, s)_{0} = (1, 0), (c, s)_{-1} = (0, 0); s-vector
// histories cleared
__global__ void k_mr_start(KrylovArgs a, const int* mask) {
  const int k = blockIdx.x;
  if (!mask[k]) return;
  for (int m = threadIdx.x; m < a.SMAX; m += blockDim.x) {
    const size_t i = (size_t)k * a.SMAX + m;
    a.b1[i] = a.b2[i] = a.h1[i] = a.h2[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    SolveState S = a.st[k];
    S.beta_l = sqrt(fmax(S.rho, 0.0));
    S.zeta = S.beta_l;
    S.cm1 = 1.0;
    S.sm1 = 0.0;
    S.cm2 = 0.0;
    S.sm2 = 0.0;
    S.inv_bn = S.beta_l > 0.0 ? 1.0 / S.beta_l : 0.0;
    a.st[k] = S;
  }
}

// v_1 = r_0 / beta_1 (in place: the init left p = r_0), v_0 = vt_0 = vt_{-1} = 0
template <typename T>
__global__ void k_mr_vinit(KrylovArgs a, T* v, T* vprev, T* y1, T* y2, const int* mask) {
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!mask[ch.pair]) return;
  const PairDev pr = a.pairs[ch.pair];
  const T sc = (T)a.st[ch.pair].inv_bn;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long gi = pr.off + ch.start + t;
    v[gi] = v[gi] * sc;
    vprev[gi] = T(0);
    y1[gi] = T(0);
    y2[gi] = T(0);
  }
}

// alpha_k = v_k^T H v_k, C^T H v_k into c, Z^T H v_k into e (from the Hessian-action partials)
__global__ void k_mr_scalar1(KrylovArgs a, int use_tiles, int nsc) {
  const int k = blockIdx.x;
  if (!a.st[k].active) return;
  const PairDev pr = a.pairs[k];
  const int s = a.s_k[k];
  const int nz = (nsc && a.hasz[k]) ? s : 0;
  const int ncomp = 1 + 2 * a.SMAX;
  const double* part = use_tiles ? a.tpart : a.cpart;
  const int beg = use_tiles ? pr.tbeg : pr.cbeg, end = use_tiles ? pr.tend : pr.cend;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int m = wid; m < 1 + s + nz; m += nwarp) {
    const int slot = m <= s ? m : 1 + a.SMAX + (m - 1 - s);
    double t = 0.0;
    for (int u = beg + lane; u < end; u += 32) t += part[(size_t)u * ncomp + slot];
    t = warp_sum(t);
    if (lane != 0) continue;
    if (m == 0) a.st[k].alpha = t;
    else if (m <= s) a.c[k * a.SMAX + m - 1] = t;
    else a.e[k * a.SMAX + m - 1 - s] = t;
  }
}

// Lanczos: vn = H v_k - C (C^T H v_k) - alpha_k v_k - beta_k v_{k-1} (into r); partial ||vn||^2
template <typename T>
__global__ void k_mr_lanczos(KrylovArgs a, T* vn, const T* v, const T* vprev, const T* q, const T* C) {
  __shared__ double red[40];
  __shared__ T cs[64];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const SolveState S = a.st[ch.pair];
  if (!S.active) return;
  const PairDev pr = a.pairs[ch.pair];
  const int s = a.s_k[ch.pair];
  if ((int)threadIdx.x < s) cs[threadIdx.x] = (T)a.c[ch.pair * a.SMAX + threadIdx.x];
  __syncthreads();
  const T* Cb = C + pr.off * a.SMAX;
  const T al = (T)S.alpha, be = (T)S.beta_l;
  Accum<T> acc;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    T ccv = 0;
    for (int j = 0; j < s; ++j) ccv = fma(cs[j], Cb[(long long)j * pr.n + li], ccv);
    const T x = q[gi] - ccv - al * v[gi] - be * vprev[gi];
    vn[gi] = x;
    acc.add(x * x);
  }
  const double tot = block_total<kChunkThreads>(acc, red);
  if (threadIdx.x == 0) a.cpart[blockIdx.x] = tot;
}

// beta_{k+1}, the Givens rotation of step k, zeta_k, the s-vector recurrences and the stopping test
__global__ void k_mr_scalar2(KrylovArgs a, int stop_nsc, int* flag) {
  __shared__ double sh[8];
  __shared__ double bt[64];
  const int k = blockIdx.x;
  if (!a.st[k].active) return;
  const PairDev pr = a.pairs[k];
  const int s = a.s_k[k];
  const int nz = (stop_nsc && a.hasz[k]) ? s : 0;
  double t = 0.0;
  if (threadIdx.x < 32) {
    for (int u = pr.cbeg + (int)threadIdx.x; u < pr.cend; u += 32) t += a.cpart[u];
    t = warp_sum(t);
  }
  if (threadIdx.x == 0) {
    SolveState S = a.st[k];
    const double bn = sqrt(fmax(t, 0.0));
    const double gam = S.sm2 * S.beta_l;
    const double del = S.cm1 * S.cm2 * S.beta_l + S.sm1 * S.alpha;
    const double eps = -S.sm1 * S.cm2 * S.beta_l + S.cm1 * S.alpha;
    const double et = hypot(eps, bn);
    const double ck = et > 0.0 ? eps / et : 1.0, sk = et > 0.0 ? bn / et : 0.0;
    const double zprev = S.zeta;
    S.zeta = -sk * zprev;
    S.gam = gam;
    S.del = del;
    S.inv_et = et > 0.0 ? 1.0 / et : 0.0;
    S.coef = ck * zprev;
    S.inv_bn = bn > 0.0 ? 1.0 / bn : 0.0;
    S.cm2 = S.cm1;
    S.sm2 = S.sm1;
    S.cm1 = ck;
    S.sm1 = sk;
    S.beta_l = bn;
    S.iters += 1;
    if (!(et > 0.0) || !isfinite(et)) {
      S.active = 0;
      S.status = BL_EBREAKDOWN;
      S.coef = 0.0;
    }
    a.st[k] = S;
    sh[0] = S.gam;
    sh[1] = S.del;
    sh[2] = S.inv_et;
    sh[3] = S.coef;
  }
  __syncthreads();
  const double gam = sh[0], del = sh[1], iet = sh[2], coef = sh[3];
  // beta~_k = (C^T H v_k - gamma beta~_{k-2} - delta beta~_{k-1}) / eps~;  z -= c_k zeta_{k-1} beta~_k
  for (int m = threadIdx.x; m < s; m += blockDim.x) {
    const size_t i = (size_t)k * a.SMAX + m;
    const double b = (a.c[i] - gam * a.b2[i] - del * a.b1[i]) * iet;
    a.b2[i] = a.b1[i];
    a.b1[i] = b;
    a.zc[i] -= coef * b;
    bt[m] = b;
  }
  __syncthreads();
  // Z^T Hvt_k = (Z^T H v_k - gamma Z^T Hvt_{k-2} - delta Z^T Hvt_{k-1}) / eps~;
  // Z^T res -= c_k zeta_{k-1} (Z^T Hvt_k - (Z^T C) beta~_k)
  for (int m = threadIdx.x; m < nz; m += blockDim.x) {
    const size_t i = (size_t)k * a.SMAX + m;
    const double h = (a.e[i] - gam * a.h2[i] - del * a.h1[i]) * iet;
    a.h2[i] = a.h1[i];
    a.h1[i] = h;
    double zc = 0.0;
    for (int j = 0; j < s; ++j) zc += a.ztc[((size_t)k * a.SMAX + m) * a.SMAX + j] * bt[j];
    a.ztr[i] -= coef * (h - zc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SolveState S = a.st[k];
    if (S.active) {
      if (nz > 0) {
        double z2 = 0.0;
        for (int m = 0; m < nz; ++m) z2 += a.ztr[k * a.SMAX + m] * a.ztr[k * a.SMAX + m];
        S.est = sqrt(z2);
      } else {
        S.est = fabs(S.zeta);
      }
      S.rho = S.zeta * S.zeta;
      if (!isfinite(S.est)) {
        S.active = 0;
        S.status = BL_EBREAKDOWN;
      } else if (S.est < S.tol || S.beta_l == 0.0) {
        S.active = 0;
      } else if (S.iters >= S.maxit) {
        S.active = 0;
        S.status = BL_ENOCONV;
      }
      a.st[k] = S;
      if (S.active) atomicAdd(flag, 1);
    }
  }
}

// vt_k = (v_k - gamma vt_{k-2} - delta vt_{k-1}) / eps~; w += c_k zeta_{k-1} vt_k; V[:, k] = v_k;
// v_{k-1} <- v_k; v_{k+1} = vn / beta_{k+1}.  Runs for the pairs active at the start of the step.
template <typename T>
__global__ void k_mr_update(KrylovArgs a, const int* itmask, T* w, T* v, T* vprev, const T* vn, T* y1, T* y2,
                            T* V, int store) {
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!itmask[ch.pair]) return;
  const SolveState S = a.st[ch.pair];
  const PairDev pr = a.pairs[ch.pair];
  T* Vc = store ? V + pr.off * a.KMAX + (long long)((S.iters - 1) % a.KMAX) * pr.n : nullptr;
  const T gam = (T)S.gam, del = (T)S.del, iet = (T)S.inv_et, coef = (T)S.coef, ibn = (T)S.inv_bn;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    const T vk = v[gi];
    const T yo1 = y1[gi];
    const T y = (vk - gam * y2[gi] - del * yo1) * iet;
    w[gi] = fma(coef, y, w[gi]);
    y2[gi] = yo1;
    y1[gi] = y;
    if (store) Vc[li] = vk;
    vprev[gi] = vk;
    v[gi] = vn[gi] * ibn;
  }
}

// WHILE-node condition: another body run while some pair is active and the hard cap is not reached.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* flag, int* loop) {
  const int ran = ++loop[0];
  cudaGraphSetConditional(h, (*flag > 0 && ran < loop[1]) ? 1u : 0u);
}

template <typename F>
static bl_status build_krylov_graph(bl_problem* P, const KrylovGraphKey& key, F&& iteration) {
  destroy_krylov_graph(P);
  if (!P->cstream) BL_CUDA_TRY(cudaStreamCreateWithFlags(&P->cstream, cudaStreamNonBlocking));
  KrylovGraph* G = new KrylovGraph();
  G->key = key;
  P->kgraph = G;
  BL_CUDA_TRY(cudaGraphCreate(&G->graph, 0));
  cudaGraphConditionalHandle h;
  BL_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, G->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  BL_CUDA_TRY(cudaGraphAddNode(&node, G->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  // capture one iteration into the body on a private stream (capture only records)
  cudaStream_t user = P->stream;
  const bool prof = P->prof;
  const int64_t l0 = P->launches;
  P->stream = P->cstream;
  P->prof = false;
  P->capturing = true;
  bl_status st = BL_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(P->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = iteration();
    if (st == BL_OK) {
      k_loop_cond<<<1, 1, 0, P->stream>>>(h, P->d_flag, P->d_loop);
      ++P->launches;
      e = cudaGetLastError();
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(P->stream, &out);
    if (e == cudaSuccess) e = e2;
  }
  G->body_kernels = (int)(P->launches - l0);
  P->launches = l0;
  P->stream = user;
  P->prof = prof;
  P->capturing = false;
  if (st != BL_OK) {
    destroy_krylov_graph(P);
    return st;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  if (e != cudaSuccess) {
    destroy_krylov_graph(P);
    return fail(BL_ECUDA, std::string("Krylov graph: ") + cudaGetErrorString(e));
  }
  return BL_OK;
}

void destroy_krylov_graph(bl_problem* P) {
  destroy_lbfgs_graph(P);
  if (!P->kgraph) return;
  if (P->kgraph->exec) cudaGraphExecDestroy(P->kgraph->exec);
  if (P->kgraph->graph) cudaGraphDestroy(P->kgraph->graph);
  delete P->kgraph;
  P->kgraph = nullptr;
}

__global__ void k_copy_active(const SolveState* st, int* out, int K) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) out[k] = st[k].active;
}

template <typename T>
static bl_status solve_impl(bl_problem* P, const int* mask_host, const bl_krylov_opts* o, const void* g,
                            const double* nsc_scale, std::vector<bl_solve_info>& info) {
  const int K = P->K;
  const bool minres = o->method == BL_SOLVE_MINRES || o->method == BL_SOLVE_RMINRES;
  const bool recyc = o->method == BL_SOLVE_RCG || o->method == BL_SOLVE_RMINRES;
  // effective recycle dims and NSC flags for this solve
  std::vector<int> s_eff(K, 0), hz_eff(K, 0);
  for (int k = 0; k < K; ++k) {
    if (!mask_host[k]) continue;
    s_eff[k] = recyc ? P->s_k[k] : 0;
    hz_eff[k] = (recyc && o->stop == BL_STOP_NSC && P->hz_k[k]) ? 1 : 0;
  }
  if (minres && !P->mv_prev) {
    const size_t nb = (size_t)P->n_tot * P->esz;
    bl_status sa = dalloc(&P->mv_prev, nb);
    if (sa == BL_OK) sa = dalloc(&P->my1, nb);
    if (sa == BL_OK) sa = dalloc(&P->my2, nb);
    if (sa == BL_OK) sa = dalloc((void**)&P->mrs, (size_t)4 * K * std::max(P->SMAX, 1) * sizeof(double));
    if (sa != BL_OK) return sa;
  }
  int* d_seff = P->d_cols;          // reuse: per-pair ints
  int* d_hz = P->d_cols + K;
  const int* d_nohz = P->d_zero;    // zeros: no Z^T q in the Hessian-action epilogue
  BL_CUDA_TRY(cudaMemcpyAsync(d_seff, s_eff.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync(d_hz, hz_eff.data(), K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  double* d_scale = P->vals;        // K doubles
  if (nsc_scale)
    BL_CUDA_TRY(cudaMemcpyAsync(d_scale, nsc_scale, K * sizeof(double), cudaMemcpyHostToDevice, P->stream));

  bl_status st = ensure_cpart(P, (size_t)P->n_chunks * (1 + 2 * P->SMAX));
  if (st != BL_OK) return st;
  const bool fused = hvp_fused_dots(P);
  if (fused) {
    st = ensure_tpart(P, (size_t)P->n_tiles * (1 + 2 * P->SMAX));
    if (st != BL_OK) return st;
  }
  KrylovArgs a{};
  a.pairs = P->d_pairs;
  a.chunks = P->d_chunks;
  a.st = P->st;
  a.s_k = d_seff;
  a.hasz = d_hz;
  a.SMAX = P->SMAX;
  a.KMAX = P->KMAX;
  a.c = P->c;
  a.zc = P->zc;
  a.e = P->e;
  a.ztr = P->ztr;
  a.ztc = P->ztc;
  a.cpart = P->cpart;
  a.tpart = P->tpart;
  a.n_tiles = P->n_tiles;
  a.n_chunks = P->n_chunks;
  a.lanczos = (o->store_basis == BL_STORE_LANCZOS && P->KMAX > 0) ? 1 : 0;
  a.lz_alpha = P->lz_alpha;
  a.lz_rho = P->lz_rho;
  a.lz_c = P->lz_c;
  a.nbytes = bytes_counter(P, BL_KC_KRYLOV_VEC);
  if (minres) {
    const size_t ks = (size_t)K * std::max(P->SMAX, 1);
    a.b1 = P->mrs;
    a.b2 = P->mrs + ks;
    a.h1 = P->mrs + 2 * ks;
    a.h2 = P->mrs + 3 * ks;
  }
  const int* mask = P->d_active;
  T* w = (T*)P->w;
  T* r = (T*)P->r;
  T* p = (T*)P->pv;
  T* q = (T*)P->q;
  const T* U = (const T*)P->U;
  const T* C = (const T*)P->C;
  const T* Z = (const T*)P->Z;
  const bool warm = o->warm_start != 0;

  // ---- init ----
  if (warm) {
    st = launch_hvp(P, w, q, 0, 0, mask, nullptr, nullptr);
    if (st != BL_OK) return st;
  }
  {
  ProfScope ps(P, BL_KC_KRYLOV);
  k_init_r<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, (const T*)g, q, r, w, C, warm ? 1 : 0, mask);
  BL_LAUNCH_CHECK(P);
  k_scalar_init1<<<K, 128, 0, P->stream>>>(a, mask);
  BL_LAUNCH_CHECK(P);
  k_init2<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, w, r, p, U, C, Z, mask);
  BL_LAUNCH_CHECK(P);
  BL_CUDA_TRY(cudaMemsetAsync(P->d_flag, 0, sizeof(int), P->stream));
  k_scalar_init2<<<K, 128, 0, P->stream>>>(a, mask, o->stop == BL_STOP_NSC ? 1 : 0, o->tol, o->relative,
                                           nsc_scale ? d_scale : nullptr, o->maxit, P->d_flag);
  BL_LAUNCH_CHECK(P);
  if (minres) {
    k_mr_start<<<K, 64, 0, P->stream>>>(a, mask);
    BL_LAUNCH_CHECK(P);
    k_mr_vinit<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, p, (T*)P->mv_prev, (T*)P->my1, (T*)P->my2, mask);
    BL_LAUNCH_CHECK(P);
  }
  }
  BL_CUDA_TRY(cudaMemcpyAsync(P->h_flag, P->d_flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));

  // ---- iterations ----
  // the per-pair `active` flags gate every kernel; the loop ends when no pair is active
  int* d_itmask = P->d_active + K; // per-pair active copy for the stencil mask
  const int store = P->KMAX > 0 ? (o->store_basis == BL_STORE_LANCZOS ? 2 : (o->store_basis ? 1 : 0)) : 0;
  const int nsc = o->stop == BL_STOP_NSC ? 1 : 0;
  // dot products of the unfused path: all components of a chunk per CTA for aligned FP32 problems
  auto launch_dots = [&](const KrylovArgs& a0) -> bl_status {
    if (sizeof(T) == 4 && P->vec4)
      k_dots_v4<<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a0, (const float*)(const void*)p,
                                                               (const float*)(const void*)q,
                                                               (const float*)(const void*)C,
                                                               (const float*)(const void*)Z);
    else
      k_dots<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a0, p, q, C, Z);
    BL_LAUNCH_CHECK(P);
    return BL_OK;
  };
  auto iteration = [&]() -> bl_status {
    {
      ProfScope ps(P, BL_KC_KRYLOV);
      k_copy_active<<<1, 128, 0, P->stream>>>(P->st, d_itmask, K);
      BL_LAUNCH_CHECK(P);
    }
    bl_status s2 = launch_hvp(P, p, q, 0, 0, d_itmask, fused ? d_seff : nullptr, fused ? d_nohz : nullptr);
    if (s2 != BL_OK) return s2;
    if (!fused) {
      ProfScope ps(P, BL_KC_KRYLOV_VEC);
      KrylovArgs a0 = a;
      a0.hasz = d_nohz;   // the NSC sums come from the update pass
      if ((s2 = launch_dots(a0)) != BL_OK) return s2;
    }
    {
      ProfScope ps(P, BL_KC_KRYLOV);
      k_scalar1<<<K, 128, 0, P->stream>>>(a, fused ? 1 : 0);
      BL_LAUNCH_CHECK(P);
    }
    {
      ProfScope ps(P, BL_KC_KRYLOV_VEC);
      if (sizeof(T) == 4 && P->vec4)
        k_update_v4<<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, (float*)(void*)w, (float*)(void*)r,
                                                                   (const float*)(const void*)p,
                                                                   (const float*)(const void*)q,
                                                                   (const float*)(const void*)C,
                                                                   (const float*)(const void*)Z, (float*)P->V, store,
                                                                   nsc);
      else
        k_update<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, w, r, p, q, C, Z, (T*)P->V, store, nsc);
      BL_LAUNCH_CHECK(P);
    }
    {
      ProfScope ps(P, BL_KC_KRYLOV);
      BL_CUDA_TRY(cudaMemsetAsync(P->d_flag, 0, sizeof(int), P->stream));
      k_scalar2<<<K, 32, 0, P->stream>>>(a, nsc, P->d_flag);
      BL_LAUNCH_CHECK(P);
    }
    {
      ProfScope ps(P, BL_KC_KRYLOV_VEC);
      k_pupdate<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, r, p);
      BL_LAUNCH_CHECK(P);
    }
    return BL_OK;
  };
  // MINRES step: q = H v_k (with v^T q, C^T q and, for the NSC rule, Z^T q), Lanczos vector,
  // rotation and stopping test, direction and solution update
  auto mr_iteration = [&]() -> bl_status {
    {
      ProfScope ps(P, BL_KC_KRYLOV);
      k_copy_active<<<1, 128, 0, P->stream>>>(P->st, d_itmask, K);
      BL_LAUNCH_CHECK(P);
    }
    const int* zflags = nsc ? d_hz : d_nohz;
    bl_status s2 = launch_hvp(P, p, q, 0, 0, d_itmask, fused ? d_seff : nullptr, fused ? zflags : nullptr);
    if (s2 != BL_OK) return s2;
    ProfScope ps(P, BL_KC_KRYLOV);
    if (!fused) {
      KrylovArgs a0 = a;
      a0.hasz = zflags;
      if ((s2 = launch_dots(a0)) != BL_OK) return s2;
    }
    k_mr_scalar1<<<K, 128, 0, P->stream>>>(a, fused ? 1 : 0, nsc);
    BL_LAUNCH_CHECK(P);
    k_mr_lanczos<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, r, p, (const T*)P->mv_prev, q, C);
    BL_LAUNCH_CHECK(P);
    BL_CUDA_TRY(cudaMemsetAsync(P->d_flag, 0, sizeof(int), P->stream));
    k_mr_scalar2<<<K, 64, 0, P->stream>>>(a, nsc, P->d_flag);
    BL_LAUNCH_CHECK(P);
    k_mr_update<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, d_itmask, w, p, (T*)P->mv_prev, r, (T*)P->my1,
                                                                 (T*)P->my2, (T*)P->V, store);
    BL_LAUNCH_CHECK(P);
    return BL_OK;
  };
  auto step = [&]() -> bl_status { return minres ? mr_iteration() : iteration(); };
  bool use_graph = *P->h_flag > 0 && o->graph && !P->prof && !P->graph_failed;
  if (use_graph) {
    const KrylovGraphKey key{fused, store, nsc, minres ? 1 : 0, P->tpart, P->cpart, P->V};
    if (!P->kgraph || !(P->kgraph->key == key)) {
      if (build_krylov_graph(P, key, step) != BL_OK) {
        // the stream path below runs the same kernels; remember not to retry the capture
        P->graph_error = error_copy();
        P->graph_failed = true;
        use_graph = false;
        (void)cudaGetLastError();
      }
    }
  }
  P->graph_used = use_graph;
  if (use_graph) {
    // one graph launch runs the whole loop: a WHILE node whose body is one iteration, its
    // condition set on the device from the any-active count (the iteration caps of every pair
    // bound it; a loop counter adds a hard cap of maxit + 1 body runs)
    const int cap[2] = {0, o->maxit + 1};
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_loop, cap, sizeof(cap), cudaMemcpyHostToDevice, P->stream));
    BL_CUDA_TRY(cudaGraphLaunch(P->kgraph->exec, P->stream));
    int ran = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(&ran, P->d_loop, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    P->launches += (int64_t)ran * P->kgraph->body_kernels + 1;
  } else {
    for (int it = 0; it < o->maxit && *P->h_flag > 0; ++it) {
      st = step();
      if (st != BL_OK) return st;
      BL_CUDA_TRY(cudaMemcpyAsync(P->h_flag, P->d_flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
      BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    }
  }
  {
    ProfScope ps(P, BL_KC_KRYLOV);
    if (a.lanczos) {
      k_store_last<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, r, (T*)P->V, mask);
      BL_LAUNCH_CHECK(P);
    }
    k_finalize<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(a, w, U, mask);
    BL_LAUNCH_CHECK(P);
  }

  // ---- results ----
  std::vector<SolveState> hs(K);
  BL_CUDA_TRY(cudaMemcpyAsync(hs.data(), P->st, K * sizeof(SolveState), cudaMemcpyDeviceToHost, P->stream));
  std::vector<double> hztr((size_t)K * P->SMAX);
  if (P->SMAX)
    BL_CUDA_TRY(cudaMemcpyAsync(hztr.data(), P->ztr, hztr.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  info.assign(K, bl_solve_info{});
  for (int k = 0; k < K; ++k) {
    if (!mask_host[k]) continue;
    const SolveState& S = hs[k];
    info[k].iters = S.iters;
    info[k].status = S.status;
    info[k].resid = std::sqrt(std::max(S.rho, 0.0));
    double z2 = 0.0;
    if (hz_eff[k])
      for (int m = 0; m < s_eff[k]; ++m) z2 += hztr[(size_t)k * P->SMAX + m] * hztr[(size_t)k * P->SMAX + m];
    info[k].nsc_est = std::sqrt(z2);
    info[k].rhs_norm = std::sqrt(std::max(S.gnorm2, 0.0));
    if (o->store_basis && P->KMAX > 0) {
      // Lanczos record: v_0 .. v_{m-1} form the basis, v_m closes the relation
      P->kb_k[k] = a.lanczos ? std::min(S.iters, P->KMAX - 1) : std::min(S.iters, P->KMAX);
      P->head_k[k] = S.iters;
      P->lz_k[k] = a.lanczos;
      P->lz_u[k] = s_eff[k] == P->s_k[k] ? 1 : 0;
    }
  }
  return BL_OK;
}

bl_status run_hessian_solve(bl_problem* P, const int* mask_host, const bl_krylov_opts* o, const void* g,
                            const double* nsc_scale, std::vector<bl_solve_info>& info) {
  const bl_status st = P->prec == BL_FP32 ? solve_impl<float>(P, mask_host, o, g, nsc_scale, info)
                                          : solve_impl<double>(P, mask_host, o, g, nsc_scale, info);
  const bl_status ke = check_kernel_error(P);
  return ke != BL_OK ? ke : st;
}

}  // namespace bl
