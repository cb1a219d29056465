// Batched lower-level solve: L-BFGS with Armijo backtracking (Section 5.1), all pairs together.
//
// Per iteration and pair: the L-BFGS direction d = -H g over the m most recent (s, y) pairs with
// initial scaling gamma = s^T y / y^T y of the newest pair (1 before any pair exists).  The
// direction is formed in the compact representation of the L-BFGS matrix (Byrd, Nocedal and
// Schnabel 1994), algebraically the two-loop recursion's result:
//   H g = gamma g + S R^{-T} ((D + gamma Y^T Y) R^{-1} S^T g - gamma Y^T g) - gamma Y R^{-1} S^T g,
// R the upper triangle of S^T Y and D its diagonal (columns oldest first), so one pass forms the 4m
// dot products S^T g, Y^T g, S^T y_new, Y^T y_new, an m x m FP64 solve per pair gives the
// coefficients, and a second pass forms d.  Then a
// descent check (restart from -grad if g^T d >= 0), Armijo backtracking with c1 = 1e-4 from
// step 1 halving the step (an optional slack eps |Phi| on the sufficient-decrease test lets FP32
// runs accept steps whose change is below FP32 resolution of Phi), and the pair update only
// when s^T y > 1e-12 ||s|| ||y||.
// Vectors are FP32 or FP64 by problem precision; every scalar is FP64 on the device.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "device.cuh"

namespace bl {

struct LbArgs {
  const PairDev* pairs;
  const ChunkDev* chunks;
  LbfgsState* st;
  int MH;             // memory m; the ring holds m + 1 slots
  double* cpart;      // per chunk partial sums
  double *sy, *yy;    // K x (m + 1)^2 by slot
  double *cs, *cy;    // K x (m + 1) direction coefficients by slot
};

// Slot of the i-th oldest valid pair (ring of RS = m + 1 slots).
__device__ __forceinline__ int lb_age_slot(const LbfgsState& S, int i, int RS) {
  return (S.hist_head - S.hist_count + i + 2 * RS) % RS;
}

// Pass A: per chunk partial sums [4 * RS * chunk + 4 i + q] for the i-th oldest pair, q = 0..3:
// s_i^T g, y_i^T g, s_i^T y_new, y_i^T y_new (y_new: the newest stored y).
template <typename T>
__global__ void k_lb_dots(LbArgs a, const T* g, const T* Sm, const T* Ym, double* part) {
  __shared__ double red[8][4 * (kMaxHistory + 1)];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbDir || S.hist_count == 0) return;
  const PairDev pr = a.pairs[ch.pair];
  const int RS = a.MH + 1, c = S.hist_count;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* yn = Ym + pr.off * RS + (long long)lb_age_slot(S, c - 1, RS) * pr.n;
  for (int i = 0; i < c; ++i) {
    const int sl = lb_age_slot(S, i, RS);
    const T* sc = Sm + pr.off * RS + (long long)sl * pr.n;
    const T* yc = Ym + pr.off * RS + (long long)sl * pr.n;
    Accum<T> sg, yg, sy, yy;
    for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
      const long long li = ch.start + t;
      const T sv = sc[li], yv = yc[li], gv = g[pr.off + li], ynv = yn[li];
      sg.add(sv * gv);
      yg.add(yv * gv);
      sy.add(sv * ynv);
      yy.add(yv * ynv);
    }
    const double v0 = warp_total(sg), v1 = warp_total(yg), v2 = warp_total(sy), v3 = warp_total(yy);
    if (lane == 0) {
      red[wid][4 * i + 0] = v0;
      red[wid][4 * i + 1] = v1;
      red[wid][4 * i + 2] = v2;
      red[wid][4 * i + 3] = v3;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 4 * c; q += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kChunkThreads / 32; ++w) t += red[w][q];
    part[(size_t)blockIdx.x * 4 * RS + q] = t;
  }
}

// Per pair: update S^T Y and Y^T Y for the newest pair, solve with R (FP64) and write the direction
// coefficients by slot: d = -gamma g + sum_i cs_i s_i + cy_i y_i.
__global__ void k_lb_compact(LbArgs a, const double* part) {
  constexpr int M = kMaxHistory;
  __shared__ double v[4 * (M + 1)];
  __shared__ double R[M][M], YY[M][M];   // by age: R = upper triangle of S^T Y, YY = Y^T Y
  __shared__ double u[M], w[M], top[M];
  __shared__ int sl[M];
  const int k = blockIdx.x;
  const LbfgsState S = a.st[k];
  if (!S.active || S.phase != kLbDir) return;
  const PairDev pr = a.pairs[k];
  const int RS = a.MH + 1, c = S.hist_count;
  double* sy = a.sy + (size_t)k * RS * RS;    // sy[i * RS + j] = s_i^T y_j (slots)
  double* yy = a.yy + (size_t)k * RS * RS;
  double* cs = a.cs + (size_t)k * RS;
  double* cy = a.cy + (size_t)k * RS;
  // chunk partials: a warp per value, its lanes over the pair's chunks
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int q = wid; q < 4 * c; q += nwarp) {
    double t = 0.0;
    for (int un = pr.cbeg + lane; un < pr.cend; un += 32) t += part[(size_t)un * 4 * RS + q];
    t = warp_sum(t);
    if (lane == 0) v[q] = t;
  }
  for (int j = threadIdx.x; j < RS; j += blockDim.x) cs[j] = cy[j] = 0.0;
  for (int i = threadIdx.x; i < c; i += blockDim.x) sl[i] = lb_age_slot(S, i, RS);
  __syncthreads();
  if (c == 0) return;
  // the newest pair's column of S^T Y and row / column of Y^T Y (slots, kept across iterations)
  const int nw = sl[c - 1];
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    sy[sl[i] * RS + nw] = v[4 * i + 2];
    yy[sl[i] * RS + nw] = v[4 * i + 3];
    yy[nw * RS + sl[i]] = v[4 * i + 3];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < c * c; idx += blockDim.x) {
    const int i = idx / c, j = idx - (idx / c) * c;
    R[i][j] = (j >= i) ? sy[sl[i] * RS + sl[j]] : 0.0;
    YY[i][j] = yy[sl[i] * RS + sl[j]];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double gam = S.gamma;
  // u = R^{-1} (S^T g)
  for (int i = c - 1; i >= 0; --i) {
    double t = v[4 * i + 0];
    for (int j = i + 1; j < c; ++j) t -= R[i][j] * u[j];
    u[i] = t / R[i][i];
  }
  // w = (D + gamma Y^T Y) u - gamma Y^T g
  for (int i = 0; i < c; ++i) {
    double t = R[i][i] * u[i] - gam * v[4 * i + 1];
    for (int j = 0; j < c; ++j) t += gam * YY[i][j] * u[j];
    w[i] = t;
  }
  // top = R^{-T} w
  for (int i = 0; i < c; ++i) {
    double t = w[i];
    for (int j = 0; j < i; ++j) t -= R[j][i] * top[j];
    top[i] = t / R[i][i];
  }
  for (int i = 0; i < c; ++i) {
    cs[sl[i]] = -top[i];
    cy[sl[i]] = gam * u[i];
  }
}

// Pass B: d = -gamma g + sum_i cs_i s_i + cy_i y_i; partial g^T d.
template <typename T>
__global__ void k_lb_dir(LbArgs a, T* d, const T* g, const T* Sm, const T* Ym, double* part) {
  __shared__ double red[40];
  __shared__ T cf[2 * (kMaxHistory + 1)];
  __shared__ int sl[kMaxHistory + 1];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbDir) return;
  const PairDev pr = a.pairs[ch.pair];
  const int RS = a.MH + 1, c = S.hist_count;
  if ((int)threadIdx.x < c) {
    const int s_ = lb_age_slot(S, threadIdx.x, RS);
    sl[threadIdx.x] = s_;
    cf[2 * threadIdx.x] = (T)a.cs[(size_t)ch.pair * RS + s_];
    cf[2 * threadIdx.x + 1] = (T)a.cy[(size_t)ch.pair * RS + s_];
  }
  __syncthreads();
  const T mg = (T)(-S.gamma);
  Accum<T> acc;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    const T gv = g[gi];
    T x = mg * gv;
    for (int i = 0; i < c; ++i) {
      const long long col = pr.off * RS + (long long)sl[i] * pr.n + li;
      x = fma(cf[2 * i], Sm[col], fma(cf[2 * i + 1], Ym[col], x));
    }
    d[gi] = x;
    acc.add(gv * x);
  }
  const double tot = block_total<kChunkThreads>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// g^T d from the partials of the direction pass; descent check (restart flag if >= 0)
__global__ void k_lb_gtd(LbArgs a, const double* part) {
  const int k = blockIdx.x;
  LbfgsState& S = a.st[k];
  if (!S.active || S.phase != kLbDir) return;
  const PairDev pr = a.pairs[k];
  double sum = 0.0;
  for (int u = pr.cbeg + (int)threadIdx.x; u < pr.cend; u += 32) sum += part[u];
  sum = warp_sum(sum);
  if (threadIdx.x != 0) return;
  S.gtd = sum;
  S.accepted = (sum >= 0.0) ? -1 : 0;   // -1: not a descent direction
}

// d = -g for pairs flagged by the descent check; history cleared
template <typename T>
__global__ void k_lb_restart(LbArgs a, T* d, const T* g) {
  __shared__ double red[40];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbDir || S.accepted != -1) return;
  const PairDev pr = a.pairs[ch.pair];
  Accum<T> acc;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long gi = pr.off + ch.start + t;
    d[gi] = -g[gi];
    acc.add(-g[gi] * g[gi]);
  }
  const double tot = block_total<kChunkThreads>(acc, red);
  if (threadIdx.x == 0) a.cpart[blockIdx.x] = tot;
}

__global__ void k_lb_restart_fix(LbArgs a) {
  const int k = blockIdx.x;
  LbfgsState& S = a.st[k];
  if (!S.active || S.phase != kLbDir || S.accepted != -1) return;
  const PairDev pr = a.pairs[k];
  double sum = 0.0;
  for (int u = pr.cbeg + (int)threadIdx.x; u < pr.cend; u += 32) sum += a.cpart[u];
  sum = warp_sum(sum);
  if (threadIdx.x != 0) return;
  S.gtd = sum;
  S.hist_count = 0;
  S.accepted = 0;
}

// pairs with a new direction start their line search at t = 1; pairs still searching continue
__global__ void k_lb_begin_search(LbArgs a, int* search_mask) {
  const int k = blockIdx.x;
  LbfgsState& S = a.st[k];
  if (threadIdx.x != 0) return;
  if (S.active && S.phase == kLbDir) {
    S.t = 1.0;
    S.backtracks = 0;
    S.accepted = 0;
    S.phase = kLbTrial;
  }
  search_mask[k] = S.active && S.phase == kLbTrial;
}

// x_t = x + t d for searching pairs
template <typename T>
__global__ void k_lb_trial(LbArgs a, const int* search_mask, T* xt, const T* x, const T* d) {
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!search_mask[ch.pair]) return;
  const PairDev pr = a.pairs[ch.pair];
  const T t = (T)a.st[ch.pair].t;
  for (int i = threadIdx.x; i < ch.len; i += blockDim.x) {
    const long long gi = pr.off + ch.start + i;
    xt[gi] = fma(t, d[gi], x[gi]);
  }
}

// Armijo test on the trial values (with the relative slack of the options); halve the step of
// the pairs that fail
__global__ void k_lb_armijo(LbArgs a, int* search_mask, const double* vals, double l2, int max_bt, double slack,
                            int* flag) {
  const int k = blockIdx.x;
  if (threadIdx.x != 0 || !search_mask[k]) return;
  LbfgsState& S = a.st[k];
  const double ft = vals[k * 3 + 0] + vals[k * 3 + 1] + 0.5 * l2 * vals[k * 3 + 2];
  if (ft <= S.f + 1e-4 * S.t * S.gtd + slack * fabs(S.f) || S.backtracks + 1 >= max_bt) {
    S.f_trial = ft;
    S.accepted = 1;
    S.phase = kLbAccepted;
    search_mask[k] = 0;
  } else {
    S.t *= 0.5;
    S.backtracks += 1;
    if (flag) atomicAdd(flag, 1);
  }
}

// store s = x_t - x, y = g_t - g in the head slot, x = x_t, g = g_t; partials s^T y, y^T y, s^T s, g^T g
template <typename T>
__global__ void k_lb_accept(LbArgs a, T* x, T* g, const T* xt, const T* gt, T* Sm, T* Ym) {
  __shared__ double red[40];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbAccepted) return;
  const PairDev pr = a.pairs[ch.pair];
  T* sc = Sm + pr.off * (a.MH + 1) + (long long)S.hist_head * pr.n;
  T* yc = Ym + pr.off * (a.MH + 1) + (long long)S.hist_head * pr.n;
  Accum<T> sy, yy, ss, gg;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long li = ch.start + t, gi = pr.off + li;
    const T xn = xt[gi], gn = gt[gi];
    const T sv = xn - x[gi], yv = gn - g[gi];
    sc[li] = sv;
    yc[li] = yv;
    x[gi] = xn;
    g[gi] = gn;
    sy.add(sv * yv);
    yy.add(yv * yv);
    ss.add(sv * sv);
    gg.add(gn * gn);
  }
  const double t0 = block_total<kChunkThreads>(sy, red);
  const double t1 = block_total<kChunkThreads>(yy, red);
  const double t2 = block_total<kChunkThreads>(ss, red);
  const double t3 = block_total<kChunkThreads>(gg, red);
  if (threadIdx.x == 0) {
    a.cpart[(size_t)blockIdx.x * 4 + 0] = t0;
    a.cpart[(size_t)blockIdx.x * 4 + 1] = t1;
    a.cpart[(size_t)blockIdx.x * 4 + 2] = t2;
    a.cpart[(size_t)blockIdx.x * 4 + 3] = t3;
  }
}

// 128-bit versions of the four vector passes for FP32 problems whose images are multiples of 4
// pixels (every column start 16-byte aligned; a chunk is kChunk pixels, PB float4 per thread).
// Each thread keeps its blocks of g (and y_new) in registers and streams the history columns.
constexpr int kLbPB = kChunk / 4 / kChunkThreads;
static_assert(kLbPB * 4 * kChunkThreads == kChunk, "PB 128-bit blocks per thread");

__device__ __forceinline__ void add4(Accum<float>& acc, float4 u, float4 v) {
  acc.add(u.x * v.x);
  acc.add(u.y * v.y);
  acc.add(u.z * v.z);
  acc.add(u.w * v.w);
}

__global__ void __launch_bounds__(kChunkThreads) k_lb_dots_v4(LbArgs a, const float* g, const float* Sm,
                                                              const float* Ym, double* part) {
  __shared__ double red[kChunkThreads / 32][4 * (kMaxHistory + 1)];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbDir || S.hist_count == 0) return;
  const PairDev pr = a.pairs[ch.pair];
  const int RS = a.MH + 1, c = S.hist_count, nv = ch.len >> 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const float4* g4 = reinterpret_cast<const float4*>(g + pr.off + ch.start);
  const float4* yn4 =
      reinterpret_cast<const float4*>(Ym + pr.off * RS + (long long)lb_age_slot(S, c - 1, RS) * pr.n + ch.start);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 gv[kLbPB], ynv[kLbPB];
#pragma unroll
  for (int m = 0; m < kLbPB; ++m) {
    const int i = threadIdx.x + m * kChunkThreads;
    gv[m] = i < nv ? g4[i] : z4;
    ynv[m] = i < nv ? yn4[i] : z4;
  }
  for (int h = 0; h < c; ++h) {
    const long long col = pr.off * RS + (long long)lb_age_slot(S, h, RS) * pr.n + ch.start;
    const float4* s4 = reinterpret_cast<const float4*>(Sm + col);
    const float4* y4 = reinterpret_cast<const float4*>(Ym + col);
    Accum<float> sg, yg, sy, yy;
#pragma unroll
    for (int m = 0; m < kLbPB; ++m) {
      const int i = threadIdx.x + m * kChunkThreads;
      if (i < nv) {
        const float4 sv = s4[i], yv = y4[i];
        add4(sg, sv, gv[m]);
        add4(yg, yv, gv[m]);
        add4(sy, sv, ynv[m]);
        add4(yy, yv, ynv[m]);
      }
    }
    const double v0 = warp_total(sg), v1 = warp_total(yg), v2 = warp_total(sy), v3 = warp_total(yy);
    if (lane == 0) {
      red[wid][4 * h + 0] = v0;
      red[wid][4 * h + 1] = v1;
      red[wid][4 * h + 2] = v2;
      red[wid][4 * h + 3] = v3;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 4 * c; q += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kChunkThreads / 32; ++w) t += red[w][q];
    part[(size_t)blockIdx.x * 4 * RS + q] = t;
  }
}

__global__ void __launch_bounds__(kChunkThreads) k_lb_dir_v4(LbArgs a, float* d, const float* g, const float* Sm,
                                                             const float* Ym, double* part) {
  __shared__ double red[40];
  __shared__ float cf[2 * (kMaxHistory + 1)];
  __shared__ int sl[kMaxHistory + 1];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbDir) return;
  const PairDev pr = a.pairs[ch.pair];
  const int RS = a.MH + 1, c = S.hist_count, nv = ch.len >> 2;
  if ((int)threadIdx.x < c) {
    const int s_ = lb_age_slot(S, threadIdx.x, RS);
    sl[threadIdx.x] = s_;
    cf[2 * threadIdx.x] = (float)a.cs[(size_t)ch.pair * RS + s_];
    cf[2 * threadIdx.x + 1] = (float)a.cy[(size_t)ch.pair * RS + s_];
  }
  __syncthreads();
  const float mg = (float)(-S.gamma);
  const float4* g4 = reinterpret_cast<const float4*>(g + pr.off + ch.start);
  float4* d4 = reinterpret_cast<float4*>(d + pr.off + ch.start);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 gv[kLbPB], x[kLbPB];
#pragma unroll
  for (int m = 0; m < kLbPB; ++m) {
    const int i = threadIdx.x + m * kChunkThreads;
    gv[m] = i < nv ? g4[i] : z4;
    x[m] = make_float4(mg * gv[m].x, mg * gv[m].y, mg * gv[m].z, mg * gv[m].w);
  }
  for (int h = 0; h < c; ++h) {
    const long long col = pr.off * RS + (long long)sl[h] * pr.n + ch.start;
    const float4* s4 = reinterpret_cast<const float4*>(Sm + col);
    const float4* y4 = reinterpret_cast<const float4*>(Ym + col);
    const float cs_ = cf[2 * h], cy_ = cf[2 * h + 1];
#pragma unroll
    for (int m = 0; m < kLbPB; ++m) {
      const int i = threadIdx.x + m * kChunkThreads;
      if (i < nv) {
        const float4 sv = s4[i], yv = y4[i];
        x[m].x = fmaf(cs_, sv.x, fmaf(cy_, yv.x, x[m].x));
        x[m].y = fmaf(cs_, sv.y, fmaf(cy_, yv.y, x[m].y));
        x[m].z = fmaf(cs_, sv.z, fmaf(cy_, yv.z, x[m].z));
        x[m].w = fmaf(cs_, sv.w, fmaf(cy_, yv.w, x[m].w));
      }
    }
  }
  Accum<float> acc;
#pragma unroll
  for (int m = 0; m < kLbPB; ++m) {
    const int i = threadIdx.x + m * kChunkThreads;
    if (i < nv) {
      d4[i] = x[m];
      add4(acc, gv[m], x[m]);
    }
  }
  const double tot = block_total<kChunkThreads>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kChunkThreads) k_lb_trial_v4(LbArgs a, const int* search_mask, float* xt,
                                                               const float* x, const float* d) {
  const ChunkDev ch = a.chunks[blockIdx.x];
  if (!search_mask[ch.pair]) return;
  const PairDev pr = a.pairs[ch.pair];
  const float t = (float)a.st[ch.pair].t;
  const long long g0 = pr.off + ch.start;
  const float4* x4 = reinterpret_cast<const float4*>(x + g0);
  const float4* d4 = reinterpret_cast<const float4*>(d + g0);
  float4* t4 = reinterpret_cast<float4*>(xt + g0);
  for (int i = threadIdx.x; i < (ch.len >> 2); i += blockDim.x) {
    const float4 xv = x4[i], dv = d4[i];
    t4[i] = make_float4(fmaf(t, dv.x, xv.x), fmaf(t, dv.y, xv.y), fmaf(t, dv.z, xv.z), fmaf(t, dv.w, xv.w));
  }
}

__global__ void __launch_bounds__(kChunkThreads) k_lb_accept_v4(LbArgs a, float* x, float* g, const float* xt,
                                                                const float* gt, float* Sm, float* Ym) {
  __shared__ double red[kChunkThreads / 32][4];
  const ChunkDev ch = a.chunks[blockIdx.x];
  const LbfgsState S = a.st[ch.pair];
  if (!S.active || S.phase != kLbAccepted) return;
  const PairDev pr = a.pairs[ch.pair];
  const long long g0 = pr.off + ch.start;
  const long long col = pr.off * (a.MH + 1) + (long long)S.hist_head * pr.n + ch.start;
  float4* s4 = reinterpret_cast<float4*>(Sm + col);
  float4* y4 = reinterpret_cast<float4*>(Ym + col);
  float4* x4 = reinterpret_cast<float4*>(x + g0);
  float4* g4 = reinterpret_cast<float4*>(g + g0);
  const float4* xt4 = reinterpret_cast<const float4*>(xt + g0);
  const float4* gt4 = reinterpret_cast<const float4*>(gt + g0);
  Accum<float> sy, yy, ss, gg;
  for (int i = threadIdx.x; i < (ch.len >> 2); i += blockDim.x) {
    const float4 xn = xt4[i], gn = gt4[i], xo = x4[i], go = g4[i];
    const float4 sv = make_float4(xn.x - xo.x, xn.y - xo.y, xn.z - xo.z, xn.w - xo.w);
    const float4 yv = make_float4(gn.x - go.x, gn.y - go.y, gn.z - go.z, gn.w - go.w);
    s4[i] = sv;
    y4[i] = yv;
    x4[i] = xn;
    g4[i] = gn;
    add4(sy, sv, yv);
    add4(yy, yv, yv);
    add4(ss, sv, sv);
    add4(gg, gn, gn);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double v0 = warp_total(sy), v1 = warp_total(yy), v2 = warp_total(ss), v3 = warp_total(gg);
  if (lane == 0) {
    red[wid][0] = v0;
    red[wid][1] = v1;
    red[wid][2] = v2;
    red[wid][3] = v3;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kChunkThreads / 32; ++w) t += red[w][threadIdx.x];
    a.cpart[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// take the accepted steps (history, scaling, convergence test); count the pairs still running
__global__ void k_lb_post(LbArgs a, int maxit, int* flag) {
  const int k = blockIdx.x;
  LbfgsState& S = a.st[k];
  if (!S.active) return;
  if (S.phase == kLbAccepted) {
    const PairDev pr = a.pairs[k];
    double v[4] = {0, 0, 0, 0};
    for (int u = pr.cbeg + (int)threadIdx.x; u < pr.cend; u += 32)
      for (int c = 0; c < 4; ++c) v[c] += a.cpart[(size_t)u * 4 + c];
    for (int c = 0; c < 4; ++c) v[c] = warp_sum(v[c]);
    if (threadIdx.x != 0) return;
    const double sy = v[0], yy = v[1], ss = v[2], gg = v[3];
    if (sy > 1e-12 * sqrt(ss) * sqrt(yy)) {
      S.gamma = sy / yy;
      S.hist_head = (S.hist_head + 1) % (a.MH + 1);
      S.hist_count = min(S.hist_count + 1, a.MH);
    }
    if (S.hist_count == 0) S.gamma = 1.0;
    S.f = S.f_trial;
    S.gnorm = sqrt(gg);
    S.iters += 1;
    S.phase = kLbDir;
    if (!isfinite(S.f) || !isfinite(S.gnorm)) {
      S.active = 0;
      S.status = BL_EBREAKDOWN;
    } else if (S.gnorm <= S.gtol) {
      S.active = 0;
    } else if (S.iters >= maxit) {
      S.active = 0;
      S.status = BL_ENOCONV;
    }
  }
  if (threadIdx.x == 0 && S.active) atomicAdd(flag, 1);
}

__global__ void k_lb_init(LbArgs a, const int* mask, const double* vals, const double* gn2, const double* ay2,
                          double l2, double gtol, int relative, int* flag) {
  const int k = blockIdx.x;
  if (threadIdx.x != 0) return;
  LbfgsState& S = a.st[k];
  if (!mask[k]) {
    S.active = 0;
    return;
  }
  S.f = vals[k * 3 + 0] + vals[k * 3 + 1] + 0.5 * l2 * vals[k * 3 + 2];
  S.gnorm = sqrt(gn2[k]);
  S.gtol = relative ? gtol * 2.0 * sqrt(ay2[k]) : gtol;
  S.hist_count = 0;
  S.hist_head = 0;
  S.gamma = 1.0;
  S.iters = 0;
  S.status = BL_OK;
  S.phase = kLbDir;
  S.active = (S.gnorm > S.gtol) ? 1 : 0;
  if (!isfinite(S.f) || !isfinite(S.gnorm)) {
    S.active = 0;
    S.status = BL_EBREAKDOWN;
  }
  if (S.active) atomicAdd(flag, 1);
}

__global__ void k_lb_mask(const LbfgsState* st, int* out, int K) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) out[k] = st[k].active;
}

// WHILE-node condition of the L-BFGS loop: another body run while some pair is active and the
// run cap is not reached.
__global__ void k_lb_loop_cond(cudaGraphConditionalHandle h, const int* flag, int* loop) {
  const int ran = ++loop[0];
  cudaGraphSetConditional(h, (*flag > 0 && ran < loop[1]) ? 1u : 0u);
}

template <typename F>
static bl_status build_lbfgs_graph(bl_problem* P, const LbfgsGraphKey& key, F&& body) {
  destroy_lbfgs_graph(P);
  if (!P->cstream) BL_CUDA_TRY(cudaStreamCreateWithFlags(&P->cstream, cudaStreamNonBlocking));
  KrylovGraph* G = new KrylovGraph();
  P->lgraph = G;
  P->lgraph_key = key;
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
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  // capture one body run on a private stream (capture only records)
  cudaStream_t user = P->stream;
  const bool prof = P->prof;
  const int64_t l0 = P->launches;
  P->stream = P->cstream;
  P->prof = false;
  P->capturing = true;
  bl_status st = BL_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(P->stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = body();
    if (st == BL_OK) {
      k_lb_loop_cond<<<1, 1, 0, P->stream>>>(h, P->d_flag, P->d_loop);
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
    destroy_lbfgs_graph(P);
    return st;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  if (e != cudaSuccess) {
    destroy_lbfgs_graph(P);
    return fail(BL_ECUDA, std::string("L-BFGS graph: ") + cudaGetErrorString(e));
  }
  return BL_OK;
}

template <typename T>
static bl_status lbfgs_impl(bl_problem* P, const std::vector<int>& mask_host, const bl_lbfgs_opts* o,
                            std::vector<bl_solve_info>& info) {
  const int K = P->K, MH = P->MH;
  bl_status st = ensure_cpart(P, (size_t)P->n_chunks * (4 * (MH + 1) + 1));
  if (st != BL_OK) return st;
  LbArgs a{};
  a.pairs = P->d_pairs;
  a.chunks = P->d_chunks;
  a.st = P->lst;
  a.MH = MH;
  a.cpart = P->cpart;
  a.sy = P->lsy;
  a.yy = P->lyy;
  a.cs = P->lcs;
  a.cy = P->lcy;
  const int* mask = P->d_active;
  int* smask = P->d_active + K;
  T* x = (T*)P->lx;
  T* g = (T*)P->lg;
  T* d = (T*)P->ld;
  T* xt = (T*)P->lxt;
  T* gt = (T*)P->lgt;
  T* Sm = (T*)P->S;
  T* Ym = (T*)P->Yh;
  double* vals = P->vals;              // K x 3
  double* gn2 = P->vals + 3 * K;       // K
  double* ay2 = P->vals + 4 * K;       // K
  const double l2 = P->reg.l2_eps;
  const dim3 cg(P->n_chunks), ct(kChunkThreads);
  // 128-bit vector passes for FP32 problems with 16-byte aligned columns
  const bool v4 = sizeof(T) == 4 && P->vec4;

  // initial value and gradient; ||2 A y|| = ||grad Phi(0)|| for the relative tolerance
  st = launch_grad(P, x, g, mask, vals);
  if (st != BL_OK) return st;
  st = batched_dot(P, g, g, mask, gn2);
  if (st != BL_OK) return st;
  if (o->gtol_relative) {
    st = launch_forward(P, P->y, xt, mask);
    if (st != BL_OK) return st;
    st = batched_dot(P, xt, xt, mask, ay2);
    if (st != BL_OK) return st;
  }
  BL_CUDA_TRY(cudaMemsetAsync(P->d_flag, 0, sizeof(int), P->stream));
  k_lb_init<<<K, 32, 0, P->stream>>>(a, mask, vals, gn2, ay2, l2, o->gtol, o->gtol_relative, P->d_flag);
  BL_LAUNCH_CHECK(P);
  BL_CUDA_TRY(cudaMemcpyAsync(P->h_flag, P->d_flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  // One body run advances every active pair by one phase: pairs needing a direction get one and
  // take their first trial point; pairs still searching take their next (halved) trial point;
  // accepted steps update x, g and the history.  Each pair follows exactly the sequential
  // algorithm; pairs only drift apart in how many body runs their backtracking takes.
  const int max_bt = std::max(1, o->max_backtrack);
  auto body = [&]() -> bl_status {
    {
      ProfScope ps(P, BL_KC_LBFGS);
      if (v4)
        k_lb_dots_v4<<<cg, ct, 0, P->stream>>>(a, (const float*)(const void*)g, (const float*)(const void*)Sm,
                                               (const float*)(const void*)Ym, P->cpart);
      else
        k_lb_dots<T><<<cg, ct, 0, P->stream>>>(a, g, Sm, Ym, P->cpart);
      BL_LAUNCH_CHECK(P);
      k_lb_compact<<<K, 256, 0, P->stream>>>(a, P->cpart);
      BL_LAUNCH_CHECK(P);
      double* pd = P->cpart + (size_t)P->n_chunks * 4 * (MH + 1);
      if (v4)
        k_lb_dir_v4<<<cg, ct, 0, P->stream>>>(a, (float*)(void*)d, (const float*)(const void*)g,
                                              (const float*)(const void*)Sm, (const float*)(const void*)Ym, pd);
      else
        k_lb_dir<T><<<cg, ct, 0, P->stream>>>(a, d, g, Sm, Ym, pd);
      BL_LAUNCH_CHECK(P);
      k_lb_gtd<<<K, 32, 0, P->stream>>>(a, pd);
      BL_LAUNCH_CHECK(P);
      k_lb_restart<T><<<cg, ct, 0, P->stream>>>(a, d, g);
      BL_LAUNCH_CHECK(P);
      k_lb_restart_fix<<<K, 32, 0, P->stream>>>(a);
      BL_LAUNCH_CHECK(P);
      k_lb_begin_search<<<K, 32, 0, P->stream>>>(a, smask);
      BL_LAUNCH_CHECK(P);
      if (v4)
        k_lb_trial_v4<<<cg, ct, 0, P->stream>>>(a, smask, (float*)(void*)xt, (const float*)(const void*)x,
                                                (const float*)(const void*)d);
      else
        k_lb_trial<T><<<cg, ct, 0, P->stream>>>(a, smask, xt, x, d);
      BL_LAUNCH_CHECK(P);
    }
    bl_status s2 = launch_grad(P, xt, gt, smask, vals);
    if (s2 != BL_OK) return s2;
    ProfScope ps(P, BL_KC_LBFGS);
    k_lb_armijo<<<K, 32, 0, P->stream>>>(a, smask, vals, l2, max_bt, o->armijo_slack, nullptr);
    BL_LAUNCH_CHECK(P);
    if (v4)
      k_lb_accept_v4<<<cg, ct, 0, P->stream>>>(a, (float*)(void*)x, (float*)(void*)g, (const float*)(const void*)xt,
                                               (const float*)(const void*)gt, (float*)(void*)Sm, (float*)(void*)Ym);
    else
      k_lb_accept<T><<<cg, ct, 0, P->stream>>>(a, x, g, xt, gt, Sm, Ym);
    BL_LAUNCH_CHECK(P);
    BL_CUDA_TRY(cudaMemsetAsync(P->d_flag, 0, sizeof(int), P->stream));
    k_lb_post<<<K, 32, 0, P->stream>>>(a, o->max_iters, P->d_flag);
    BL_LAUNCH_CHECK(P);
    return BL_OK;
  };
  // every accepted step takes at most max_bt body runs
  const long long cap = (long long)o->max_iters * max_bt + 1;
  bool use_graph = *P->h_flag > 0 && o->graph && !P->prof && !P->graph_failed;
  if (use_graph) {
    const LbfgsGraphKey key{P->cpart, P->tpart, P->S, MH, max_bt, o->max_iters, o->armijo_slack};
    if (!P->lgraph || !(P->lgraph_key == key)) {
      if (build_lbfgs_graph(P, key, body) != BL_OK) {
        P->graph_error = error_copy();
        P->graph_failed = true;
        use_graph = false;
        (void)cudaGetLastError();
      }
    }
  }
  if (use_graph) {
    const int capi[2] = {0, (int)std::min<long long>(cap, 1 << 30)};
    BL_CUDA_TRY(cudaMemcpyAsync(P->d_loop, capi, sizeof(capi), cudaMemcpyHostToDevice, P->stream));
    BL_CUDA_TRY(cudaGraphLaunch(P->lgraph->exec, P->stream));
    int ran = 0;
    BL_CUDA_TRY(cudaMemcpyAsync(&ran, P->d_loop, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    P->launches += (int64_t)ran * P->lgraph->body_kernels + 1;
  } else {
    for (long long run = 0; run < cap && *P->h_flag > 0; ++run) {
      st = body();
      if (st != BL_OK) return st;
      BL_CUDA_TRY(cudaMemcpyAsync(P->h_flag, P->d_flag, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
      BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    }
  }
  std::vector<LbfgsState> hs(K);
  BL_CUDA_TRY(cudaMemcpyAsync(hs.data(), P->lst, K * sizeof(LbfgsState), cudaMemcpyDeviceToHost, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  info.assign(K, bl_solve_info{});
  for (int k = 0; k < K; ++k) {
    if (!mask_host[k]) continue;
    info[k].iters = hs[k].iters;
    info[k].status = hs[k].status;
    info[k].resid = hs[k].gnorm;
    info[k].nsc_est = hs[k].f;
    info[k].rhs_norm = hs[k].gtol;
  }
  return BL_OK;
}

void destroy_lbfgs_graph(bl_problem* P) {
  if (!P->lgraph) return;
  if (P->lgraph->exec) cudaGraphExecDestroy(P->lgraph->exec);
  if (P->lgraph->graph) cudaGraphDestroy(P->lgraph->graph);
  delete P->lgraph;
  P->lgraph = nullptr;
}

bl_status run_lower_solve(bl_problem* P, const std::vector<int>& mask_host, const bl_lbfgs_opts* o,
                          std::vector<bl_solve_info>& info) {
  return P->prec == BL_FP32 ? lbfgs_impl<float>(P, mask_host, o, info) : lbfgs_impl<double>(P, mask_host, o, info);
}

}  // namespace bl
