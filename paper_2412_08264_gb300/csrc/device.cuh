// Device-side helpers: penalty functions of eq. (5.1), reductions, per-pair addressing.
#pragma once

#include "common.cuh"

namespace bl {

// phi and its derivatives (eq. (5.1)); kind = bl_phi_kind.
template <typename T>
__device__ __forceinline__ void phi_all(T s, T eps, int kind, T& f, T& d1, T& d2) {
  if (kind == BL_PHI_CHARBONNIER) {
    T q = s * s + eps * eps;
    T inv = rsqrt(q);
    f = q * inv;
    d1 = s * inv;
    d2 = eps * eps * inv * inv * inv;
  } else if (kind == BL_PHI_SQ) {
    f = s * s;
    d1 = T(2) * s;
    d2 = T(2);
  } else {
    T q = T(1) + s * s;
    T iq = T(1) / q;
    f = log(q);
    d1 = T(2) * s * iq;
    d2 = T(2) * (T(1) - s * s) * iq * iq;
  }
}

template <typename T>
__device__ __forceinline__ T phi_d1(T s, T eps, int kind) {
  if (kind == BL_PHI_CHARBONNIER) return s * rsqrt(s * s + eps * eps);
  if (kind == BL_PHI_SQ) return T(2) * s;
  return T(2) * s / (T(1) + s * s);
}

template <typename T>
__device__ __forceinline__ T phi_d2(T s, T eps, int kind) {
  if (kind == BL_PHI_CHARBONNIER) {
    T inv = rsqrt(s * s + eps * eps);
    return eps * eps * inv * inv * inv;
  }
  if (kind == BL_PHI_SQ) return T(2);
  T q = T(1) + s * s;
  return T(2) * (T(1) - s * s) / (q * q);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum one value over the block; result valid in every thread.  red: >= 33 doubles of smem.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Per-thread running sums.  GB300 issues FP64 at about 1/64 of the FP32 rate, so FP32 problems
// accumulate long sums in compensated FP32 (Kahan: the running error term c is fed back into each
// addition) and switch to FP64 only for the warp / block / tile combine; FP64 problems sum in FP64.
template <typename T>
struct Accum;
template <>
struct Accum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct Accum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp total of per-lane accumulators as a double (valid in every lane): the FP32 variant sums the
// running sums and the error terms separately in FP32 and combines them in FP64.
__device__ __forceinline__ double warp_total(const Accum<float>& a) {
  return (double)warp_sum_f(a.s) - (double)warp_sum_f(a.c);
}
__device__ __forceinline__ double warp_total(const Accum<double>& a) { return warp_sum(a.s); }

// Block total of per-thread accumulators (valid in every thread).  red: >= 33 doubles of smem.
template <int NT, typename A>
__device__ __forceinline__ double block_total(const A& acc, double* red) {
  const double v = warp_total(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// acc[yy][xx] += sum_{a,b} tap(a, b) src[(yy + a) * ld + xx + b]; tap = k[a][b] or k flipped.
// ALIGNED: the caller guarantees src and ld are 16-byte multiples, so FP32 row windows whose
// length is a multiple of 4 are read with 128-bit shared loads.
template <int F, int BY, int BX, bool FLIP, bool ALIGNED = false, typename T>
__device__ __forceinline__ void corr_block(const T* __restrict__ src, int ld, const T (&k)[F * F],
                                           T (&acc)[BY][BX]) {
  constexpr int NS = BX + F - 1;
  constexpr bool kVec = ALIGNED && sizeof(T) == 4 && NS % 4 == 0;
#pragma unroll
  for (int ry = 0; ry < BY + F - 1; ++ry) {
    T seg[NS];
    if constexpr (kVec) {
#pragma unroll
      for (int c = 0; c < NS; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(&src[ry * ld + c]);
        seg[c] = v.x;
        seg[c + 1] = v.y;
        seg[c + 2] = v.z;
        seg[c + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NS; ++c) seg[c] = src[ry * ld + c];
    }
#pragma unroll
    for (int yy = 0; yy < BY; ++yy) {
      const int a = ry - yy;
      if (a < 0 || a >= F) continue;
#pragma unroll
      for (int b = 0; b < F; ++b) {
        const T tap = FLIP ? k[(F - 1 - a) * F + (F - 1 - b)] : k[a * F + b];
#pragma unroll
        for (int xx = 0; xx < BX; ++xx) acc[yy][xx] = fma(tap, seg[xx + b], acc[yy][xx]);
      }
    }
  }
}

// Column j of pair `pr` in a batched n x mult matrix (mult = 0: plain batched vector).
template <typename T>
__device__ __forceinline__ T* col_ptr(T* base, const PairDev& pr, int mult, int j) {
  return mult ? base + pr.off * mult + (long long)j * pr.n : base + pr.off;
}
template <typename T>
__device__ __forceinline__ const T* col_ptr(const T* base, const PairDev& pr, int mult, int j) {
  return mult ? base + pr.off * mult + (long long)j * pr.n : base + pr.off;
}

}  // namespace bl
