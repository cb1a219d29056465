// Tall-skinny products of the recycle refresh (Section 3): per pair, the Gram block A^T B of two
// batched n x t matrices (t <= 96 columns, n up to millions of rows) and the product A M of a
// batched n x t matrix with a small FP64 t x t' coefficient matrix.
//
// FP32 problems.  Both kernels walk a 4096-row chunk of one pair in stages of rows that
// cp.async copies into shared memory column by column (the layout of the batched matrices),
// double-buffered so the next stage lands while the current one is multiplied.  The column
// stride of a staged block is a multiple of 4 floats with an odd number of 16-byte units, so the
// 128-bit reads of consecutive columns by the lanes of a warp hit distinct bank groups.
//   Gram: each thread owns 4 columns of A x 8 columns of B, strided by the number of thread
//   blocks per side (conflict-free reads, every operand value reused 8 or 4 times from a
//   register); four rows per 128-bit read.  Products are summed in FP32 over one stage, then
//   added into an FP32 (hi, lo) pair by the error-free TwoSum; chunks combine in FP64.  When a
//   product has few columns, row groups split the stage and are summed through shared memory.
//   GEMM: each warp owns 8 output columns, each lane 4 consecutive rows: one 128-bit read of A
//   and two broadcast reads of M per 32 FMA.  The output may alias A (rows are staged first).
// FP64 problems use plain FP64 loops (test-size problems).
#include <algorithm>

#include "common.cuh"
#include "device.cuh"

namespace bl {
namespace {

constexpr int kGR = 64;           // Gram rows per stage
constexpr int kGLd = kGR + 4;     // staged column stride (floats): 17 16-byte units
constexpr int kMR = 128;          // GEMM rows per stage
constexpr int kMLd = kMR + 4;     // 33 16-byte units

__device__ __forceinline__ void cp16(float* dst, const float* src, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Copy rows [r0, r0 + R) of columns [0, nc) of one pair's column-major block (column stride n,
// first row `base`) into smem columns [c0, c0 + nc) of stride LD; rows past `nr` are zero-filled.
template <int R, int LD, bool VEC4>
__device__ __forceinline__ void stage_cols(float* buf, int c0, const float* base, long long n, int nc, int nr,
                                           int tid, int nt) {
  if (VEC4) {
    constexpr int nq = R / 4;
    for (int it = tid; it < nc * nq; it += nt) {
      const int c = it / nq, q = it - c * nq;
      const int valid = max(0, min(4, nr - 4 * q));
      const float* src = valid ? base + (long long)c * n + 4 * q : base;
      cp16(buf + (c0 + c) * LD + 4 * q, src, 4 * valid);
    }
  } else {
    for (int it = tid; it < nc * R; it += nt) {
      const int c = it / R, r = it - c * R;
      const bool valid = r < nr;
      cp4(buf + (c0 + c) * LD + r, valid ? base + (long long)c * n + r : base, valid ? 4 : 0);
    }
  }
}

// part[chunk][i * TM + j] = sum over the chunk's rows of A[row][i] B[row][j] (zeros outside
// ta x tb).  Thread layout: nbi x nbj blocks of 4 x 8 columns, G row groups.
template <bool VEC4>
__global__ void __launch_bounds__(384, 1)
    k_gram_f32(const PairDev* pairs, const ChunkDev* chunks, const float* A, int multA, const int* colsA,
               const float* B, int multB, const int* colsB, int sym, const int* mask, int TM, int nbi, int nbj,
               int G, double* part) {
  extern __shared__ __align__(16) float gsm[];
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  const int ca = 4 * nbi, cb = 8 * nbj;
  const int ta = min(max(colsA[ch.pair], 0), ca), tb = min(max(colsB[ch.pair], 0), cb);
  const int tid = threadIdx.x, nt = blockDim.x;
  double* outp = part + (size_t)blockIdx.x * TM * TM;
  for (int idx = tid; idx < TM * TM; idx += nt) {
    const int i = idx / TM, j = idx - (idx / TM) * TM;
    if (i >= ta || j >= tb) outp[idx] = 0.0;
  }
  if (ta == 0 || tb == 0) return;
  const int cA = sym ? max(ca, cb) : ca;                 // staged A columns (B shares them if sym)
  const int stage = (cA + (sym ? 0 : cb)) * kGLd;
  // columns that are never copied stay zero in both buffers
  for (int b = 0; b < 2; ++b) {
    for (int idx = tid; idx < (cA - ta) * kGLd; idx += nt) gsm[b * stage + ta * kGLd + idx] = 0.f;
    if (!sym)
      for (int idx = tid; idx < (cb - tb) * kGLd; idx += nt) gsm[b * stage + (cA + tb) * kGLd + idx] = 0.f;
  }
  const float* Ab = A + pr.off * multA + ch.start;
  const float* Bb = B + pr.off * multB + ch.start;
  const int nst = (ch.len + kGR - 1) / kGR;
  auto load = [&](int s) {
    float* bf = gsm + (s & 1) * stage;
    const int r0 = s * kGR, nr = min(kGR, ch.len - r0);
    stage_cols<kGR, kGLd, VEC4>(bf, 0, Ab + r0, pr.n, ta, nr, tid, nt);
    if (!sym) stage_cols<kGR, kGLd, VEC4>(bf, cA, Bb + r0, pr.n, tb, nr, tid, nt);
  };
  const int nblk = nbi * nbj;
  const int g = tid / nblk, blk = tid - g * nblk;
  const bool act = g < G;
  const int bi = blk / nbj, bj = blk - bi * nbj;
  float hi[4][8], lo[4][8];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) hi[k][kk] = lo[k][kk] = 0.f;
  load(0);
  cp_commit();
  for (int s = 0; s < nst; ++s) {
    if (s + 1 < nst) load(s + 1);
    cp_commit();
    cp_wait1();
    __syncthreads();
    if (act) {
      const float* cur = gsm + (s & 1) * stage;
      const float4* As4 = reinterpret_cast<const float4*>(cur);
      const float4* Bs4 = reinterpret_cast<const float4*>(cur + (sym ? 0 : cA * kGLd));
      float ps[4][8];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) ps[k][kk] = 0.f;
      for (int q = g; q < kGR / 4; q += G) {
        float4 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = As4[(bi + k * nbi) * (kGLd / 4) + q];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float4 b = Bs4[(bj + kk * nbj) * (kGLd / 4) + q];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            ps[k][kk] = fmaf(a[k].w, b.w, fmaf(a[k].z, b.z, fmaf(a[k].y, b.y, fmaf(a[k].x, b.x, ps[k][kk]))));
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const float sum = hi[k][kk] + ps[k][kk];
          const float bv = sum - hi[k][kk];
          lo[k][kk] += (hi[k][kk] - (sum - bv)) + (ps[k][kk] - bv);
          hi[k][kk] = sum;
        }
    }
    __syncthreads();
  }
  if (G > 1) {
    double* red = reinterpret_cast<double*>(gsm);   // G x nblk x 32 (fits: sized by the host)
    if (act)
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) red[((size_t)g * nblk + blk) * 32 + k * 8 + kk] = (double)hi[k][kk] + (double)lo[k][kk];
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          double v = 0.0;
          for (int gg = 0; gg < G; ++gg) v += red[((size_t)gg * nblk + blk) * 32 + k * 8 + kk];
          const int ci = bi + k * nbi, cj = bj + kk * nbj;
          if (ci < ta && cj < tb) outp[ci * TM + cj] = v;
        }
    }
    return;
  }
  if (!act) return;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int ci = bi + k * nbi, cj = bj + kk * nbj;
      if (ci < ta && cj < tb) outp[ci * TM + cj] = (double)hi[k][kk] + (double)lo[k][kk];
    }
}

// O1[row][j] = sum_l A[row][l] M1[l][j] (j < cols1), O2 likewise with M2 (optional).  M: FP64,
// ld TM, per pair.  Warp w owns output columns [8w, 8w + 8) of the concatenation [O1 | O2].
template <bool VEC4>
__global__ void __launch_bounds__(384)
    k_gemm_f32(const PairDev* pairs, const ChunkDev* chunks, const float* A, int multA, const int* colsA, int cmaxA,
               int TM, const double* M1, float* O1, int mult1, const int* cols1, const double* M2, float* O2,
               int mult2, const int* cols2, const int* mask) {
  extern __shared__ __align__(16) float msm[];
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int cbp = 8 * (nt / 32);                           // padded output columns
  const int ta = min(max(colsA[ch.pair], 0), cmaxA);
  const int t1 = min(max(cols1[ch.pair], 0), cbp);
  const int t2 = O2 ? min(max(cols2[ch.pair], 0), cbp - t1) : 0;
  if (t1 + t2 == 0) return;
  float* Ms = msm;                                         // cmaxA x cbp
  float* buf0 = Ms + cmaxA * cbp;                          // two stages of cmaxA x kMLd
  const double* M1k = M1 + (size_t)ch.pair * TM * TM;
  const double* M2k = M2 ? M2 + (size_t)ch.pair * TM * TM : nullptr;
  for (int idx = tid; idx < cmaxA * cbp; idx += nt) {
    const int l = idx / cbp, j = idx - (idx / cbp) * cbp;
    float v = 0.f;
    if (l < ta) {
      if (j < t1) v = (float)M1k[l * TM + j];
      else if (j - t1 < t2) v = (float)M2k[l * TM + (j - t1)];
    }
    Ms[idx] = v;
  }
  const float* Ab = A + pr.off * multA + ch.start;
  const int nst = (ch.len + kMR - 1) / kMR;
  auto load = [&](int s) {
    const int r0 = s * kMR;
    stage_cols<kMR, kMLd, VEC4>(buf0 + (s & 1) * cmaxA * kMLd, 0, Ab + r0, pr.n, ta, min(kMR, ch.len - r0), tid, nt);
  };
  const int lane = tid & 31, grp = tid >> 5;
  load(0);
  cp_commit();
  for (int s = 0; s < nst; ++s) {
    if (s + 1 < nst) load(s + 1);
    cp_commit();
    cp_wait1();
    __syncthreads();
    const float4* As4 = reinterpret_cast<const float4*>(buf0 + (s & 1) * cmaxA * kMLd);
    const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[r][j] = 0.f;
    for (int l = 0; l < ta; ++l) {
      const float4 a = As4[l * (kMLd / 4) + lane];
      const float4 m0 = Ms4[l * (cbp / 4) + 2 * grp], m1 = Ms4[l * (cbp / 4) + 2 * grp + 1];
      const float mv[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[0][j] = fmaf(a.x, mv[j], acc[0][j]);
        acc[1][j] = fmaf(a.y, mv[j], acc[1][j]);
        acc[2][j] = fmaf(a.z, mv[j], acc[2][j]);
        acc[3][j] = fmaf(a.w, mv[j], acc[3][j]);
      }
    }
    // every thread has read its rows of this stage before any output row is written (O1 may
    // alias A: the rows written here were staged by this block and are not re-read)
    __syncthreads();
    const int row0 = s * kMR + 4 * lane;
    const int nr = min(4, ch.len - row0);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = 8 * grp + j;
      float* dst = nullptr;
      if (col < t1) dst = O1 + pr.off * mult1 + (long long)col * pr.n + ch.start + row0;
      else if (col - t1 < t2) dst = O2 + pr.off * mult2 + (long long)(col - t1) * pr.n + ch.start + row0;
      if (!dst || nr <= 0) continue;
      if (VEC4 && nr == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
      } else {
        for (int r = 0; r < nr; ++r) dst[r] = acc[r][j];
      }
    }
  }
}

// FP64 problems: plain loops.
__global__ void k_gram_f64(const PairDev* pairs, const ChunkDev* chunks, const double* A, int multA, const int* colsA,
                           const double* B, int multB, const int* colsB, const int* mask, int TM, double* part) {
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  const int ta = min(max(colsA[ch.pair], 0), TM), tb = min(max(colsB[ch.pair], 0), TM);
  const double* Ab = A + pr.off * multA + ch.start;
  const double* Bb = B + pr.off * multB + ch.start;
  double* out = part + (size_t)blockIdx.x * TM * TM;
  for (int e = threadIdx.x; e < TM * TM; e += blockDim.x) {
    const int i = e / TM, j = e - (e / TM) * TM;
    double s = 0.0;
    if (i < ta && j < tb)
      for (int r = 0; r < ch.len; ++r) s += Ab[(long long)i * pr.n + r] * Bb[(long long)j * pr.n + r];
    out[e] = s;
  }
}

__global__ void k_gemm_f64(const PairDev* pairs, const ChunkDev* chunks, const double* A, int multA, const int* colsA,
                           int TM, const double* M1, double* O1, int mult1, const int* cols1, const double* M2,
                           double* O2, int mult2, const int* cols2, const int* mask) {
  extern __shared__ __align__(16) double dsm[];   // 64 rows x TM
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  const int ta = min(max(colsA[ch.pair], 0), TM), t1 = min(max(cols1[ch.pair], 0), TM);
  const int t2 = O2 ? min(max(cols2[ch.pair], 0), TM) : 0;
  const double* M1k = M1 + (size_t)ch.pair * TM * TM;
  const double* M2k = M2 ? M2 + (size_t)ch.pair * TM * TM : nullptr;
  const double* Ab = A + pr.off * multA + ch.start;
  for (int r0 = 0; r0 < ch.len; r0 += 64) {
    const int nr = min(64, ch.len - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * ta; idx += blockDim.x) {
      const int l = idx / 64, r = idx - l * 64;
      dsm[r * TM + l] = r < nr ? Ab[(long long)l * pr.n + r0 + r] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * (t1 + t2); idx += blockDim.x) {
      const int col = idx / nr, r = idx - col * nr;
      const double* Mk = col < t1 ? M1k : M2k;
      const int j = col < t1 ? col : col - t1;
      double v = 0.0;
      for (int l = 0; l < ta; ++l) v += dsm[r * TM + l] * Mk[l * TM + j];
      double* dst = col < t1 ? O1 + pr.off * mult1 + (long long)j * pr.n
                             : O2 + pr.off * mult2 + (long long)j * pr.n;
      dst[ch.start + r0 + r] = v;
    }
  }
}

}  // namespace

bl_status ts_gram(bl_problem* P, const void* A, int multA, const int* colsA, int cmaxA, const void* B, int multB,
                  const int* colsB, int cmaxB, const int* mask, double* out) {
  const int TM = P->TM;
  bl_status st = ensure_cpart(P, (size_t)P->n_chunks * TM * TM);
  if (st != BL_OK) return st;
  ProfScope ps(P, BL_KC_GRAM);
  if (P->prec == BL_FP32) {
    const bool sym = A == B && multA == multB && colsA == colsB;
    const int nbi = std::max(1, (cmaxA + 3) / 4), nbj = std::max(1, (cmaxB + 7) / 8);
    const int nblk = nbi * nbj;
    const int G = nblk >= 256 ? 1 : std::min(kGR / 4, 256 / nblk);
    const int nthreads = ((nblk * G + 31) / 32) * 32;
    if (nthreads > 384) return fail(BL_EINVAL, "gram: too many columns");
    const int ca = 4 * nbi, cb = 8 * nbj, cA = sym ? std::max(ca, cb) : ca;
    const size_t stage = (size_t)(cA + (sym ? 0 : cb)) * kGLd * sizeof(float);
    const size_t sm = std::max(2 * stage, G > 1 ? (size_t)G * nblk * 32 * sizeof(double) : 0);
    if (P->vec4) {
      if (!P->capturing)
        BL_CUDA_TRY(cudaFuncSetAttribute(k_gram_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_gram_f32<true><<<P->n_chunks, nthreads, sm, P->stream>>>(P->d_pairs, P->d_chunks, (const float*)A, multA,
                                                                  colsA, (const float*)B, multB, colsB, sym ? 1 : 0,
                                                                  mask, TM, nbi, nbj, G, P->cpart);
    } else {
      if (!P->capturing)
        BL_CUDA_TRY(cudaFuncSetAttribute(k_gram_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_gram_f32<false><<<P->n_chunks, nthreads, sm, P->stream>>>(P->d_pairs, P->d_chunks, (const float*)A, multA,
                                                                   colsA, (const float*)B, multB, colsB, sym ? 1 : 0,
                                                                   mask, TM, nbi, nbj, G, P->cpart);
    }
  } else {
    k_gram_f64<<<P->n_chunks, 256, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const double*)A, multA, colsA,
                                                   (const double*)B, multB, colsB, mask, TM, P->cpart);
  }
  BL_LAUNCH_CHECK(P);
  return reduce_units(P, P->cpart, TM * TM, 1, kUnitChunks, mask, nullptr, out);
}

bl_status ts_gemm(bl_problem* P, const void* A, int multA, const int* colsA, int cmaxA, const double* M1, void* O1,
                  int mult1, const int* cols1, int cmax1, const double* M2, void* O2, int mult2, const int* cols2,
                  int cmax2, const int* mask) {
  const int TM = P->TM;
  if (P->prec == BL_FP32 && O2 && (cmax1 + cmax2 + 7) / 8 > 12) {
    // two products too wide for one pass (more than 96 output columns together): the second first,
    // since the first may overwrite A in place
    bl_status st = ts_gemm(P, A, multA, colsA, cmaxA, M2, O2, mult2, cols2, cmax2, nullptr, nullptr, 0, nullptr, 0,
                           mask);
    if (st != BL_OK) return st;
    return ts_gemm(P, A, multA, colsA, cmaxA, M1, O1, mult1, cols1, cmax1, nullptr, nullptr, 0, nullptr, 0, mask);
  }
  ProfScope ps(P, BL_KC_GEMM);
  if (P->prec == BL_FP32) {
    const int ngrp = std::max(1, (cmax1 + (O2 ? cmax2 : 0) + 7) / 8);
    if (ngrp > 12) return fail(BL_EINVAL, "gemm: too many output columns");
    const int nthreads = 32 * ngrp;
    const size_t sm = ((size_t)cmaxA * 8 * ngrp + 2 * (size_t)cmaxA * kMLd) * sizeof(float);
    if (P->vec4) {
      if (!P->capturing)
        BL_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_gemm_f32<true><<<P->n_chunks, nthreads, sm, P->stream>>>(
          P->d_pairs, P->d_chunks, (const float*)A, multA, colsA, cmaxA, TM, M1, (float*)O1, mult1, cols1, M2,
          (float*)O2, mult2, cols2, mask);
    } else {
      if (!P->capturing)
        BL_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_gemm_f32<false><<<P->n_chunks, nthreads, sm, P->stream>>>(
          P->d_pairs, P->d_chunks, (const float*)A, multA, colsA, cmaxA, TM, M1, (float*)O1, mult1, cols1, M2,
          (float*)O2, mult2, cols2, mask);
    }
  } else {
    const size_t sm = 64 * (size_t)TM * sizeof(double);
    if (!P->capturing)
      BL_CUDA_TRY(cudaFuncSetAttribute(k_gemm_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_gemm_f64<<<P->n_chunks, 256, sm, P->stream>>>(P->d_pairs, P->d_chunks, (const double*)A, multA, colsA, TM, M1,
                                                    (double*)O1, mult1, cols1, M2, (double*)O2, mult2, cols2, mask);
  }
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

}  // namespace bl
