// FP32 Hessian action of the FoE lower level (eqs. (2.6), (5.1)) with TMA-staged tiles:
//   H v = 2 A^T A v + l2 v + sum_j K_j^T (d_j .* K_j v),   d_j = e^{alpha_j} phi''(k_j * x^)
// (inpainting pairs: 2 m .* v for the data term, Section 5.1), and the same for the TV regulariser.
//
// One CTA per output tile.  Thread 0 issues the bulk tensor copies: the input tile with an 8-pixel
// halo (one 3-D TMA box per tile; the tensor map's z index selects the column of a batched matrix)
// and, one filter ahead, the field tile d_j that the step-1 region reads (double-buffered).
// Completion is tracked by shared-memory mbarriers with transaction counts; image borders come from
// the copies' zero fill, so no thread evaluates bounds while staging.  Every wait is bounded: after
// two seconds the CTA records a code in the problem's error word and returns.
//
// Arithmetic: the blur part runs as four separable passes over shared memory, each thread producing
// four consecutive outputs from 128-bit row windows; the regulariser part is the register-window
// scheme of the generic kernel (per filter 4 x 4 blocks of z_j = d_j .* (K_j v) on the tile grown by
// the filter radius, then K_j^T z_j into the owners' accumulators), with z double-buffered so each
// filter costs one barrier.  Owners write their 4 x 4 blocks with 128-bit stores.  The Krylov dot
// products are not fused here: the chunk pass that follows reads q once with every column of C and Z.
//
// Tile variants (chosen per image-size class at set-up by timing, or forced by bl_set_hvp_tile):
// the generic side tile_out(F) (a 64 x 64 step-1 region, one 4 x 4 block per thread) and, for
// 3 x 3 and 5 x 5 filters, 64 x 64 outputs (a 68 x 68 step-1 region: 289 blocks, 33 threads take
// a second), which tiles images whose sides are multiples of 64 without slivers.
//
// Requirements (checked on the host, else the generic kernel runs): FP32, every pair's width a
// multiple of 4 (so rows, pair offsets and tile origins are 16-byte aligned, and the innermost box
// coordinate of every copy is a multiple of 4 elements), and the input buffer is one whose tensor
// maps were encoded at set-up.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "device.cuh"

namespace bl {

namespace {

__host__ __device__ constexpr int round32f(int v) { return (v + 31) & ~31; }   // 128-byte granules of floats

template <int F, int TILE_>
struct TmaGeom {
  static constexpr int R = F / 2;
  static constexpr int TILE = TILE_;
  static constexpr int VD = TILE + 2 * kHalo;                 // staged input side (TMA box)
  static constexpr int E1 = TILE + 2 * R;                     // step-1 region side
  static constexpr int SB = (E1 + 3) / 4;                     // step-1 blocks per side
  static constexpr int S4 = 4 * SB;
  static constexpr int FW = R == 0 ? S4 : S4 + 4;             // staged field tile (x origin rounded down)
  static constexpr int FH = S4;
  static constexpr int P1 = TILE + 2 * BL_MAX_BLUR_RADIUS;    // pitch of the blur temporaries
  static constexpr int ZP = S4 + 4;                           // pitch of z
  static constexpr int NB = TILE / 4;                         // owner blocks per side
  static_assert(NB * NB <= kStencilThreads, "one owner block per thread");
  static constexpr int fb_off = round32f(VD * VD);
  static constexpr int fb_sz = round32f(FW * FH);
  static constexpr int un_off = fb_off + 2 * fb_sz;
  static constexpr int blur_sz = VD * P1 + P1 * P1;           // pass-1 output (VD x P1) + A v (P1 x P1)
  static constexpr int z_sz = 2 * S4 * ZP;
  static constexpr int un_sz = round32f(blur_sz > z_sz ? blur_sz : z_sz);
  static constexpr int tp_off = un_off + un_sz;
  static size_t bytes(int N) { return ((size_t)tp_off + round32f(N * F * F)) * sizeof(float) + 64; }
};
// the 64 x 64-output variant exists for 3 x 3 and 5 x 5 filters (7 x 7 would not fit two CTAs per SM)
template <int F>
constexpr bool kHas64 = F == 3 || F == 5;
constexpr int kTile64 = 64;
template <int F>
using Geom0 = TmaGeom<F, tile_out(F)>;
template <int F>
using Geom1 = TmaGeom<F, kTile64>;

struct HvpTmaArgs {
  const PairDev* pairs;
  const HTileDev* tiles;
  const CUtensorMap* in_maps[2];   // per variant, per pair: the input vector / matrix
  const CUtensorMap* f_maps[2];    // per variant, per pair: the fields d_j (z index = filter)
  const float* taps;               // N * F * F
  const double* ealpha;
  int N;
  float l2;
  float* out;
  int mult;                        // 0: batched vector, else columns of a batched n x mult matrix
  const int* cols;
  const int* mask;
  unsigned long long* pix;
  int* err;
  int colfast;                     // grid x runs over columns (tiles on y): a tile's columns share L2
};

constexpr unsigned long long kWaitNs = 2000000000ull;   // bound of every mbarrier wait

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after kWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// N consecutive floats from shared memory at an address aligned to ALIGN bytes (16 or 8)
template <int N, int ALIGN>
__device__ __forceinline__ void lds_row(const float* src, float (&v)[N]) {
  if constexpr (ALIGN == 16 && N % 4 == 0) {
#pragma unroll
    for (int c = 0; c < N; c += 4) {
      const float4 t = *reinterpret_cast<const float4*>(src + c);
      v[c] = t.x; v[c + 1] = t.y; v[c + 2] = t.z; v[c + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < N; c += 2) {
      const float2 t = *reinterpret_cast<const float2*>(src + c);
      v[c] = t.x; v[c + 1] = t.y;
    }
  }
}


// Blur part of the owners' accumulators: out = 2 A(A v) + l2 v on the tile, with the intermediate A v
// truncated to the image (zero boundary).  Passes 1-3 write shared memory (each item: four
// consecutive outputs along x); pass 4 accumulates straight into the owner's registers.
// GR (gradient mode): the intermediate is A x - y (ys: y staged like vs) and dterm gathers
// ||A x - y||^2 over the tile.
template <typename G, int RB, bool GR = false>
__device__ __forceinline__ void blur_part(const float* vs, float* h1, float* av, const PairDev& pr, int oy, int ox,
                                          float l2, bool owner, int oby, int obx, float (&acc)[4][4],
                                          const float* ys = nullptr, Accum<float>* dterm = nullptr) {
  constexpr int TILE = G::TILE, VD = G::VD, P1 = G::P1;
  constexpr int NB = 2 * RB + 1, E2 = TILE + 2 * RB, SH = kHalo - 2 * RB;
  constexpr int G1 = (E2 + 3) / 4, G3 = TILE / 4;
  constexpr int A1 = (SH % 4 == 0) ? 16 : 8;       // alignment of pass 1's row windows
  constexpr int W1 = ((4 + 2 * RB) + (A1 == 16 ? 3 : 1)) / (A1 == 16 ? 4 : 2) * (A1 == 16 ? 4 : 2);
  constexpr int W3 = ((4 + 2 * RB) + 3) / 4 * 4;
  float g[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) g[b] = pr.gf[b];
  const int tid = threadIdx.x;
  // pass 1 (horizontal): h1[y][x] = sum_b g[b] vs[y][x + b + SH], y < VD, x < E2
  for (int it = tid; it < VD * G1; it += kStencilThreads) {
    const int y = it / G1, x0 = (it - y * G1) * 4;
    float win[W1];
    lds_row<W1, A1>(vs + y * VD + x0 + SH, win);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = fmaf(g[b], win[j + b], o[j]);
    *reinterpret_cast<float4*>(h1 + y * P1 + x0) = make_float4(o[0], o[1], o[2], o[3]);
  }
  __syncthreads();
  // pass 2 (vertical): av[i][x] = sum_a g[a] h1[i + a + SH][x], kept inside the image only
  for (int it = tid; it < E2 * G1; it += kStencilThreads) {
    const int i = it / G1, x0 = (it - i * G1) * 4;
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      const float4 t = *reinterpret_cast<const float4*>(h1 + (i + a + SH) * P1 + x0);
      o[0] = fmaf(g[a], t.x, o[0]);
      o[1] = fmaf(g[a], t.y, o[1]);
      o[2] = fmaf(g[a], t.z, o[2]);
      o[3] = fmaf(g[a], t.w, o[3]);
    }
    const int iy = oy - RB + i, ix = ox - RB + x0;
    const bool rin = iy >= 0 && iy < pr.h;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = rin && ix + j >= 0 && ix + j < pr.w;
      if constexpr (GR) {
        if (in) {
          o[j] -= ys[(i - RB + kHalo) * VD + x0 + j - RB + kHalo];
          if (i >= RB && i < RB + TILE && x0 + j >= RB && x0 + j < RB + TILE) dterm->add(o[j] * o[j]);
        }
      }
      if (!in) o[j] = 0.f;
    }
    *reinterpret_cast<float4*>(av + i * P1 + x0) = make_float4(o[0], o[1], o[2], o[3]);
  }
  __syncthreads();
  // pass 3 (horizontal): h3[i][x] = sum_b g[b] av[i][x + b], i < E2, x < TILE (h3 reuses h1)
  float* h3 = h1;
  for (int it = tid; it < E2 * G3; it += kStencilThreads) {
    const int i = it / G3, x0 = (it - i * G3) * 4;
    float win[W3];
    lds_row<W3, 16>(av + i * P1 + x0, win);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = fmaf(g[b], win[j + b], o[j]);
    *reinterpret_cast<float4*>(h3 + i * P1 + x0) = make_float4(o[0], o[1], o[2], o[3]);
  }
  __syncthreads();
  // pass 4 (vertical, owners): acc = 2 sum_b g[b] h3[4 oby + yy + b][4 obx + xx] + l2 v
  if (owner) {
    float o[4][4];
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) o[yy][xx] = 0.f;
#pragma unroll
    for (int ry = 0; ry < 4 + 2 * RB; ++ry) {
      const float4 t = *reinterpret_cast<const float4*>(h3 + (4 * oby + ry) * P1 + 4 * obx);
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) {
        const int b = ry - yy;
        if (b < 0 || b >= NB) continue;
        o[yy][0] = fmaf(g[b], t.x, o[yy][0]);
        o[yy][1] = fmaf(g[b], t.y, o[yy][1]);
        o[yy][2] = fmaf(g[b], t.z, o[yy][2]);
        o[yy][3] = fmaf(g[b], t.w, o[yy][3]);
      }
    }
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
      const float4 v = *reinterpret_cast<const float4*>(vs + (4 * oby + yy + kHalo) * VD + 4 * obx + kHalo);
      acc[yy][0] = fmaf(2.f, o[yy][0], l2 * v.x);
      acc[yy][1] = fmaf(2.f, o[yy][1], l2 * v.y);
      acc[yy][2] = fmaf(2.f, o[yy][2], l2 * v.z);
      acc[yy][3] = fmaf(2.f, o[yy][3], l2 * v.w);
    }
  }
}

// One output tile of the FoE Hessian action with geometry G (see the file comment).
template <int F, typename G>
__device__ __forceinline__ void hvp_tile(const HvpTmaArgs& a, const HTileDev& tl, int col, float* sm) {
  constexpr int R = G::R, TILE = G::TILE, VD = G::VD, E1 = G::E1, SB = G::SB, FW = G::FW, FH = G::FH;
  constexpr int ZP = G::ZP, S4 = G::S4, NB = G::NB;
  const PairDev pr = a.pairs[tl.pair];
  if (a.pix && threadIdx.x == 0)
    atomicAdd(a.pix, (unsigned long long)(min(TILE, pr.h - tl.oy) * min(TILE, pr.w - tl.ox)));
  float* vs = sm;
  float* fb0 = sm + G::fb_off;
  float* un = sm + G::un_off;
  float* tps = sm + G::tp_off;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tps + round32f(a.N * F * F));   // [0] input, [1..2] fields
  const int tid = threadIdx.x;
  const int oy = tl.oy, ox = tl.ox;
  const int fx0 = (ox - R) & ~3, foff = ox - R - fx0;       // field box origin (16-byte aligned x)
  constexpr int V = (kHas64<F> && TILE == kTile64) ? 1 : 0;   // the variant (constant index into the maps)
  const CUtensorMap* imap = a.in_maps[V] + tl.pair;
  const CUtensorMap* fmap = a.f_maps[V] + tl.pair;
  const uint32_t bar_in = smem_u32(bars), bar_f0 = smem_u32(bars + 1);
  constexpr uint32_t kInBytes = VD * VD * sizeof(float), kFBytes = FW * FH * sizeof(float);
  if (tid == 0) {
    mbar_init(bar_in, 1);
    mbar_init(bar_f0, 1);
    mbar_init(bar_f0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    tmap_acquire(imap);
    tmap_acquire(fmap);
    mbar_expect_tx(bar_in, kInBytes);
    tma_load_3d(smem_u32(vs), imap, ox - kHalo, oy - kHalo, a.mult ? col : 0, bar_in);
    if (a.N > 0) {
      mbar_expect_tx(bar_f0, kFBytes);
      tma_load_3d(smem_u32(fb0), fmap, fx0, oy - R, 0, bar_f0);
    }
  }
  for (int idx = tid; idx < a.N * F * F; idx += kStencilThreads) tps[idx] = a.taps[idx];
  const bool owner = tid < NB * NB;
  const int oby = owner ? tid / NB : 0, obx = owner ? tid - (tid / NB) * NB : 0;
  float outacc[4][4];
#pragma unroll
  for (int yy = 0; yy < 4; ++yy)
#pragma unroll
    for (int xx = 0; xx < 4; ++xx) outacc[yy][xx] = 0.f;
  // field copies issued / waited for (the same count in every thread; thread 0 issues them)
  int f_issued = a.N > 0 ? 1 : 0, f_done = 0;
  const bool in_done = mbar_wait(bar_in, 0);
  bool ok = in_done;
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(a.err, 1);
    goto drain;
  }
  if (pr.opm) {
    // inpainting data term: A^T A = diag(m), so 2 m v
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int iy = oy + 4 * oby + yy, ix = ox + 4 * obx + xx;
        const float vv = vs[(4 * oby + yy + kHalo) * VD + 4 * obx + xx + kHalo];
        const bool m = owner && iy < pr.h && ix < pr.w && pr.opm[(long long)iy * pr.w + ix];
        outacc[yy][xx] = (m ? 2.f * vv : 0.f) + a.l2 * vv;
      }
  } else {
    float* h1 = un;
    float* av = un + VD * G::P1;
    switch (pr.rb) {
      case 0: blur_part<G, 0>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      case 1: blur_part<G, 1>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      case 2: blur_part<G, 2>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      case 3: blur_part<G, 3>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      default: blur_part<G, 4>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
    }
  }
  __syncthreads();   // the blur temporaries are dead: the union region now holds z

  {
    // regulariser part: per filter z_j = d_j .* (K_j v) on the tile grown by R, then K_j^T z_j
    constexpr bool kAligned = (kHalo - 2 * R) % 4 == 0 && VD % 4 == 0 && ZP % 4 == 0;
    const bool s2_live = owner && oy + 4 * oby < pr.h && ox + 4 * obx < pr.w;
    float* zs = un;
    for (int jf = 0; jf < a.N; ++jf) {
      if (tid == 0 && jf + 1 < a.N) {
        // the buffer was last read before the previous filter's barrier
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bar = bar_f0 + 8 * ((jf + 1) & 1);
        mbar_expect_tx(bar, kFBytes);
        tma_load_3d(smem_u32(fb0 + ((jf + 1) & 1) * G::fb_sz), fmap, fx0, oy - R, jf + 1, bar);
      }
      if (jf + 1 < a.N) f_issued = jf + 2;
      float k[F * F];
#pragma unroll
      for (int t = 0; t < F * F; ++t) k[t] = tps[jf * F * F + t];
      const float* fb = fb0 + (jf & 1) * G::fb_sz;
      float* zb = zs + (jf & 1) * (S4 * ZP);
      bool waited = false;
      // step-1 blocks of this thread: b = tid, tid + 256 (SB^2 <= 2 * 256)
      for (int b = tid; b < SB * SB; b += kStencilThreads) {
        const int sby = b / SB, sbx = b - (b / SB) * SB;
        const bool s1_live = 4 * sby < E1 && 4 * sbx < E1 && oy - R + 4 * sby < pr.h && ox - R + 4 * sbx < pr.w &&
                             oy - R + 4 * sby + 3 >= 0 && ox - R + 4 * sbx + 3 >= 0;
        float u[4][4];
#pragma unroll
        for (int yy = 0; yy < 4; ++yy)
#pragma unroll
          for (int xx = 0; xx < 4; ++xx) u[yy][xx] = 0.f;
        if (s1_live)
          corr_block<F, 4, 4, false, kAligned>(&vs[(4 * sby + kHalo - 2 * R) * VD + 4 * sbx + kHalo - 2 * R], VD, k, u);
        if (!waited) {
          ok = mbar_wait(bar_f0 + 8 * (jf & 1), (jf >> 1) & 1);
          waited = true;
        }
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) {
          float z[4];
#pragma unroll
          for (int xx = 0; xx < 4; ++xx)
            z[xx] = s1_live ? fb[(4 * sby + yy) * FW + 4 * sbx + xx + foff] * u[yy][xx] : 0.f;
          *reinterpret_cast<float4*>(zb + (4 * sby + yy) * ZP + 4 * sbx) = make_float4(z[0], z[1], z[2], z[3]);
        }
      }
      if (!waited) ok = mbar_wait(bar_f0 + 8 * (jf & 1), (jf >> 1) & 1);
      if (ok) f_done = jf + 1;
      // one barrier per filter (z is double-buffered); it also agrees on the wait's outcome
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(a.err, 2);
        goto drain;
      }
      if (s2_live) corr_block<F, 4, 4, true, kAligned>(&zb[(4 * oby) * ZP + 4 * obx], ZP, k, outacc);
    }
  }

  {
    // owners write their blocks (128-bit stores: rows, pair offsets and tile origins are 16-byte aligned)
    float* out = col_ptr(a.out, pr, a.mult, col);
    if (owner) {
      const int ix = ox + 4 * obx;
      if (ix < pr.w) {
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) {
          const int iy = oy + 4 * oby + yy;
          if (iy < pr.h)
            *reinterpret_cast<float4*>(out + (long long)iy * pr.w + ix) =
                make_float4(outacc[yy][0], outacc[yy][1], outacc[yy][2], outacc[yy][3]);
        }
      }
    }
  }
  return;

drain:
  // a wait gave up: let the copies still in flight land (each wait bounded) before the CTA exits
  if (tid == 0) {
    if (!in_done) (void)mbar_wait(bar_in, 0);
    for (int c = f_done; c < f_issued; ++c) (void)mbar_wait(bar_f0 + 8 * (c & 1), (c >> 1) & 1);
  }
  __syncthreads();
}

template <int F>
__global__ void __launch_bounds__(kStencilThreads, 2) k_hvp_tma(HvpTmaArgs a) {
  const HTileDev tl = a.tiles[a.colfast ? blockIdx.y : blockIdx.x];
  const int col = a.colfast ? blockIdx.x : blockIdx.y;
  if (a.mask && !a.mask[tl.pair]) return;
  if (a.mult && col >= a.cols[tl.pair]) return;
  extern __shared__ __align__(128) float sm[];
  if constexpr (kHas64<F>) {
    if (tl.var) {
      hvp_tile<F, Geom1<F>>(a, tl, col, sm);
      return;
    }
  }
  hvp_tile<F, Geom0<F>>(a, tl, col, sm);
}

// ---------------------------------------------------------------------------------------------
// Gradient and value partials of Phi (eq. (5.1)) at x, with the same tiles and staging:
//   grad = 2 A^T (A x - y) + l2 x + sum_j e^{alpha_j} K_j^T phi'(K_j x)
// (inpainting: 2 m (x - y)); per tile the partials ||A x - y||^2, sum_j e^{alpha_j} sum phi(K_j x)
// and ||x||^2 over its own pixels.  x and y arrive as two TMA boxes on one mbarrier; the step-1
// values phi'(K_j x) are formed from the staged x (no field tiles).
struct GradTmaArgs {
  const PairDev* pairs;
  const HTileDev* tiles;
  const CUtensorMap* x_maps[2];    // per variant, per pair: the point x
  const CUtensorMap* y_maps[2];    // per variant, per pair: the measurements y
  const float* taps;
  const double* ealpha;
  int N, phi;
  float l2, eps;
  float* out;
  const int* mask;
  double* tpart;                   // [tile][3]
  unsigned long long* pix;
  int* err;
};

template <typename G>
struct GradLayout {
  static constexpr int ys_off = round32f(G::VD * G::VD);
  static constexpr int un_off = ys_off + round32f(G::VD * G::VD);
  static constexpr int tp_off = un_off + G::un_sz;
  static size_t bytes(int N, int F) { return ((size_t)tp_off + round32f(N * F * F)) * sizeof(float) + 64; }
};

template <int F, typename G>
__device__ __forceinline__ void grad_tile(const GradTmaArgs& a, const HTileDev& tl, int ti, float* sm) {
  using L = GradLayout<G>;
  constexpr int R = G::R, TILE = G::TILE, VD = G::VD, E1 = G::E1, SB = G::SB, ZP = G::ZP, S4 = G::S4, NB = G::NB;
  constexpr int V = (kHas64<F> && TILE == kTile64) ? 1 : 0;
  const PairDev pr = a.pairs[tl.pair];
  if (a.pix && threadIdx.x == 0)
    atomicAdd(a.pix, (unsigned long long)(min(TILE, pr.h - tl.oy) * min(TILE, pr.w - tl.ox)));
  float* vs = sm;
  float* ys = sm + L::ys_off;
  float* un = sm + L::un_off;
  float* tps = sm + L::tp_off;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tps + round32f(a.N * F * F));
  const int tid = threadIdx.x;
  const int oy = tl.oy, ox = tl.ox;
  const uint32_t b = smem_u32(bar);
  constexpr uint32_t kBox = VD * VD * sizeof(float);
  if (tid == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const CUtensorMap* xm = a.x_maps[V] + tl.pair;
    const CUtensorMap* ym = a.y_maps[V] + tl.pair;
    tmap_acquire(xm);
    tmap_acquire(ym);
    mbar_expect_tx(b, 2 * kBox);
    tma_load_3d(smem_u32(vs), xm, ox - kHalo, oy - kHalo, 0, b);
    tma_load_3d(smem_u32(ys), ym, ox - kHalo, oy - kHalo, 0, b);
  }
  for (int idx = tid; idx < a.N * F * F; idx += kStencilThreads) tps[idx] = a.taps[idx];
  const bool owner = tid < NB * NB;
  const int oby = owner ? tid / NB : 0, obx = owner ? tid - (tid / NB) * NB : 0;
  float outacc[4][4];
#pragma unroll
  for (int yy = 0; yy < 4; ++yy)
#pragma unroll
    for (int xx = 0; xx < 4; ++xx) outacc[yy][xx] = 0.f;
  Accum<float> dterm, rterm, xx2;
  const bool ok = mbar_wait(b, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicExch(a.err, 4);
      (void)mbar_wait(b, 0);                                     // bounded: let the copies land
    }
    __syncthreads();
    return;
  }
  if (pr.opm) {
    // inpainting data term: 2 m (x - y), ||m (x - y)||^2 over the owned pixels
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int iy = oy + 4 * oby + yy, ix = ox + 4 * obx + xx;
        const int c = (4 * oby + yy + kHalo) * VD + 4 * obx + xx + kHalo;
        const float xv = vs[c];
        float dv = 0.f;
        if (owner && iy < pr.h && ix < pr.w && pr.opm[(long long)iy * pr.w + ix]) {
          dv = xv - ys[c];
          dterm.add(dv * dv);
        }
        outacc[yy][xx] = 2.f * dv + a.l2 * xv;
      }
  } else {
    float* h1 = un;
    float* av = un + VD * G::P1;
    switch (pr.rb) {
      case 0: blur_part<G, 0, true>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc, ys, &dterm); break;
      case 1: blur_part<G, 1, true>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc, ys, &dterm); break;
      case 2: blur_part<G, 2, true>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc, ys, &dterm); break;
      case 3: blur_part<G, 3, true>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc, ys, &dterm); break;
      default: blur_part<G, 4, true>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc, ys, &dterm); break;
    }
  }
  __syncthreads();   // blur temporaries dead: the union region holds z
  {
    constexpr bool kAligned = (kHalo - 2 * R) % 4 == 0 && VD % 4 == 0 && ZP % 4 == 0;
    const bool s2_live = owner && oy + 4 * oby < pr.h && ox + 4 * obx < pr.w;
    float* zs = un;
    for (int jf = 0; jf < a.N; ++jf) {
      float k[F * F];
#pragma unroll
      for (int t = 0; t < F * F; ++t) k[t] = tps[jf * F * F + t];
      const float ea = (float)a.ealpha[jf];
      float* zb = zs + (jf & 1) * (S4 * ZP);
      for (int bb = tid; bb < SB * SB; bb += kStencilThreads) {
        const int sby = bb / SB, sbx = bb - (bb / SB) * SB;
        const bool s1_live = 4 * sby < E1 && 4 * sbx < E1 && oy - R + 4 * sby < pr.h && ox - R + 4 * sbx < pr.w &&
                             oy - R + 4 * sby + 3 >= 0 && ox - R + 4 * sbx + 3 >= 0;
        float u[4][4];
#pragma unroll
        for (int yy = 0; yy < 4; ++yy)
#pragma unroll
          for (int xx = 0; xx < 4; ++xx) u[yy][xx] = 0.f;
        if (s1_live)
          corr_block<F, 4, 4, false, kAligned>(&vs[(4 * sby + kHalo - 2 * R) * VD + 4 * sbx + kHalo - 2 * R], VD, k, u);
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) {
          float z[4];
#pragma unroll
          for (int xx = 0; xx < 4; ++xx) {
            const int ey = 4 * sby + yy, ex = 4 * sbx + xx;
            const int iy = oy - R + ey, ix = ox - R + ex;
            z[xx] = 0.f;
            if (s1_live && ey < E1 && ex < E1 && iy >= 0 && iy < pr.h && ix >= 0 && ix < pr.w) {
              float f0, d1, d2;
              phi_all(u[yy][xx], a.eps, a.phi, f0, d1, d2);
              z[xx] = ea * d1;
              if (ey >= R && ey < R + TILE && ex >= R && ex < R + TILE) rterm.add(ea * f0);
            }
          }
          *reinterpret_cast<float4*>(zb + (4 * sby + yy) * ZP + 4 * sbx) = make_float4(z[0], z[1], z[2], z[3]);
        }
      }
      __syncthreads();   // z is double-buffered: one barrier per filter
      if (s2_live) corr_block<F, 4, 4, true, kAligned>(&zb[(4 * oby) * ZP + 4 * obx], ZP, k, outacc);
    }
  }
  // owners write their blocks and gather ||x||^2
  if (owner) {
    const int ix = ox + 4 * obx;
    if (ix < pr.w) {
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) {
        const int iy = oy + 4 * oby + yy;
        if (iy < pr.h) {
          *reinterpret_cast<float4*>(a.out + pr.off + (long long)iy * pr.w + ix) =
              make_float4(outacc[yy][0], outacc[yy][1], outacc[yy][2], outacc[yy][3]);
#pragma unroll
          for (int xx = 0; xx < 4; ++xx) {
            const float xv = vs[(4 * oby + yy + kHalo) * VD + 4 * obx + xx + kHalo];
            xx2.add(xv * xv);
          }
        }
      }
    }
  }
  __syncthreads();   // every thread is done with z: the union region takes the reduction scratch
  double* red = reinterpret_cast<double*>(un);
  const double t0 = block_total<kStencilThreads>(dterm, red);
  const double t1 = block_total<kStencilThreads>(rterm, red);
  const double t2 = block_total<kStencilThreads>(xx2, red);
  if (tid == 0) {
    a.tpart[(size_t)ti * 3 + 0] = t0;
    a.tpart[(size_t)ti * 3 + 1] = t1;
    a.tpart[(size_t)ti * 3 + 2] = t2;
  }
}

template <int F>
__global__ void __launch_bounds__(kStencilThreads, 2) k_grad_tma(GradTmaArgs a) {
  const int ti = blockIdx.x;
  const HTileDev tl = a.tiles[ti];
  if (a.mask && !a.mask[tl.pair]) return;
  extern __shared__ __align__(128) float sm[];
  if constexpr (kHas64<F>) {
    if (tl.var) {
      grad_tile<F, Geom1<F>>(a, tl, ti, sm);
      return;
    }
  }
  grad_tile<F, Geom0<F>>(a, tl, ti, sm);
}

struct TvTmaArgs {
  const PairDev* pairs;
  const HTileDev* tiles;
  const CUtensorMap* in_maps;
  const CUtensorMap* x_maps;
  const double* ealpha;
  float l2, eps;
  float* out;
  int mult;
  const int* cols;
  const int* mask;
  unsigned long long* pix;
  int* err;
  int colfast;
};


struct TvGeom {
  using G1 = TmaGeom<1, kTile64>;
  static constexpr int TILE = G1::TILE, VD = G1::VD, P1 = G1::P1;
  static constexpr int QN = TILE + 1, QP = TILE + 4;            // q region side and pitch
  static constexpr int xs_off = round32f(VD * VD);
  static constexpr int un_off = xs_off + round32f(VD * VD);
  static constexpr int blur_sz = VD * P1 + P1 * P1;
  static constexpr int q_sz = 2 * QN * QP;
  static constexpr int un_sz = round32f(blur_sz > q_sz ? blur_sz : q_sz);
  static constexpr size_t bytes = ((size_t)un_off + un_sz) * sizeof(float) + 64;
};

__global__ void __launch_bounds__(kStencilThreads, 2) k_tv_hvp_tma(TvTmaArgs a) {
  using G = TvGeom;
  constexpr int TILE = G::TILE, VD = G::VD, QN = G::QN, QP = G::QP;
  const HTileDev tl = a.tiles[a.colfast ? blockIdx.y : blockIdx.x];
  const int col = a.colfast ? blockIdx.x : blockIdx.y;
  if (a.mask && !a.mask[tl.pair]) return;
  if (a.mult && col >= a.cols[tl.pair]) return;
  const PairDev pr = a.pairs[tl.pair];
  if (a.pix && threadIdx.x == 0)
    atomicAdd(a.pix, (unsigned long long)(min(TILE, pr.h - tl.oy) * min(TILE, pr.w - tl.ox)));
  extern __shared__ __align__(128) float sm[];
  float* vs = sm;
  float* xs = sm + G::xs_off;
  float* un = sm + G::un_off;
  uint64_t* bar = reinterpret_cast<uint64_t*>(un + G::un_sz);
  const int tid = threadIdx.x;
  const int oy = tl.oy, ox = tl.ox;
  const uint32_t b = smem_u32(bar);
  constexpr uint32_t kBox = VD * VD * sizeof(float);
  if (tid == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const CUtensorMap* im = a.in_maps + tl.pair;
    const CUtensorMap* xm = a.x_maps + tl.pair;
    tmap_acquire(im);
    tmap_acquire(xm);
    mbar_expect_tx(b, 2 * kBox);
    tma_load_3d(smem_u32(vs), im, ox - kHalo, oy - kHalo, a.mult ? col : 0, b);
    tma_load_3d(smem_u32(xs), xm, ox - kHalo, oy - kHalo, 0, b);
  }
  const int oby = tid >> 4, obx = tid & 15;                     // 16 x 16 owners of 4 x 4 blocks
  float acc[4][4];
  const bool ok = mbar_wait(b, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      atomicExch(a.err, 3);
      (void)mbar_wait(b, 0);                                     // bounded: let the copies land
    }
    __syncthreads();
    return;
  }
  {
    float* h1 = un;
    float* av = un + VD * G::P1;
    switch (pr.rb) {
      case 0: blur_part<TvGeom::G1, 0>(vs, h1, av, pr, oy, ox, a.l2, true, oby, obx, acc); break;
      case 1: blur_part<TvGeom::G1, 1>(vs, h1, av, pr, oy, ox, a.l2, true, oby, obx, acc); break;
      case 2: blur_part<TvGeom::G1, 2>(vs, h1, av, pr, oy, ox, a.l2, true, oby, obx, acc); break;
      case 3: blur_part<TvGeom::G1, 3>(vs, h1, av, pr, oy, ox, a.l2, true, oby, obx, acc); break;
      default: blur_part<TvGeom::G1, 4>(vs, h1, av, pr, oy, ox, a.l2, true, oby, obx, acc); break;
    }
  }
  __syncthreads();   // blur temporaries dead: the union region holds q
  float* q0s = un;
  float* q1s = un + QN * QP;
  const float eps2 = a.eps * a.eps;
  // q on rows / columns [-1, TILE) of the tile (zero outside the image)
  for (int it = tid; it < QN * QN; it += kStencilThreads) {
    const int i = it / QN - 1, j = it - (it / QN) * QN - 1;
    const int gy = oy + i, gx = ox + j;
    float q0 = 0.f, q1 = 0.f;
    if (gy >= 0 && gy < pr.h && gx >= 0 && gx < pr.w) {
      const int c = (i + kHalo) * VD + j + kHalo;
      const float a0 = gy + 1 < pr.h ? xs[c + VD] - xs[c] : 0.f;
      const float a1 = gx + 1 < pr.w ? xs[c + 1] - xs[c] : 0.f;
      const float d0 = gy + 1 < pr.h ? vs[c + VD] - vs[c] : 0.f;
      const float d1 = gx + 1 < pr.w ? vs[c + 1] - vs[c] : 0.f;
      const float s2 = fmaf(a0, a0, fmaf(a1, a1, eps2));
      const float is = rsqrtf(s2);
      const float ad = fmaf(a0, d0, a1 * d1) / s2;
      q0 = (d0 - a0 * ad) * is;
      q1 = (d1 - a1 * ad) * is;
    }
    q0s[(i + 1) * QP + j + 1] = q0;
    q1s[(i + 1) * QP + j + 1] = q1;
  }
  __syncthreads();
  const float et = (float)a.ealpha[0];
  float* out = col_ptr(a.out, pr, a.mult, col);
  const int gx0 = ox + 4 * obx;
  if (gx0 >= pr.w) return;
#pragma unroll
  for (int yy = 0; yy < 4; ++yy) {
    const int i = 4 * oby + yy, gy = oy + i;
    if (gy >= pr.h) break;
    float o[4];
#pragma unroll
    for (int xx = 0; xx < 4; ++xx) {
      const int j = 4 * obx + xx, gx = ox + j;
      float dv = 0.f;
      if (gy + 1 < pr.h) dv -= q0s[(i + 1) * QP + j + 1];
      if (gx + 1 < pr.w) dv -= q1s[(i + 1) * QP + j + 1];
      if (gy >= 1) dv += q0s[i * QP + j + 1];
      if (gx >= 1) dv += q1s[(i + 1) * QP + j];
      o[xx] = fmaf(et, dv, acc[yy][xx]);
    }
    *reinterpret_cast<float4*>(out + (long long)gy * pr.w + gx0) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

// ---------------------------------------------------------------------------------------------
// Host side: tensor maps and the launcher
// ---------------------------------------------------------------------------------------------
// Host side: tensor maps, the tile list and its tuning, launchers

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <int F>
size_t smem_for(int N) {
  size_t b = Geom0<F>::bytes(N);
  if constexpr (kHas64<F>) b = std::max(b, Geom1<F>::bytes(N));
  return b;
}

size_t kernel_smem(const bl_problem* P) {
  if (P->reg.kind == BL_REG_TV) return TvGeom::bytes;
  switch (P->F) {
    case 1: return smem_for<1>(P->N);
    case 3: return smem_for<3>(P->N);
    case 5: return smem_for<5>(P->N);
    default: return smem_for<7>(P->N);
  }
}

// box shapes of a variant: staged input side, field tile width and height
struct Boxes { int vd, fw, fh, tile; };
template <typename G>
Boxes boxes_of() { return Boxes{G::VD, G::FW, G::FH, G::TILE}; }
Boxes boxes(int F, int var) {
  switch (F) {
    case 1: return boxes_of<Geom0<1>>();
    case 3: return var ? boxes_of<Geom1<3>>() : boxes_of<Geom0<3>>();
    case 5: return var ? boxes_of<Geom1<5>>() : boxes_of<Geom0<5>>();
    default: return boxes_of<Geom0<7>>();
  }
}

// 3-D map over a pair's image (x: width, y: rows, z: columns of a batched matrix or the filter index)
bl_status encode(PFN_cuTensorMapEncodeTiled_v12000 fn, CUtensorMap* m, const void* base, int w, int h, long long depth,
                 long long zstride_elems, int box_x, int box_y) {
  cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)std::max<long long>(1, depth)};
  cuuint64_t strides[2] = {(cuuint64_t)w * sizeof(float), (cuuint64_t)zstride_elems * sizeof(float)};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(BL_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return BL_OK;
}

int tile_side(const bl_problem* P, int var) { return var ? kTile64 : tile_out(P->F); }

void build_htiles(const bl_problem* P, const std::vector<int>& var, const std::vector<int>& pairs,
                  std::vector<HTileDev>& out) {
  out.clear();
  for (int k : pairs) {
    const int T = tile_side(P, var[k]);
    const auto& ph = P->ph[k];
    for (int ty = 0; ty < ph.h; ty += T)
      for (int tx = 0; tx < ph.w; tx += T) out.push_back(HTileDev{k, ty, tx, var[k]});
  }
}

bl_status upload_htiles(bl_problem* P, const std::vector<HTileDev>& t) {
  if ((int)t.size() > P->htiles_cap) {
    if (P->d_htiles) {
      BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
      cudaFree(P->d_htiles);
      P->d_htiles = nullptr;
    }
    bl_status st = dalloc((void**)&P->d_htiles, t.size() * sizeof(HTileDev));
    if (st != BL_OK) return st;
    P->htiles_cap = (int)t.size();
  }
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_htiles, t.data(), t.size() * sizeof(HTileDev), cudaMemcpyHostToDevice, P->stream));
  // per-pair ranges of the list (pairs appear in one contiguous run each) for the tile reductions
  for (auto& d : P->pd_host) d.htbeg = d.htend = 0;
  for (int i = 0; i < (int)t.size(); ++i) {
    PairDev& d = P->pd_host[t[i].pair];
    if (d.htend == 0) d.htbeg = i;
    d.htend = i + 1;
  }
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_pairs, P->pd_host.data(), P->pd_host.size() * sizeof(PairDev),
                              cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  P->n_htiles = (int)t.size();
  return BL_OK;
}

}  // namespace

bl_status launch_hvp_tma(bl_problem* P, int slot, const void* in, void* out, int mult, int cols, const int* mask);

// Per image-size class (height, width, blur radius, operator), the variant with the shorter measured
// Hessian action: a warm-up and three timed launches of each variant on that class's pairs (on zero
// fields and input: the arithmetic does not depend on the values).  Classes under 65,536 pixels take
// the variant with fewer tiles (ties: the generic one), their launches being too short to time.
static bl_status tune_htiles(bl_problem* P) {
  const int K = P->K;
  std::vector<int> var(K, 0), all(K);
  for (int k = 0; k < K; ++k) all[k] = k;
  std::vector<HTileDev> list;
  if (P->tma_nvar == 2) {
    BL_CUDA_TRY(cudaMemsetAsync(P->fd, 0, (size_t)P->N * P->n_tot * sizeof(float), P->stream));
    BL_CUDA_TRY(cudaMemsetAsync(P->pv, 0, (size_t)P->n_tot * sizeof(float), P->stream));
    std::map<std::tuple<int, int, int, bool>, std::vector<int>> classes;
    for (int k = 0; k < K; ++k) {
      const auto& ph = P->ph[k];
      classes[std::make_tuple(ph.h, ph.w, ph.rb, ph.masked)].push_back(k);
    }
    cudaEvent_t e0, e1;
    BL_CUDA_TRY(cudaEventCreate(&e0));
    BL_CUDA_TRY(cudaEventCreate(&e1));
    bl_status st = BL_OK;
    for (const auto& cl : classes) {
      const int h = std::get<0>(cl.first), w = std::get<1>(cl.first);
      long long px = 0;
      for (int k : cl.second) px += P->ph[k].n;
      int best = 0;
      if (px < 65536) {
        const int T0 = tile_side(P, 0), T1 = tile_side(P, 1);
        const long long n0 = (long long)((h + T0 - 1) / T0) * ((w + T0 - 1) / T0);
        const long long n1 = (long long)((h + T1 - 1) / T1) * ((w + T1 - 1) / T1);
        best = n1 < n0 ? 1 : 0;
      } else {
        float t[2] = {0.f, 0.f};
        for (int v = 0; v < 2 && st == BL_OK; ++v) {
          for (int k : cl.second) var[k] = v;
          build_htiles(P, var, cl.second, list);
          if ((st = upload_htiles(P, list)) != BL_OK) break;
          for (int rep = 0; rep < 4 && st == BL_OK; ++rep) {
            if (rep == 1 && cudaEventRecord(e0, P->stream) != cudaSuccess) st = fail(BL_ECUDA, "cudaEventRecord");
            if (st == BL_OK) st = launch_hvp_tma(P, 0, P->pv, P->q, 0, 0, nullptr);
          }
          if (st == BL_OK && (cudaEventRecord(e1, P->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&t[v], e0, e1) != cudaSuccess))
            st = fail(BL_ECUDA, "timing the Hessian-action tile variants");
        }
        best = t[1] < t[0] ? 1 : 0;
      }
      for (int k : cl.second) var[k] = best;
      if (st != BL_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != BL_OK) return st;
    if ((st = check_kernel_error(P)) != BL_OK) return st;
  }
  P->hvar = var;
  build_htiles(P, var, all, list);
  return upload_htiles(P, list);
}

template <int F>
size_t grad_smem(int N) {
  size_t b = GradLayout<Geom0<F>>::bytes(N, F);
  if constexpr (kHas64<F>) b = std::max(b, GradLayout<Geom1<F>>::bytes(N, F));
  return b;
}

bl_status hvp_tma_setup(bl_problem* P) {
  P->tma = false;
  if (P->prec != BL_FP32) return BL_OK;
  const bool tv = P->reg.kind == BL_REG_TV;
  if (!tv && P->N < 1) return BL_OK;
  for (const auto& ph : P->ph)
    if (ph.w % 4 != 0) return BL_OK;           // rows or tile origins would not be 16-byte aligned
  if (P->n_tot % 4 != 0) return BL_OK;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return BL_OK;                       // driver without tensor maps: the generic kernel runs
  const int nvar = (!tv && (P->F == 3 || P->F == 5)) ? 2 : 1;
  // per variant: slot 0 the fields (FoE) or x^ (TV); slots 1..: the inputs the Hessian action runs on
  struct In { const void* ptr; int mult; };
  const In ins[] = {{P->pv, 0}, {P->w, 0}, {P->r, 0}, {P->Wt, P->TM}, {P->U, P->SMAX},
                    {P->lx, 0}, {P->lxt, 0}, {P->y, 0}};
  const int nslots = 1 + (int)(sizeof(ins) / sizeof(ins[0]));
  std::vector<CUtensorMap> maps((size_t)nvar * nslots * P->K);
  for (int v = 0; v < nvar; ++v) {
    const Boxes b = boxes(P->F, v);
    CUtensorMap* mv = maps.data() + (size_t)v * nslots * P->K;
    for (int k = 0; k < P->K; ++k) {
      const auto& ph = P->ph[k];
      bl_status st = tv ? encode(fn, &mv[k], (const float*)P->xhat + ph.off, ph.w, ph.h, 1, ph.n, b.vd, b.vd)
                        : encode(fn, &mv[k], (const float*)P->fd + ph.off, ph.w, ph.h, P->N, P->n_tot, b.fw, b.fh);
      if (st != BL_OK) return st;
      for (int s = 0; s + 1 < nslots; ++s) {
        const In& in = ins[s];
        const float* base = (const float*)in.ptr + ph.off * std::max(1, in.mult);
        st = encode(fn, &mv[(size_t)(s + 1) * P->K + k], base, ph.w, ph.h, std::max(1, in.mult), ph.n, b.vd, b.vd);
        if (st != BL_OK) return st;
      }
    }
  }
  bl_status st = dalloc((void**)&P->d_tmaps, maps.size() * sizeof(CUtensorMap));
  if (st != BL_OK) return st;
  BL_CUDA_TRY(cudaMemcpy(P->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
  for (int s = 0; s + 1 < nslots; ++s) {
    P->tma_in_ptr[s] = ins[s].ptr;
    P->tma_in_mult[s] = ins[s].mult;
  }
  P->tma_slots = nslots - 1;
  P->tma_nvar = nvar;
  P->tma = true;
  const size_t sm = kernel_smem(P);
  switch (tv ? 0 : P->F) {
    case 0: BL_CUDA_TRY(cudaFuncSetAttribute(k_tv_hvp_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    case 1: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    case 3: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    case 5: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    default: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
  }
  if (!tv) {
    // the gradient kernel's limit too (graph capture of the L-BFGS loop cannot change attributes)
    switch (P->F) {
      case 1: BL_CUDA_TRY(cudaFuncSetAttribute(k_grad_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<1>(P->N))); break;
      case 3: BL_CUDA_TRY(cudaFuncSetAttribute(k_grad_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<3>(P->N))); break;
      case 5: BL_CUDA_TRY(cudaFuncSetAttribute(k_grad_tma<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<5>(P->N))); break;
      default: BL_CUDA_TRY(cudaFuncSetAttribute(k_grad_tma<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<7>(P->N))); break;
    }
  }
  return tune_htiles(P);
}

int hvp_tma_slot(const bl_problem* P, const void* in, int mult) {
  if (!P->tma) return -1;
  for (int s = 0; s < P->tma_slots; ++s)
    if (P->tma_in_ptr[s] == in && P->tma_in_mult[s] == mult) return s;
  return -1;
}


int hvp_tma_grad_slot(const bl_problem* P, const void* x) {
  if (!P->tma || P->reg.kind != BL_REG_FOE) return -1;
  const int s = hvp_tma_slot(P, x, 0);
  return (s >= 0 && (x == P->lx || x == P->lxt)) ? s : -1;
}

template <int F>
static bl_status launch_grad_f(bl_problem* P, const GradTmaArgs& a) {
  const size_t sm = grad_smem<F>(P->N);
  if (!P->capturing)
    BL_CUDA_TRY(cudaFuncSetAttribute(k_grad_tma<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_grad_tma<F><<<P->n_htiles, kStencilThreads, sm, P->stream>>>(a);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

bl_status launch_grad_tma(bl_problem* P, int slot, void* grad, const int* mask, double* tpart) {
  GradTmaArgs a{};
  a.pairs = P->d_pairs;
  a.tiles = P->d_htiles;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->d_tmaps);
  const int nslots = 1 + P->tma_slots;
  int yslot = -1;
  for (int s2 = 0; s2 < P->tma_slots; ++s2)
    if (P->tma_in_ptr[s2] == P->y) yslot = s2;
  if (yslot < 0) return fail(BL_ESTATE, "no tensor maps for the measurements");
  for (int v = 0; v < 2; ++v) {
    const CUtensorMap* mv = maps + (size_t)std::min(v, P->tma_nvar - 1) * nslots * P->K;
    a.x_maps[v] = mv + (size_t)(slot + 1) * P->K;
    a.y_maps[v] = mv + (size_t)(yslot + 1) * P->K;
  }
  a.taps = P->taps_f;
  a.ealpha = P->ealpha;
  a.N = P->N;
  a.phi = P->reg.phi;
  a.l2 = (float)P->reg.l2_eps;
  a.eps = (float)P->reg.phi_eps;
  a.out = (float*)grad;
  a.mask = mask;
  a.tpart = tpart;
  a.pix = pix_counter(P, BL_KC_GRAD);
  a.err = P->d_kerr;
  ProfScope ps(P, BL_KC_GRAD);
  switch (P->F) {
    case 1: return launch_grad_f<1>(P, a);
    case 3: return launch_grad_f<3>(P, a);
    case 5: return launch_grad_f<5>(P, a);
    case 7: return launch_grad_f<7>(P, a);
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
}

template <int F>
static bl_status launch_f(bl_problem* P, const HvpTmaArgs& a, dim3 grid) {
  const size_t sm = kernel_smem(P);
  if (!P->capturing)
    BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_hvp_tma<F><<<grid, kStencilThreads, sm, P->stream>>>(a);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

static bl_status launch_tv(bl_problem* P, int slot, void* out, int mult, int cols, const int* mask) {
  TvTmaArgs a{};
  a.pairs = P->d_pairs;
  a.tiles = P->d_htiles;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->d_tmaps);
  a.x_maps = maps;
  a.in_maps = maps + (size_t)(slot + 1) * P->K;
  a.ealpha = P->ealpha;
  a.l2 = (float)P->reg.l2_eps;
  a.eps = (float)P->reg.phi_eps;
  a.out = (float*)out;
  a.mult = mult;
  a.cols = P->d_cols;
  a.mask = mask;
  const int cls = mult ? BL_KC_HVP_MULTI : BL_KC_HVP;
  a.pix = pix_counter(P, cls);
  a.err = P->d_kerr;
  ProfScope ps(P, cls);
  a.colfast = (mult && cols > 1 && P->n_htiles <= 65535) ? 1 : 0;
  const dim3 grid = a.colfast ? dim3(cols, P->n_htiles) : dim3(P->n_htiles, mult ? cols : 1);
  if (!P->capturing)
    BL_CUDA_TRY(cudaFuncSetAttribute(k_tv_hvp_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TvGeom::bytes));
  k_tv_hvp_tma<<<grid, kStencilThreads, TvGeom::bytes, P->stream>>>(a);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

bl_status launch_hvp_tma(bl_problem* P, int slot, const void* in, void* out, int mult, int cols, const int* mask) {
  (void)in;
  if (P->reg.kind == BL_REG_TV) return launch_tv(P, slot, out, mult, cols, mask);
  HvpTmaArgs a{};
  a.pairs = P->d_pairs;
  a.tiles = P->d_htiles;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->d_tmaps);
  const int nslots = 1 + P->tma_slots;
  for (int v = 0; v < 2; ++v) {
    const CUtensorMap* mv = maps + (size_t)std::min(v, P->tma_nvar - 1) * nslots * P->K;
    a.f_maps[v] = mv;
    a.in_maps[v] = mv + (size_t)(slot + 1) * P->K;
  }
  a.taps = P->taps_f;
  a.ealpha = P->ealpha;
  a.N = P->N;
  a.l2 = (float)P->reg.l2_eps;
  a.out = (float*)out;
  a.mult = mult;
  a.cols = P->d_cols;
  a.mask = mask;
  const int cls = mult ? BL_KC_HVP_MULTI : BL_KC_HVP;
  a.pix = pix_counter(P, cls);
  a.err = P->d_kerr;
  ProfScope ps(P, cls);
  // several columns: the columns of one tile run next to each other, so its field tiles stay in L2
  a.colfast = (mult && cols > 1 && P->n_htiles <= 65535) ? 1 : 0;
  const dim3 grid = a.colfast ? dim3(cols, P->n_htiles) : dim3(P->n_htiles, mult ? cols : 1);
  switch (P->F) {
    case 1: return launch_f<1>(P, a, grid);
    case 3: return launch_f<3>(P, a, grid);
    case 5: return launch_f<5>(P, a, grid);
    case 7: return launch_f<7>(P, a, grid);
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
}

bl_status prepare_hvp_tma(bl_problem* P) {
  (void)P;   // the shared-memory limit is raised when the tensor maps are encoded
  return BL_OK;
}

int hvp_tma_tile(const bl_problem* P, int pair) {
  if (!P->tma || pair < 0 || pair >= P->K) return 0;
  return tile_side(P, P->hvar[pair]);
}

bl_status hvp_tma_force_tile(bl_problem* P, int pair, int side) {
  if (!P->tma) return fail(BL_EINVAL, "this problem's Hessian action does not run the TMA-staged kernel");
  if (pair < 0 || pair >= P->K) return fail(BL_EINVAL, "pair out of range");
  int v = -1;
  for (int c = 0; c < P->tma_nvar; ++c)
    if (tile_side(P, c) == side) v = c;
  if (v < 0) return fail(BL_EINVAL, "unsupported tile side for this filter size");
  P->hvar[pair] = v;
  std::vector<int> all(P->K);
  for (int k = 0; k < P->K; ++k) all[k] = k;
  std::vector<HTileDev> list;
  build_htiles(P, P->hvar, all, list);
  destroy_krylov_graph(P);   // captured launches hold the old list's size
  return upload_htiles(P, list);
}

}  // namespace bl
