// FP32 Hessian action of the FoE lower level (eqs. (2.6), (5.1)) with TMA-staged tiles:
//   H v = 2 A^T A v + l2 v + sum_j K_j^T (d_j .* K_j v),   d_j = e^{alpha_j} phi''(k_j * x^)
// (inpainting pairs: 2 m .* v for the data term, Section 5.1).
//
// One CTA per output tile (tile_out(F) square).  Thread 0 issues the bulk tensor copies: the input
// tile with an 8-pixel halo (one 3-D TMA box per tile; the tensor map's z index selects the column of
// a batched matrix) and, one filter ahead, the 64-row field tile d_j that the step-1 region reads
// (double-buffered).  Completion is tracked by shared-memory mbarriers with transaction counts; image
// borders come from the copies' zero fill, so no thread evaluates bounds while staging.  Every wait
// is bounded: after two seconds the CTA records a code in the problem's error word and returns.
//
// Arithmetic: the blur part runs as four separable passes over shared memory, each thread producing
// four consecutive outputs from 128-bit row windows; the regulariser part is the register-window
// scheme of the generic kernel (per filter a 4 x 4 block of z_j = d_j .* (K_j v) on the tile grown by
// the filter radius, then K_j^T z_j into the owners' accumulators), with z double-buffered so each
// filter costs one barrier.  Owners write their 4 x 4 blocks with 128-bit stores.  The Krylov dot
// products are not fused here: the chunk pass that follows reads q once with every column of C and Z.
//
// Requirements (checked on the host, else the generic kernel runs): FP32, every pair's width a
// multiple of 4 (so rows, pair offsets and tile origins are 16-byte aligned, and the innermost box
// coordinate of every copy is a multiple of 4 elements), and the input buffer is one whose tensor
// maps were encoded at set-up.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "device.cuh"

namespace bl {

namespace {

template <int F>
struct TmaGeom {
  static constexpr int R = F / 2;
  static constexpr int TILE = tile_out(F);
  static constexpr int VD = TILE + 2 * kHalo;                 // staged input side (TMA box)
  static constexpr int E1 = TILE + 2 * R;                     // step-1 region side
  static constexpr int FW = F == 1 ? kTileRegion : kTileRegion + 4;   // staged field tile width
  static constexpr int FH = kTileRegion;                      // staged field tile height
  static constexpr int P1 = TILE + 2 * BL_MAX_BLUR_RADIUS;    // pitch of the blur temporaries
  static constexpr int ZP = kTileRegion + 4;                  // pitch of z
  __host__ __device__ static constexpr int r32(int v) { return (v + 31) & ~31; }   // 128-byte granules of floats
  static constexpr int fb_off = r32(VD * VD);
  static constexpr int fb_sz = r32(FW * FH);
  static constexpr int un_off = fb_off + 2 * fb_sz;
  static constexpr int blur_sz = VD * P1 + P1 * P1;           // pass-1 output (VD x P1) + A v (P1 x P1)
  static constexpr int z_sz = 2 * kTileRegion * ZP;
  static constexpr int un_sz = r32(blur_sz > z_sz ? blur_sz : z_sz);
  static constexpr int tp_off = un_off + un_sz;
  static size_t bytes(int N) { return ((size_t)tp_off + r32(N * F * F)) * sizeof(float) + 64; }
};

struct HvpTmaArgs {
  const PairDev* pairs;
  const TileDev* tiles;
  const CUtensorMap* in_maps;   // per pair: the input vector / matrix
  const CUtensorMap* f_maps;    // per pair: the fields d_j (z index = filter)
  const float* taps;            // N * F * F
  const double* ealpha;
  int N;
  float l2;
  float* out;
  int mult;                     // 0: batched vector, else columns of a batched n x mult matrix
  const int* cols;
  const int* mask;
  unsigned long long* pix;
  int* err;
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
template <int F, int RB>
__device__ __forceinline__ void blur_part(const float* vs, float* h1, float* av, const PairDev& pr, int oy, int ox,
                                          float l2, bool owner, int oby, int obx, float (&acc)[4][4]) {
  using G = TmaGeom<F>;
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
    for (int j = 0; j < 4; ++j)
      if (!(rin && ix + j >= 0 && ix + j < pr.w)) o[j] = 0.f;
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

template <int F>
__global__ void __launch_bounds__(kStencilThreads, 2) k_hvp_tma(HvpTmaArgs a) {
  using G = TmaGeom<F>;
  constexpr int R = G::R, TILE = G::TILE, VD = G::VD, E1 = G::E1, FW = G::FW, FH = G::FH, ZP = G::ZP;
  constexpr int NB = TILE / 4;                               // owner blocks per side
  const TileDev tl = a.tiles[blockIdx.x];
  const int col = blockIdx.y;
  if (a.mask && !a.mask[tl.pair]) return;
  if (a.mult && col >= a.cols[tl.pair]) return;
  const PairDev pr = a.pairs[tl.pair];
  if (a.pix && threadIdx.x == 0)
    atomicAdd(a.pix, (unsigned long long)(min(TILE, pr.h - tl.oy) * min(TILE, pr.w - tl.ox)));

  extern __shared__ __align__(128) float sm[];
  float* vs = sm;
  float* fb0 = sm + G::fb_off;
  float* un = sm + G::un_off;
  float* tps = sm + G::tp_off;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tps + G::r32(a.N * F * F));   // [0] input, [1..2] fields
  const int tid = threadIdx.x;
  const int oy = tl.oy, ox = tl.ox;
  const int fx0 = (ox - R) & ~3, foff = ox - R - fx0;       // field box origin (16-byte aligned x)
  const CUtensorMap* imap = a.in_maps + tl.pair;
  const CUtensorMap* fmap = a.f_maps + tl.pair;
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
  bool in_done = mbar_wait(bar_in, 0);
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
      case 0: blur_part<F, 0>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      case 1: blur_part<F, 1>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      case 2: blur_part<F, 2>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      case 3: blur_part<F, 3>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
      default: blur_part<F, 4>(vs, h1, av, pr, oy, ox, a.l2, owner, oby, obx, outacc); break;
    }
  }
  __syncthreads();   // the blur temporaries are dead: the union region now holds z

  {
    // regulariser part: per filter z_j = d_j .* (K_j v) on the tile grown by R, then K_j^T z_j
    const int sby = tid >> 4, sbx = tid & 15;               // step-1 block of this thread
    constexpr bool kAligned = (kHalo - 2 * R) % 4 == 0 && VD % 4 == 0 && ZP % 4 == 0;
    const bool s1_live = 4 * sby < E1 && 4 * sbx < E1 && oy - R + 4 * sby < pr.h && ox - R + 4 * sbx < pr.w &&
                         oy - R + 4 * sby + 3 >= 0 && ox - R + 4 * sbx + 3 >= 0;
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
      float u[4][4];
#pragma unroll
      for (int yy = 0; yy < 4; ++yy)
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) u[yy][xx] = 0.f;
      if (s1_live)
        corr_block<F, 4, 4, false, kAligned>(&vs[(4 * sby + kHalo - 2 * R) * VD + 4 * sbx + kHalo - 2 * R], VD, k, u);
      ok = mbar_wait(bar_f0 + 8 * (jf & 1), (jf >> 1) & 1);
      if (ok) f_done = jf + 1;
      const float* fb = fb0 + (jf & 1) * G::fb_sz;
      float* zb = zs + (jf & 1) * (kTileRegion * ZP);
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) {
        float z[4];
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) z[xx] = s1_live ? fb[(4 * sby + yy) * FW + 4 * sbx + xx + foff] * u[yy][xx] : 0.f;
        *reinterpret_cast<float4*>(zb + (4 * sby + yy) * ZP + 4 * sbx) = make_float4(z[0], z[1], z[2], z[3]);
      }
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

// ---------------------------------------------------------------------------------------------
// Host side: tensor maps and the launcher

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
size_t smem_bytes(int N) { return TmaGeom<F>::bytes(N); }

size_t hvp_tma_smem(int F, int N) {
  switch (F) {
    case 1: return smem_bytes<1>(N);
    case 3: return smem_bytes<3>(N);
    case 5: return smem_bytes<5>(N);
    default: return smem_bytes<7>(N);
  }
}

int box_side(int F) { return tile_out(F) + 2 * kHalo; }
int field_width(int F) { return F == 1 ? kTileRegion : kTileRegion + 4; }

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

}  // namespace

bl_status hvp_tma_setup(bl_problem* P) {
  P->tma = false;
  if (P->prec != BL_FP32 || P->reg.kind != BL_REG_FOE || P->N < 1) return BL_OK;
  for (const auto& ph : P->ph)
    if (ph.w % 4 != 0) return BL_OK;           // rows or tile origins would not be 16-byte aligned
  if (P->n_tot % 4 != 0) return BL_OK;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return BL_OK;                       // driver without tensor maps: the generic kernel runs
  // slot 0: fields; slots 1..: the inputs the Hessian action is launched on
  struct In { const void* ptr; int mult; };
  const In ins[] = {{P->pv, 0}, {P->w, 0}, {P->r, 0}, {P->Wt, P->TM}, {P->U, P->SMAX}};
  const int nslots = 1 + (int)(sizeof(ins) / sizeof(ins[0]));
  std::vector<CUtensorMap> maps((size_t)nslots * P->K);
  const int VD = box_side(P->F), FW = field_width(P->F);
  for (int k = 0; k < P->K; ++k) {
    const auto& ph = P->ph[k];
    bl_status st = encode(fn, &maps[k], (const float*)P->fd + ph.off, ph.w, ph.h, P->N, P->n_tot, FW, kTileRegion);
    if (st != BL_OK) return st;
    for (int s = 0; s + 1 < nslots; ++s) {
      const In& in = ins[s];
      const float* base = (const float*)in.ptr + ph.off * std::max(1, in.mult);
      st = encode(fn, &maps[(size_t)(s + 1) * P->K + k], base, ph.w, ph.h, std::max(1, in.mult), ph.n, VD, VD);
      if (st != BL_OK) return st;
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
  P->tma = true;
  return BL_OK;
}

int hvp_tma_slot(const bl_problem* P, const void* in, int mult) {
  if (!P->tma) return -1;
  for (int s = 0; s < P->tma_slots; ++s)
    if (P->tma_in_ptr[s] == in && P->tma_in_mult[s] == mult) return s;
  return -1;
}

template <int F>
static bl_status launch_f(bl_problem* P, const HvpTmaArgs& a, dim3 grid) {
  const size_t sm = TmaGeom<F>::bytes(P->N);
  if (!P->capturing)
    BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_hvp_tma<F><<<grid, kStencilThreads, sm, P->stream>>>(a);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

bl_status launch_hvp_tma(bl_problem* P, int slot, const void* in, void* out, int mult, int cols, const int* mask) {
  (void)in;
  HvpTmaArgs a{};
  a.pairs = P->d_pairs;
  a.tiles = P->d_tiles;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P->d_tmaps);
  a.f_maps = maps;
  a.in_maps = maps + (size_t)(slot + 1) * P->K;
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
  dim3 grid(P->n_tiles, mult ? cols : 1);
  switch (P->F) {
    case 1: return launch_f<1>(P, a, grid);
    case 3: return launch_f<3>(P, a, grid);
    case 5: return launch_f<5>(P, a, grid);
    case 7: return launch_f<7>(P, a, grid);
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
}

bl_status prepare_hvp_tma(bl_problem* P) {
  if (!P->tma) return BL_OK;
  const size_t sm = hvp_tma_smem(P->F, P->N);
  switch (P->F) {
    case 1: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    case 3: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    case 5: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
    default: BL_CUDA_TRY(cudaFuncSetAttribute(k_hvp_tma<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); break;
  }
  return BL_OK;
}

}  // namespace bl
