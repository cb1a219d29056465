// Stencil kernels of the lower-level functional (eqs. (1.1), (2.6), (2.7), (5.1)).
//
// FoE problems use one fused tile kernel for both the Hessian action
//   H v = 2 A^T A v + l2 v + sum_j K_j^T (d_j .* K_j v),  d_j = e^{alpha_j} phi''(K_j x^)
// and the gradient
//   grad Phi = 2 A^T (A x - y) + l2 x + sum_j e^{alpha_j} K_j^T phi'(K_j x).
// A CTA stages the input tile with an 8-pixel halo in shared memory, applies the separable
// blur twice (the intermediate A v is truncated to the image, as the zero boundary requires),
// and for every filter forms z_j = d_j .* (K_j v) on the tile grown by the filter radius
// before accumulating K_j^T z_j into registers.  Each thread owns a 4x4 pixel block and
// runs both correlations from register windows.
//
// TV problems (small, FP64 configurations) use simple per-pixel kernels.
#include "common.cuh"
#include "device.cuh"

namespace bl {

// Asynchronous global -> shared copies of single elements (cp.async, L1-allocating).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T>
struct StencilArgs {
  const PairDev* pairs;
  const TileDev* tiles;
  const T* in;
  int mult;            // 0: plain batched vector, else columns of a batched n x mult matrix
  T* out;
  const T* y;          // GRAD: measurements
  const T* fd;         // HVP: fields d_j (N x n_tot)
  const T* taps;       // N * F * F
  const double* ealpha;
  int N;
  T l2, eps;
  int phi;
  const int* mask;     // per pair, may be null
  const int* cols;     // per pair column counts (mult != 0)
  long long n_tot;
  // fused dot products (HVP with dots): p^T q, C^T q, Z^T q
  int dots;
  const T* C;
  const T* Z;
  int SMAX;
  const int* s_k;
  const int* hasz;
  double* tpart;
  int ncomp;
  unsigned long long* pix;   // work counter (profiling), may be null
};

constexpr int kModeHvp = 0;
constexpr int kModeGrad = 1;

template <typename T, int F>
struct StencilSmem {
  static constexpr int R = F / 2;
  static constexpr int TILE = tile_out(F);
  static constexpr int VD = TILE + 2 * kHalo;       // staged input side
  static constexpr int ZP = kTileRegion + 4;        // pitch of the z buffer
  static constexpr int E2MAX = TILE + 2 * BL_MAX_BLUR_RADIUS;
  static constexpr size_t vs = (size_t)VD * VD;
  static constexpr size_t zs = 2 * (size_t)kTileRegion * ZP;   // double-buffered z_j
  static constexpr size_t h1 = (size_t)VD * VD;
  static constexpr size_t av = (size_t)E2MAX * E2MAX;
  __host__ __device__ static size_t taps(int N) { return ((size_t)N * F * F + 1) & ~(size_t)1; }   // keeps red 8-byte aligned
  static size_t bytes(int N) {
    return (vs + zs + h1 + av + taps(N)) * sizeof(T) + 64 * 9 * sizeof(double);
  }
};

template <typename T, int F, int MODE>
__global__ void __launch_bounds__(kStencilThreads, sizeof(T) == 4 ? 2 : 1) k_foe_stencil(StencilArgs<T> a) {
  using S = StencilSmem<T, F>;
  constexpr int R = S::R, TILE = S::TILE, VD = S::VD, ZP = S::ZP;
  constexpr int NB = TILE / 4;                       // owner blocks per side
  const TileDev tl = a.tiles[blockIdx.x];
  const PairDev pr = a.pairs[tl.pair];
  const int col = blockIdx.y;
  if (a.mask && !a.mask[tl.pair]) return;
  if (a.mult && col >= a.cols[tl.pair]) return;
  if (a.pix && threadIdx.x == 0)
    atomicAdd(a.pix, (unsigned long long)(min(TILE, pr.h - tl.oy) * min(TILE, pr.w - tl.ox)));

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vs = reinterpret_cast<T*>(smem_raw);
  T* zs = vs + S::vs;
  T* h1 = zs + S::zs;
  T* av = h1 + S::h1;
  T* tps = av + S::av;
  double* red = reinterpret_cast<double*>(tps + S::taps(a.N));   // 64 x 9 doubles

  const int tid = threadIdx.x;
  const int h = pr.h, w = pr.w, rb = pr.rb;
  const int oy = tl.oy, ox = tl.ox;
  const T* in = col_ptr(a.in, pr, a.mult, col);

  // ---- stage the input tile with halo (zero outside the image) and the taps ----
  for (int idx = tid; idx < VD * VD; idx += kStencilThreads) {
    const int i = idx / VD, j = idx - (idx / VD) * VD;
    const int iy = oy - kHalo + i, ix = ox - kHalo + j;
    vs[idx] = (iy >= 0 && iy < h && ix >= 0 && ix < w) ? in[(long long)iy * w + ix] : T(0);
  }
  for (int idx = tid; idx < a.N * F * F; idx += kStencilThreads) tps[idx] = a.taps[idx];
  __syncthreads();

  const bool owner = tid < NB * NB;
  const int oby = owner ? tid / NB : 0, obx = owner ? tid - (tid / NB) * NB : 0;
  T outacc[4][4];
  Accum<T> dterm;                                       // GRAD: ||A x - y||^2 over the tile
  if (pr.opm) {
    // ---- inpainting data term: A^T A = diag(m): 2 m v (HVP) or 2 m (x - y) (GRAD) ----
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int iy = oy + 4 * oby + yy, ix = ox + 4 * obx + xx;
        const T vv = vs[(4 * oby + yy + kHalo) * VD + 4 * obx + xx + kHalo];
        T s = 0;
        if (owner && 4 * oby + yy < TILE && 4 * obx + xx < TILE && iy < h && ix < w) {
          const long long pl = (long long)iy * w + ix;
          if (pr.opm[pl]) {
            s = MODE == kModeGrad ? vv - a.y[pr.off + pl] : vv;
            if (MODE == kModeGrad) dterm.add(s * s);
          }
        }
        outacc[yy][xx] = T(2) * s + a.l2 * vv;
      }
  } else {
  // ---- blur part: A (A v) (HVP) or A (A x - y) (GRAD), separable passes in smem ----
  const int E2 = TILE + 2 * rb;                       // region of A v: tile grown by r_b
  T g[2 * BL_MAX_BLUR_RADIUS + 1];
#pragma unroll
  for (int b = 0; b < 2 * BL_MAX_BLUR_RADIUS + 1; ++b)
    g[b] = (b <= 2 * rb) ? (sizeof(T) == 4 ? (T)pr.gf[b] : (T)pr.gd[b]) : T(0);
  const int sh = kHalo - 2 * rb;
  // h1[y][x] = sum_b g[b] vs[y][x + b + sh]   (y in [0, VD), x in [0, E2))
  for (int idx = tid; idx < VD * E2; idx += kStencilThreads) {
    const int y = idx / E2, x = idx - (idx / E2) * E2;
    T s = 0;
#pragma unroll
    for (int b = 0; b < 2 * BL_MAX_BLUR_RADIUS + 1; ++b)
      if (b <= 2 * rb) s = fma(g[b], vs[y * VD + x + b + sh], s);
    h1[y * VD + x] = s;
  }
  __syncthreads();
  // av[i][x] = sum_a g[a] h1[i + a + sh][x], masked to the image (and minus y in GRAD mode)
  for (int idx = tid; idx < E2 * E2; idx += kStencilThreads) {
    const int i = idx / E2, x = idx - (idx / E2) * E2;
    T s = 0;
#pragma unroll
    for (int b = 0; b < 2 * BL_MAX_BLUR_RADIUS + 1; ++b)
      if (b <= 2 * rb) s = fma(g[b], h1[(i + b + sh) * VD + x], s);
    const int iy = oy - rb + i, ix = ox - rb + x;
    const bool inside = iy >= 0 && iy < h && ix >= 0 && ix < w;
    if (MODE == kModeGrad && inside) {
      s -= a.y[pr.off + (long long)iy * w + ix];
      if (i >= rb && i < rb + TILE && x >= rb && x < rb + TILE) dterm.add(s * s);
    }
    av[i * S::E2MAX + x] = inside ? s : T(0);
  }
  __syncthreads();
  // second pass, horizontal: h1[i][x] = sum_b g[b] av[i][x + b]   (i in [0, E2), x in [0, TILE))
  for (int idx = tid; idx < E2 * TILE; idx += kStencilThreads) {
    const int i = idx / TILE, x = idx - (idx / TILE) * TILE;
    T s = 0;
#pragma unroll
    for (int b = 0; b < 2 * BL_MAX_BLUR_RADIUS + 1; ++b)
      if (b <= 2 * rb) s = fma(g[b], av[i * S::E2MAX + x + b], s);
    h1[i * VD + x] = s;
  }
  __syncthreads();

#pragma unroll
  for (int yy = 0; yy < 4; ++yy)
#pragma unroll
    for (int xx = 0; xx < 4; ++xx) {
      T s = 0;
#pragma unroll
      for (int b = 0; b < 2 * BL_MAX_BLUR_RADIUS + 1; ++b)
        if (b <= 2 * rb) s = fma(g[b], h1[(4 * oby + yy + b) * VD + 4 * obx + xx], s);
      outacc[yy][xx] = T(2) * s + a.l2 * vs[(4 * oby + yy + kHalo) * VD + 4 * obx + xx + kHalo];
    }
  }
  __syncthreads();

  // ---- regulariser part: per filter z_j on the tile grown by R, then K_j^T z_j ----
  const int sby = tid >> 4, sbx = tid & 15;             // step-1 block of this thread
  constexpr int E1 = TILE + 2 * R;
  constexpr bool kAligned = (kHalo - 2 * R) % 4 == 0 && VD % 4 == 0 && ZP % 4 == 0;
  Accum<T> rterm;                                       // GRAD: sum e^alpha phi(u) over the tile
  // HVP: the 16 field values d_j of this thread's step-1 block are prefetched one filter ahead
  // with cp.async into a per-thread slot of a double buffer that reuses the (now dead) blur
  // buffers; element e of thread t sits at e * 256 + t, so the reads are conflict-free.
  T* dbuf = h1;
  // 4x4 blocks wholly outside the image (ragged tiles) or beyond the region skip their arithmetic
  const bool s1_live = 4 * sby < E1 && 4 * sbx < E1 && oy - R + 4 * sby < h && ox - R + 4 * sbx < w &&
                       oy - R + 4 * sby + 3 >= 0 && ox - R + 4 * sbx + 3 >= 0;
  const bool s2_live = owner && oy + 4 * oby < h && ox + 4 * obx < w;
  __syncthreads();                                      // every thread is done with h1 / av
  // which of the block's 16 field values lie in the image (fixed over the filters), and the
  // offset of its top-left pixel in one field; filter jf adds jf * n_tot
  unsigned fmask = 0;
#pragma unroll
  for (int yy = 0; yy < 4; ++yy)
#pragma unroll
    for (int xx = 0; xx < 4; ++xx) {
      const int ey = 4 * sby + yy, ex = 4 * sbx + xx;
      const int iy = oy - R + ey, ix = ox - R + ex;
      if (ey < E1 && ex < E1 && iy >= 0 && iy < h && ix >= 0 && ix < w) fmask |= 1u << (yy * 4 + xx);
    }
  const long long fofs = pr.off + (long long)(oy - R + 4 * sby) * w + (ox - R + 4 * sbx);
  auto prefetch = [&](int jf, int buf) {
    const T* fb = a.fd + (long long)jf * a.n_tot + fofs;
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        T* dst = &dbuf[(buf * 16 + yy * 4 + xx) * kStencilThreads + tid];
        if (fmask & (1u << (yy * 4 + xx)))
          cp_async_elem(dst, fb + yy * w + xx);
        else
          *dst = T(0);
      }
  };
  if (MODE == kModeHvp && a.N > 0) prefetch(0, 0);
  cp_async_commit();
  for (int jf = 0; jf < a.N; ++jf) {
    if (MODE == kModeHvp && jf + 1 < a.N) prefetch(jf + 1, (jf + 1) & 1);
    cp_async_commit();
    T k[F * F];
#pragma unroll
    for (int t = 0; t < F * F; ++t) k[t] = tps[jf * F * F + t];
    const T ea = (T)a.ealpha[jf];
    T u[4][4];
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) u[yy][xx] = 0;
    if (s1_live)
      corr_block<F, 4, 4, false, kAligned>(&vs[(4 * sby + kHalo - 2 * R) * VD + 4 * sbx + kHalo - 2 * R], VD, k, u);
    T* zb = zs + (jf & 1) * (kTileRegion * ZP);
    if (MODE == kModeHvp) cp_async_wait_prev();       // this thread's d_j values have landed
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int ey = 4 * sby + yy, ex = 4 * sbx + xx;
        T z = 0;
        if (MODE == kModeHvp) {
          z = dbuf[((jf & 1) * 16 + yy * 4 + xx) * kStencilThreads + tid] * u[yy][xx];
        } else {
          const int iy = oy - R + ey, ix = ox - R + ex;
          if (ey < E1 && ex < E1 && iy >= 0 && iy < h && ix >= 0 && ix < w) {
            T f0, d1, d2;
            phi_all(u[yy][xx], a.eps, a.phi, f0, d1, d2);
            z = ea * d1;
            if (ey >= R && ey < R + TILE && ex >= R && ex < R + TILE) rterm.add(ea * f0);
          }
        }
        zb[ey * ZP + ex] = z;
      }
    // one barrier per filter: z is double-buffered, so the buffer written next iteration was last
    // read before this barrier
    __syncthreads();
    if (s2_live) corr_block<F, 4, 4, true, kAligned>(&zb[(4 * oby) * ZP + 4 * obx], ZP, k, outacc);
  }
  __syncthreads();

  // ---- write the owned block ----
  T* out = col_ptr(a.out, pr, a.mult, col);
  if (owner) {
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int iy = oy + 4 * oby + yy, ix = ox + 4 * obx + xx;
        if (4 * oby + yy < TILE && 4 * obx + xx < TILE && iy < h && ix < w)
          out[(long long)iy * w + ix] = outacc[yy][xx];
      }
  }

  if (MODE == kModeGrad) {
    // value partials of this tile: ||A x - y||^2, sum e^alpha phi, ||x||^2 (owned pixels)
    Accum<T> xx2;
    if (owner) {
      for (int yy = 0; yy < 4; ++yy)
        for (int xx = 0; xx < 4; ++xx) {
          const int iy = oy + 4 * oby + yy, ix = ox + 4 * obx + xx;
          if (4 * oby + yy < TILE && 4 * obx + xx < TILE && iy < h && ix < w) {
            const T v = vs[(4 * oby + yy + kHalo) * VD + 4 * obx + xx + kHalo];
            xx2.add(v * v);
          }
        }
    }
    const double t0 = block_total<kStencilThreads>(dterm, red);
    const double t1 = block_total<kStencilThreads>(rterm, red);
    const double t2 = block_total<kStencilThreads>(xx2, red);
    if (tid == 0) {
      a.tpart[(size_t)blockIdx.x * 3 + 0] = t0;
      a.tpart[(size_t)blockIdx.x * 3 + 1] = t1;
      a.tpart[(size_t)blockIdx.x * 3 + 2] = t2;
    }
  }

  if (MODE == kModeHvp && a.dots) {
    // tile partials: [0] p^T q, [1 .. s] C^T q, [1 + SMAX .. 1 + SMAX + s) Z^T q.  q is staged in the
    // (now free) z buffer; each warp then streams whole columns of C or Z over the tile's rows
    // (coalesced), summing in compensated FP32 per lane and in FP64 across lanes.
    const int s = a.s_k[tl.pair];
    const int nz = a.hasz[tl.pair] ? s : 0;
    const int lane = tid & 31, wid = tid >> 5;
    const int vh = min(TILE, h - oy), vw = min(TILE, w - ox);
    T* qs = zs;
    if (owner) {
#pragma unroll
      for (int yy = 0; yy < 4; ++yy)
#pragma unroll
        for (int xx = 0; xx < 4; ++xx)
          if (4 * oby + yy < vh && 4 * obx + xx < vw) qs[(4 * oby + yy) * TILE + 4 * obx + xx] = outacc[yy][xx];
    }
    __syncthreads();
    const T* Cb = a.C + pr.off * a.SMAX;
    const T* Zb = a.Z + pr.off * a.SMAX;
    for (int cc = wid; cc < 1 + s + nz; cc += kStencilThreads / 32) {
      Accum<T> acc;
      if (cc == 0) {
        for (int i = 0; i < vh; ++i)
          for (int j = lane; j < vw; j += 32) acc.add(vs[(i + kHalo) * VD + j + kHalo] * qs[i * TILE + j]);
      } else {
        // 8 rows x 2 lane positions of loads are issued before their products are accumulated,
        // so a warp keeps 16 global loads in flight instead of one
        const T* col = cc <= s ? Cb + (long long)(cc - 1) * pr.n : Zb + (long long)(cc - 1 - s) * pr.n;
        for (int i0 = 0; i0 < vh; i0 += 8) {
          T v[8][2];
#pragma unroll
          for (int ii = 0; ii < 8; ++ii)
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
              const int i = i0 + ii, j = lane + 32 * jj;
              v[ii][jj] = (i < vh && j < vw) ? col[(long long)(oy + i) * w + ox + j] : T(0);
            }
#pragma unroll
          for (int ii = 0; ii < 8; ++ii)
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
              const int i = i0 + ii, j = lane + 32 * jj;
              if (i < vh && j < vw) acc.add(v[ii][jj] * qs[i * TILE + j]);
            }
        }
      }
      const double v = warp_total(acc);
      if (lane == 0) {
        const int slot = cc <= s ? cc : cc - s + a.SMAX;   // Z^T q after SMAX C slots
        a.tpart[(size_t)blockIdx.x * a.ncomp + slot] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Fields at the current point: u_j = k_j * x^ and d_j = e^{alpha_j} phi''(u_j) (eq. (5.1)).
template <typename T, int F>
__global__ void k_fields(const PairDev* pairs, const ChunkDev* chunks, const T* x, const T* taps,
                         const double* ealpha, int N, T eps, int phi, long long n_tot, T* fu, T* fd,
                         const int* mask) {
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  constexpr int R = F / 2;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long pl = ch.start + t;
    const int i = (int)(pl / pr.w), j = (int)(pl - (long long)(pl / pr.w) * pr.w);
    T win[F * F];
#pragma unroll
    for (int a = 0; a < F; ++a)
#pragma unroll
      for (int b = 0; b < F; ++b) {
        const int ii = i + a - R, jj = j + b - R;
        win[a * F + b] = (ii >= 0 && ii < pr.h && jj >= 0 && jj < pr.w)
                             ? x[pr.off + (long long)ii * pr.w + jj] : T(0);
      }
    for (int jf = 0; jf < N; ++jf) {
      T u = 0;
#pragma unroll
      for (int o = 0; o < F * F; ++o) u = fma(taps[jf * F * F + o], win[o], u);
      const long long idx = (long long)jf * n_tot + pr.off + pl;
      fu[idx] = u;
      fd[idx] = (T)ealpha[jf] * phi_d2(u, eps, phi);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// J w for FoE (eq. (2.7) with eq. (5.1)): per filter j, with u = k_j * x^, e = phi'(u),
//   (J w)_{alpha_j}  = -e^{alpha_j} sum_p e_p (k_j * w)_p
//   (J w)_{k_j[o]}   = -e^{alpha_j} sum_p [ e_p w_{p+o} + phi''(u_p) (k_j * w)_p x^_{p+o} ]
// Tile partials: tpart[((col * n_tiles) + tile) * p + m].
// Row pitch of the staged w and x^ tiles of the J w kernel.  FP32: a multiple of 4 floats with an
// odd number of 16-byte units, so the 128-bit row-segment reads of the lanes of a warp (consecutive
// 4-pixel blocks, several block rows) fall in distinct bank groups.  FP64 keeps the plain side
// (its scalar reads gain nothing, and the 7x7 FP64 tile needs the shared memory).
template <typename T>
__host__ __device__ constexpr int jw_pitch(int rs) {
  return sizeof(T) != 4 ? rs : (((rs + 3) / 4) % 2 == 1 ? ((rs + 3) / 4) * 4 : ((rs + 3) / 4) * 4 + 4);
}

template <typename T, int F>
__global__ void __launch_bounds__(kStencilThreads, sizeof(T) == 4 ? 2 : 1)
k_foe_jw(const PairDev* pairs, const TileDev* tiles, int n_tiles, const T* win, int mult,
         const int* cols, const T* xhat, const T* fu, const T* taps, const double* ealpha, int N,
         T eps, int phi, long long n_tot, const int* mask, double* tpart, int p, unsigned long long* pix,
         int colfast) {
  constexpr int R = F / 2, TILE = jw_tile_out<T>(F), RS = TILE + 2 * R;   // staged region side
  constexpr int RP = jw_pitch<T>(RS);                                 // its row pitch
  constexpr int NB = TILE / 4, FF = F * F;
  // colfast: grid x runs over the columns of one tile, so its x^ and field tiles are read from L2
  const int ti = colfast ? blockIdx.y : blockIdx.x;
  const TileDev tl = tiles[ti];
  const PairDev pr = pairs[tl.pair];
  const int col = colfast ? blockIdx.x : blockIdx.y;
  if (mask && !mask[tl.pair]) return;
  if (mult && col >= cols[tl.pair]) return;
  if (pix && threadIdx.x == 0)
    atomicAdd(pix, (unsigned long long)(min(TILE, pr.h - tl.oy) * min(TILE, pr.w - tl.ox)));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ws = reinterpret_cast<T*>(smem_raw);
  T* xs = ws + RS * RP;
  T* fbuf = xs + RS * RP;                                             // 2 x 16 x 256 prefetched u_j
  T* rf = fbuf + 2 * 16 * kStencilThreads;                            // (FF + 1) x 256 per-thread sums
  const int tid = threadIdx.x, lane = tid & 31;
  const T* wv = col_ptr(win, pr, mult, col);
  constexpr bool kAligned = RP % 4 == 0;
  for (int idx = tid; idx < RS * RS; idx += kStencilThreads) {
    const int i = idx / RS, j = idx - (idx / RS) * RS;
    const int iy = tl.oy - R + i, ix = tl.ox - R + j;
    const bool in = iy >= 0 && iy < pr.h && ix >= 0 && ix < pr.w;
    ws[i * RP + j] = in ? wv[(long long)iy * pr.w + ix] : T(0);
    xs[i * RP + j] = in ? xhat[pr.off + (long long)iy * pr.w + ix] : T(0);
  }
  __syncthreads();
  const bool owner = tid < NB * NB;
  const int oby = owner ? tid / NB : 0, obx = owner ? tid - (tid / NB) * NB : 0;
  double* outp = tpart + ((size_t)col * n_tiles + ti) * p;
  // u_j of this thread's 16 pixels is prefetched one filter ahead (cp.async, per-thread slots)
  auto prefetch = [&](int jf, int buf) {
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int iy = tl.oy + 4 * oby + yy, ix = tl.ox + 4 * obx + xx;
        T* dst = &fbuf[(buf * 16 + yy * 4 + xx) * kStencilThreads + tid];
        if (owner && 4 * oby + yy < TILE && 4 * obx + xx < TILE && iy < pr.h && ix < pr.w)
          cp_async_elem(dst, &fu[(long long)jf * n_tot + pr.off + (long long)iy * pr.w + ix]);
        else
          *dst = T(0);
      }
  };
  if (N > 0) prefetch(0, 0);
  cp_async_commit();
  for (int jf = 0; jf < N; ++jf) {
    if (jf + 1 < N) prefetch(jf + 1, (jf + 1) & 1);
    cp_async_commit();
    T k[FF];
#pragma unroll
    for (int t = 0; t < FF; ++t) k[t] = taps[jf * FF + t];
    T kw[4][4], e[4][4], d[4][4];
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) kw[yy][xx] = 0;
    corr_block<F, 4, 4, false, kAligned>(&ws[(4 * oby) * RP + 4 * obx], RP, k, kw);
    cp_async_wait_prev();
    T ga = 0;
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
      for (int xx = 0; xx < 4; ++xx) {
        const int iy = tl.oy + 4 * oby + yy, ix = tl.ox + 4 * obx + xx;
        const bool in = owner && 4 * oby + yy < TILE && 4 * obx + xx < TILE && iy < pr.h && ix < pr.w;
        T ee = 0, dd = 0;
        if (in) {
          const T uu = fbuf[((jf & 1) * 16 + yy * 4 + xx) * kStencilThreads + tid];
          ee = phi_d1(uu, eps, phi);
          dd = phi_d2(uu, eps, phi) * kw[yy][xx];
          ga = fma(ee, kw[yy][xx], ga);
        }
        e[yy][xx] = ee;
        d[yy][xx] = dd;
      }
    T gt[FF];
#pragma unroll
    for (int t = 0; t < FF; ++t) gt[t] = 0;
#pragma unroll
    for (int ry = 0; ry < 4 + F - 1; ++ry) {
      T wseg[4 + F - 1], xseg[4 + F - 1];
      const int rbase = (4 * oby + ry) * RP + 4 * obx;
      if constexpr (sizeof(T) == 4 && (4 + F - 1) % 4 == 0) {
#pragma unroll
        for (int c = 0; c < 4 + F - 1; c += 4) {
          const float4 wv4 = *reinterpret_cast<const float4*>(&ws[rbase + c]);
          const float4 xv4 = *reinterpret_cast<const float4*>(&xs[rbase + c]);
          wseg[c] = wv4.x; wseg[c + 1] = wv4.y; wseg[c + 2] = wv4.z; wseg[c + 3] = wv4.w;
          xseg[c] = xv4.x; xseg[c + 1] = xv4.y; xseg[c + 2] = xv4.z; xseg[c + 3] = xv4.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4 + F - 1; ++c) {
          wseg[c] = ws[rbase + c];
          xseg[c] = xs[rbase + c];
        }
      }
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) {
        const int aa = ry - yy;
        if (aa < 0 || aa >= F) continue;
#pragma unroll
        for (int b = 0; b < F; ++b)
#pragma unroll
          for (int xx = 0; xx < 4; ++xx)
            gt[aa * F + b] = fma(e[yy][xx], wseg[xx + b], fma(d[yy][xx], xseg[xx + b], gt[aa * F + b]));
      }
    }
    // Block reduction of the FF + 1 sums: every thread parks its values in smem (value-major,
    // rf[v * 256 + thread]); then lane l of warp w sums value v = 4 w + l / 8 over the 32 threads
    // of segment l % 8 (rotated by the lane, so the 8 segments hit distinct banks) in compensated
    // FP32, and the 8 segment totals of a value combine in FP64 through 3 shuffles.
    rf[tid] = ga;
#pragma unroll
    for (int t = 0; t < FF; ++t) rf[(1 + t) * kStencilThreads + tid] = gt[t];
    __syncthreads();
    const double scale = -ealpha[jf];
    for (int job = tid; job < 8 * ((FF + 1 + 3) / 4) * 4; job += kStencilThreads) {
      const int v = job >> 3, seg = job & 7;
      Accum<T> acc;
      if (v < FF + 1) {
#pragma unroll 8
        for (int i = 0; i < 32; ++i) acc.add(rf[v * kStencilThreads + seg * 32 + ((i + lane) & 31)]);
      }
      double tot = acc.value();
      tot += __shfl_xor_sync(0xffffffffu, tot, 1);
      tot += __shfl_xor_sync(0xffffffffu, tot, 2);
      tot += __shfl_xor_sync(0xffffffffu, tot, 4);
      if (seg == 0 && v < FF + 1) outp[jf * (FF + 1) + v] = scale * tot;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Direct (non-fused) kernels used by the TV regulariser and by the forward operator.

// out = A in (minus y if y != null), zero boundary; one thread per pixel.  A: the pair's blur, or
// the inpainting mask.
template <typename T>
__global__ void k_blur(const PairDev* pairs, const ChunkDev* chunks, const T* in, const T* y, T* out,
                       const int* mask) {
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  if (pr.opm) {   // inpainting: A = diag(mask)
    for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
      const long long pl = ch.start + t;
      // unmeasured pixels carry no data: A x - y is zero there whatever y holds
      out[pr.off + pl] = pr.opm[pl] ? (y ? in[pr.off + pl] - y[pr.off + pl] : in[pr.off + pl]) : T(0);
    }
    return;
  }
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long pl = ch.start + t;
    const int i = (int)(pl / pr.w), j = (int)(pl - (pl / pr.w) * pr.w);
    T s = 0;
    for (int a = -pr.rb; a <= pr.rb; ++a) {
      const int ii = i + a;
      if (ii < 0 || ii >= pr.h) continue;
      T rs = 0;
      for (int b = -pr.rb; b <= pr.rb; ++b) {
        const int jj = j + b;
        if (jj < 0 || jj >= pr.w) continue;
        const T gb = sizeof(T) == 4 ? (T)pr.gf[b + pr.rb] : (T)pr.gd[b + pr.rb];
        rs = fma(gb, in[pr.off + (long long)ii * pr.w + jj], rs);
      }
      const T ga = sizeof(T) == 4 ? (T)pr.gf[a + pr.rb] : (T)pr.gd[a + pr.rb];
      s = fma(ga, rs, s);
    }
    if (y) s -= y[pr.off + pl];
    out[pr.off + pl] = s;
  }
}

template <typename T>
__device__ __forceinline__ void tv_a(const T* x, const PairDev& pr, int i, int j, T& a0, T& a1) {
  const T c = x[pr.off + (long long)i * pr.w + j];
  a0 = (i + 1 < pr.h) ? x[pr.off + (long long)(i + 1) * pr.w + j] - c : T(0);
  a1 = (j + 1 < pr.w) ? x[pr.off + (long long)i * pr.w + j + 1] - c : T(0);
}

// q_p = B_p (D v)_p with B_p = (I - a a^T / s^2) / s, a = (D x^)_p, s = sqrt(|a|^2 + eps^2)
template <typename T>
__device__ __forceinline__ void tv_q(const T* xh, const T* v, const PairDev& pr, int i, int j, T eps,
                                     T& q0, T& q1) {
  T a0, a1, d0, d1;
  tv_a(xh, pr, i, j, a0, a1);
  tv_a(v, pr, i, j, d0, d1);
  const T s2 = a0 * a0 + a1 * a1 + eps * eps;
  const T is = rsqrt(s2);
  const T ad = (a0 * d0 + a1 * d1) / s2;
  q0 = (d0 - a0 * ad) * is;
  q1 = (d1 - a1 * ad) * is;
}

// D^T q at (i, j) for a field q given pointwise by a functor.
template <typename T, typename Q>
__device__ __forceinline__ T tv_div(const PairDev& pr, int i, int j, Q qf) {
  T q0, q1, r = 0;
  qf(i, j, q0, q1);
  if (i + 1 < pr.h) r -= q0;
  if (j + 1 < pr.w) r -= q1;
  if (i >= 1) {
    T u0, u1;
    qf(i - 1, j, u0, u1);
    r += u0;
  }
  if (j >= 1) {
    T u0, u1;
    qf(i, j - 1, u0, u1);
    r += u1;
  }
  return r;
}

// out = 2 * aav + l2 v + e^{theta_0} D^T (B D v)   (aav = A A v precomputed)
template <typename T>
__global__ void k_tv_hvp(const PairDev* pairs, const ChunkDev* chunks, const T* xh, const T* v,
                         const T* aav, T* out, const double* ealpha, T l2, T eps, const int* mask) {
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  const T et = (T)ealpha[0];
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long pl = ch.start + t;
    const int i = (int)(pl / pr.w), j = (int)(pl - (pl / pr.w) * pr.w);
    const T div = tv_div<T>(pr, i, j, [&](int ii, int jj, T& a, T& b) { tv_q(xh, v, pr, ii, jj, eps, a, b); });
    out[pr.off + pl] = T(2) * aav[pr.off + pl] + l2 * v[pr.off + pl] + et * div;
  }
}

// grad = 2 * aar + l2 x + e^{theta_0} D^T (a / s);
// chunk partials: [0] ||A x - y||^2, [1] e^{theta_0} sum_p s_p, [2] ||x||^2
template <typename T>
__global__ void k_tv_grad(const PairDev* pairs, const ChunkDev* chunks, const T* x, const T* ar,
                          const T* aar, T* out, const double* ealpha, T l2, T eps, const int* mask,
                          double* cpart) {
  __shared__ double red[40];
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  const T et = (T)ealpha[0];
  double ssum = 0, xx = 0, rr = 0;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long pl = ch.start + t;
    const int i = (int)(pl / pr.w), j = (int)(pl - (pl / pr.w) * pr.w);
    const T div = tv_div<T>(pr, i, j, [&](int ii, int jj, T& a, T& b) {
      T a0, a1;
      tv_a(x, pr, ii, jj, a0, a1);
      const T is = rsqrt(a0 * a0 + a1 * a1 + eps * eps);
      a = a0 * is;
      b = a1 * is;
    });
    const T xv = x[pr.off + pl];
    out[pr.off + pl] = T(2) * aar[pr.off + pl] + l2 * xv + et * div;
    T a0, a1;
    tv_a(x, pr, i, j, a0, a1);
    ssum += sqrt((double)(a0 * a0 + a1 * a1 + eps * eps));
    xx += (double)xv * (double)xv;
    const double rv = (double)ar[pr.off + pl];
    rr += rv * rv;
  }
  const double s0 = block_sum<kChunkThreads>(ssum, red);
  const double s1 = block_sum<kChunkThreads>(xx, red);
  const double s2 = block_sum<kChunkThreads>(rr, red);
  if (threadIdx.x == 0) {
    cpart[(size_t)blockIdx.x * 3 + 0] = s2;
    cpart[(size_t)blockIdx.x * 3 + 1] = (double)et * s0;
    cpart[(size_t)blockIdx.x * 3 + 2] = s1;
  }
}

// (J w) = -e^{theta_0} sum_p <a_p / s_p, (D w)_p>; chunk partials, one per column.
template <typename T>
__global__ void k_tv_jw(const PairDev* pairs, const ChunkDev* chunks, int n_chunks, const T* win,
                        int mult, const int* cols, const T* xh, const double* ealpha, T eps,
                        const int* mask, double* cpart) {
  __shared__ double red[40];
  const ChunkDev ch = chunks[blockIdx.x];
  const int col = blockIdx.y;
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  if (mult && col >= cols[ch.pair]) return;
  const T* wv = col_ptr(win, pr, mult, col);
  double acc = 0;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long pl = ch.start + t;
    const int i = (int)(pl / pr.w), j = (int)(pl - (pl / pr.w) * pr.w);
    T a0, a1, d0, d1;
    tv_a(xh, pr, i, j, a0, a1);
    const T c = wv[pl];
    d0 = (i + 1 < pr.h) ? wv[(long long)(i + 1) * pr.w + j] - c : T(0);
    d1 = (j + 1 < pr.w) ? wv[(long long)i * pr.w + j + 1] - c : T(0);
    const T is = rsqrt(a0 * a0 + a1 * a1 + eps * eps);
    acc += (double)((a0 * d0 + a1 * d1) * is);
  }
  const double s = block_sum<kChunkThreads>(acc, red);
  if (threadIdx.x == 0) cpart[(size_t)col * n_chunks + blockIdx.x] = -ealpha[0] * s;
}

// ---------------------------------------------------------------------------------------------
// Host launchers

template <typename T>
static bl_status hvp_foe(bl_problem* P, const void* in, void* out, int mult, int cols, const int* mask,
                         const int* dots_s, const int* dots_hz) {
  const bool dots = dots_s != nullptr;
  if (sizeof(T) == 4 && !dots) {
    const int slot = hvp_tma_slot(P, in, mult);
    if (slot >= 0) return launch_hvp_tma(P, slot, in, out, mult, cols, mask);
  }
  StencilArgs<T> a{};
  a.pairs = P->d_pairs;
  a.tiles = P->d_tiles;
  a.in = (const T*)in;
  a.mult = mult;
  a.out = (T*)out;
  a.fd = (const T*)P->fd;
  a.taps = P->prec == BL_FP32 ? (const T*)(const void*)P->taps_f : (const T*)(const void*)P->taps_d;
  a.ealpha = P->ealpha;
  a.N = P->N;
  a.l2 = (T)P->reg.l2_eps;
  a.eps = (T)P->reg.phi_eps;
  a.phi = P->reg.phi;
  a.mask = mask;
  a.cols = P->d_cols;
  a.n_tot = P->n_tot;
  a.dots = dots ? 1 : 0;
  a.C = (const T*)P->C;
  a.Z = (const T*)P->Z;
  a.SMAX = P->SMAX;
  a.s_k = dots_s;
  a.hasz = dots_hz;
  a.ncomp = 1 + 2 * P->SMAX;
  if (dots) {
    bl_status st = ensure_tpart(P, (size_t)P->n_tiles * a.ncomp);
    if (st != BL_OK) return st;
  }
  a.tpart = P->tpart;
  const int cls = mult ? BL_KC_HVP_MULTI : BL_KC_HVP;
  a.pix = pix_counter(P, cls);
  ProfScope ps(P, cls);
  dim3 grid(P->n_tiles, mult ? cols : 1);
#define BL_HVP_CASE(FF)                                                                           \
  case FF: {                                                                                      \
    size_t sm = StencilSmem<T, FF>::bytes(P->N);                                                  \
    if (!P->capturing)                                                                            \
      BL_CUDA_TRY(cudaFuncSetAttribute(k_foe_stencil<T, FF, kModeHvp>,                            \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));    \
    k_foe_stencil<T, FF, kModeHvp><<<grid, kStencilThreads, sm, P->stream>>>(a);                  \
    break;                                                                                        \
  }
  switch (P->F) {
    BL_HVP_CASE(1)
    BL_HVP_CASE(3)
    BL_HVP_CASE(5)
    BL_HVP_CASE(7)
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
#undef BL_HVP_CASE
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

template <typename T>
static bl_status hvp_tv(bl_problem* P, const void* in, void* out, int mult, int cols, const int* mask) {
  // TV path: one column at a time through the direct kernels.
  T* t1 = (T*)P->tmp;
  T* t2 = t1 + P->n_tot;
  const int ncol = mult ? cols : 1;
  ProfScope ps(P, mult ? BL_KC_HVP_MULTI : BL_KC_HVP);
  for (int c = 0; c < ncol; ++c) {
    // columns of a batched matrix are addressed per pair; gather them into plain vectors first
    const T* src = (const T*)in;
    T* dst = (T*)out;
    if (mult) {
      for (int k = 0; k < P->K; ++k) {
        const auto& ph = P->ph[k];
        BL_CUDA_TRY(cudaMemcpyAsync(t2 + ph.off, src + ph.off * mult + (long long)c * ph.n,
                                    ph.n * sizeof(T), cudaMemcpyDeviceToDevice, P->stream));
      }
      src = t2;
    }
    T* t3 = t2 + P->n_tot;
    k_blur<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, src, nullptr, t1, mask);
    BL_LAUNCH_CHECK(P);
    k_blur<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, t1, nullptr, t3, mask);
    BL_LAUNCH_CHECK(P);
    T* o = mult ? t1 : dst;
    k_tv_hvp<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const T*)P->xhat,
                                                               src, t3, o, P->ealpha, (T)P->reg.l2_eps,
                                                               (T)P->reg.phi_eps, mask);
    BL_LAUNCH_CHECK(P);
    if (mult) {
      for (int k = 0; k < P->K; ++k) {
        const auto& ph = P->ph[k];
        BL_CUDA_TRY(cudaMemcpyAsync(dst + ph.off * mult + (long long)c * ph.n, t1 + ph.off,
                                    ph.n * sizeof(T), cudaMemcpyDeviceToDevice, P->stream));
      }
    }
  }
  return BL_OK;
}

bl_status launch_hvp(bl_problem* P, const void* in, void* out, int mult, int cols, const int* mask,
                     const int* dots_s, const int* dots_hz) {
  if (P->reg.kind == BL_REG_TV) {
    if (dots_s) return fail(BL_EINVAL, "fused dots are only available for FoE problems");
    const int slot = hvp_tma_slot(P, in, mult);
    if (slot >= 0) return launch_hvp_tma(P, slot, in, out, mult, cols, mask);
    return P->prec == BL_FP32 ? hvp_tv<float>(P, in, out, mult, cols, mask)
                              : hvp_tv<double>(P, in, out, mult, cols, mask);
  }
  return P->prec == BL_FP32 ? hvp_foe<float>(P, in, out, mult, cols, mask, dots_s, dots_hz)
                            : hvp_foe<double>(P, in, out, mult, cols, mask, dots_s, dots_hz);
}

template <typename T>
static bl_status grad_impl(bl_problem* P, const void* x, void* grad, const int* mask, double* values) {
  if (P->reg.kind == BL_REG_TV) {
    T* t1 = (T*)P->tmp;
    T* t2 = t1 + P->n_tot;
    bl_status cst = ensure_cpart(P, (size_t)P->n_chunks * 3);
    if (cst != BL_OK) return cst;
    ProfScope ps(P, BL_KC_GRAD);
    k_blur<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const T*)x,
                                                             (const T*)P->y, t1, mask);
    BL_LAUNCH_CHECK(P);
    k_blur<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, t1, nullptr, t2, mask);
    BL_LAUNCH_CHECK(P);
    k_tv_grad<T><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const T*)x, t1, t2,
                                                                (T*)grad, P->ealpha, (T)P->reg.l2_eps,
                                                                (T)P->reg.phi_eps, mask, P->cpart);
    BL_LAUNCH_CHECK(P);
    if (values) {
      bl_status st = reduce_chunk_partials(P, 3, mask, values);
      if (st != BL_OK) return st;
    }
    return BL_OK;
  }
  if (sizeof(T) == 4) {
    const int slot = hvp_tma_grad_slot(P, x);
    if (slot >= 0) {
      bl_status st = ensure_tpart(P, (size_t)P->n_htiles * 3);
      if (st != BL_OK) return st;
      if ((st = launch_grad_tma(P, slot, grad, mask, P->tpart)) != BL_OK) return st;
      return values ? reduce_units(P, P->tpart, 3, 1, kUnitHTiles, mask, nullptr, values) : BL_OK;
    }
  }
  StencilArgs<T> a{};
  a.pairs = P->d_pairs;
  a.tiles = P->d_tiles;
  a.in = (const T*)x;
  a.mult = 0;
  a.out = (T*)grad;
  a.y = (const T*)P->y;
  a.taps = P->prec == BL_FP32 ? (const T*)(const void*)P->taps_f : (const T*)(const void*)P->taps_d;
  a.ealpha = P->ealpha;
  a.N = P->N;
  a.l2 = (T)P->reg.l2_eps;
  a.eps = (T)P->reg.phi_eps;
  a.phi = P->reg.phi;
  a.mask = mask;
  a.cols = P->d_cols;
  a.n_tot = P->n_tot;
  bl_status st = ensure_tpart(P, (size_t)P->n_tiles * 3);
  if (st != BL_OK) return st;
  a.tpart = P->tpart;
  a.pix = pix_counter(P, BL_KC_GRAD);
  ProfScope ps(P, BL_KC_GRAD);
  dim3 grid(P->n_tiles, 1);
#define BL_GRAD_CASE(FF)                                                                          \
  case FF: {                                                                                      \
    size_t sm = StencilSmem<T, FF>::bytes(P->N);                                                  \
    if (!P->capturing)                                                                            \
      BL_CUDA_TRY(cudaFuncSetAttribute(k_foe_stencil<T, FF, kModeGrad>,                           \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));    \
    k_foe_stencil<T, FF, kModeGrad><<<grid, kStencilThreads, sm, P->stream>>>(a);                 \
    break;                                                                                        \
  }
  switch (P->F) {
    BL_GRAD_CASE(1)
    BL_GRAD_CASE(3)
    BL_GRAD_CASE(5)
    BL_GRAD_CASE(7)
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
#undef BL_GRAD_CASE
  BL_LAUNCH_CHECK(P);
  if (values) return reduce_tile_partials(P, 3, 1, mask, values);
  return BL_OK;
}

bl_status launch_grad(bl_problem* P, const void* x, void* grad, const int* mask, double* values) {
  return P->prec == BL_FP32 ? grad_impl<float>(P, x, grad, mask, values)
                            : grad_impl<double>(P, x, grad, mask, values);
}

template <typename T>
static bl_status fields_impl(bl_problem* P, const int* mask) {
  if (P->reg.kind == BL_REG_TV) return BL_OK;   // TV recomputes from x^ on the fly
  ProfScope ps(P, BL_KC_OTHER);
  const T* taps = P->prec == BL_FP32 ? (const T*)(const void*)P->taps_f : (const T*)(const void*)P->taps_d;
#define BL_FIELDS_CASE(FF)                                                                        \
  case FF:                                                                                        \
    k_fields<T, FF><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(                                \
        P->d_pairs, P->d_chunks, (const T*)P->xhat, taps, P->ealpha, P->N, (T)P->reg.phi_eps,     \
        P->reg.phi, P->n_tot, (T*)P->fu, (T*)P->fd, mask);                                        \
    break;
  switch (P->F) {
    BL_FIELDS_CASE(1)
    BL_FIELDS_CASE(3)
    BL_FIELDS_CASE(5)
    BL_FIELDS_CASE(7)
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
#undef BL_FIELDS_CASE
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

bl_status launch_fields(bl_problem* P, const int* mask) {
  return P->prec == BL_FP32 ? fields_impl<float>(P, mask) : fields_impl<double>(P, mask);
}

bl_status launch_forward(bl_problem* P, const void* x, void* out, const int* mask) {
  if (P->prec == BL_FP32)
    k_blur<float><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const float*)x,
                                                                 nullptr, (float*)out, mask);
  else
    k_blur<double><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const double*)x,
                                                                  nullptr, (double*)out, mask);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

template <typename T>
static bl_status jw_impl(bl_problem* P, const void* in, int mult, int cols, const int* mask, double* out) {
  const int ncol = mult ? cols : 1;
  if (P->reg.kind == BL_REG_TV) {
    bl_status st = ensure_cpart(P, (size_t)P->n_chunks * ncol);
    if (st != BL_OK) return st;
    ProfScope ps(P, BL_KC_JW);
    dim3 grid(P->n_chunks, ncol);
    k_tv_jw<T><<<grid, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, P->n_chunks, (const T*)in, mult,
                                                       P->d_cols, (const T*)P->xhat, P->ealpha,
                                                       (T)P->reg.phi_eps, mask, P->cpart);
    BL_LAUNCH_CHECK(P);
    return reduce_units(P, P->cpart, 1, ncol, kUnitChunks, mask, mult ? P->d_cols : nullptr, out);
  }
  bl_status st = ensure_tpart(P, (size_t)P->n_jtiles * ncol * P->p);
  if (st != BL_OK) return st;
  const T* taps = P->prec == BL_FP32 ? (const T*)(const void*)P->taps_f : (const T*)(const void*)P->taps_d;
  const int colfast = (ncol > 1 && P->n_jtiles <= 65535) ? 1 : 0;
  const dim3 grid = colfast ? dim3(ncol, P->n_jtiles) : dim3(P->n_jtiles, ncol);
  ProfScope ps(P, BL_KC_JW);
  unsigned long long* pixc = pix_counter(P, BL_KC_JW);
#define BL_JW_CASE(FF)                                                                            \
  case FF: {                                                                                      \
    constexpr int RS = jw_tile_out<T>(FF) + 2 * (FF / 2);                                         \
    size_t sm = (2 * (size_t)RS * jw_pitch<T>(RS) + 2 * 16 * kStencilThreads +                    \
                 (size_t)(FF * FF + 1) * kStencilThreads) * sizeof(T);                            \
    if (!P->capturing)                                                                            \
      BL_CUDA_TRY(cudaFuncSetAttribute(k_foe_jw<T, FF>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                       (int)sm));                                                 \
    k_foe_jw<T, FF><<<grid, kStencilThreads, sm, P->stream>>>(                                    \
        P->d_pairs, P->d_jtiles, P->n_jtiles, (const T*)in, mult, P->d_cols, (const T*)P->xhat,   \
        (const T*)P->fu, taps, P->ealpha, P->N, (T)P->reg.phi_eps, P->reg.phi, P->n_tot, mask,    \
        P->tpart, P->p, pixc, colfast);                                                           \
    break;                                                                                        \
  }
  switch (P->F) {
    BL_JW_CASE(1)
    BL_JW_CASE(3)
    BL_JW_CASE(5)
    BL_JW_CASE(7)
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
#undef BL_JW_CASE
  BL_LAUNCH_CHECK(P);
  return reduce_units(P, P->tpart, P->p, ncol, kUnitJwTiles, mask, mult ? P->d_cols : nullptr, out);
}

bl_status launch_jw(bl_problem* P, const void* in, int mult, int cols, const int* mask, double* out) {
  return P->prec == BL_FP32 ? jw_impl<float>(P, in, mult, cols, mask, out)
                            : jw_impl<double>(P, in, mult, cols, mask, out);
}

}  // namespace bl

namespace bl {

template <typename T, int F>
static bl_status prepare_one(bl_problem* P) {
  const size_t sm = StencilSmem<T, F>::bytes(P->N);
  BL_CUDA_TRY(cudaFuncSetAttribute(k_foe_stencil<T, F, kModeHvp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  BL_CUDA_TRY(cudaFuncSetAttribute(k_foe_stencil<T, F, kModeGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  constexpr int RS = jw_tile_out<T>(F) + 2 * (F / 2);
  const size_t smj = (2 * (size_t)RS * jw_pitch<T>(RS) + 2 * 16 * kStencilThreads +
                      (size_t)(F * F + 1) * kStencilThreads) * sizeof(T);
  BL_CUDA_TRY(cudaFuncSetAttribute(k_foe_jw<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smj));
  return BL_OK;
}

template <typename T>
static bl_status prepare_t(bl_problem* P) {
  switch (P->F) {
    case 1: return prepare_one<T, 1>(P);
    case 3: return prepare_one<T, 3>(P);
    case 5: return prepare_one<T, 5>(P);
    case 7: return prepare_one<T, 7>(P);
    default: return fail(BL_EINVAL, "unsupported filter size");
  }
}

bl_status prepare_kernels(bl_problem* P) {
  if (P->reg.kind != BL_REG_FOE) return BL_OK;
  return P->prec == BL_FP32 ? prepare_t<float>(P) : prepare_t<double>(P);
}

}  // namespace bl
