// C-ABI entry points of libbl: problem set-up, data movement and the call sequence of eq. (5.2).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "device.cuh"

using namespace bl;

namespace {

// theta -> per-filter taps (FP32 and FP64 copies) and exp(alpha_j)   (Section 5 layout)
__global__ void k_theta(const double* theta, int N, int F, int reg, float* tf, double* td, double* ea) {
  const int FF = F * F;
  if (reg == BL_REG_TV) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ea[0] = exp(theta[0]);
    return;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * (FF + 1); i += gridDim.x * blockDim.x) {
    const int j = i / (FF + 1), t = i - j * (FF + 1);
    if (t == 0) ea[j] = exp(theta[i]);
    else {
      td[j * FF + t - 1] = theta[i];
      tf[j * FF + t - 1] = (float)theta[i];
    }
  }
}

template <typename T>
__global__ void k_sub(const PairDev* pairs, const ChunkDev* chunks, const T* a, const T* b, T* out, const int* mask) {
  const ChunkDev ch = chunks[blockIdx.x];
  if (!mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long gi = pr.off + ch.start + t;
    out[gi] = a[gi] - b[gi];
  }
}

// rows of the listed pairs and their mean: grads[i][m] = all[pairs[i]][m]
__global__ void k_pick_rows(const double* all, const int* plist, int npairs, int p, double* grads, double* mean) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < p; m += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < npairs; ++i) {
      const double v = all[(size_t)plist[i] * p + m];
      if (grads) grads[(size_t)i * p + m] = v;
      s += v;
    }
    if (mean) mean[m] = s / npairs;
  }
}

bl_status alloc_vec(bl_problem* P, void** ptr, size_t count) { return dalloc(ptr, count * P->esz); }

std::vector<int> host_mask(const bl_problem* P, const int32_t* pairs, int32_t npairs) {
  std::vector<int> m(P->K, 0);
  for (int i = 0; i < npairs; ++i) m[pairs[i]] = 1;
  return m;
}

bl_status ensure_history(bl_problem* P, int m) {
  if (m == P->MH && P->S) return BL_OK;
  destroy_lbfgs_graph(P);
  if (P->S) {
    cudaStreamSynchronize(P->stream);
    for (void* b : {(void*)P->S, (void*)P->Yh, (void*)P->lsy, (void*)P->lyy, (void*)P->lcs, (void*)P->lcy})
      cudaFree(b);
    P->S = P->Yh = nullptr;
    P->lsy = P->lyy = P->lcs = P->lcy = nullptr;
  }
  P->MH = m;
  const size_t rs = (size_t)m + 1;
  bl_status st = alloc_vec(P, &P->S, (size_t)P->n_tot * rs);
  if (st == BL_OK) st = alloc_vec(P, &P->Yh, (size_t)P->n_tot * rs);
  if (st == BL_OK) st = dalloc((void**)&P->lsy, (size_t)P->K * rs * rs * sizeof(double));
  if (st == BL_OK) st = dalloc((void**)&P->lyy, (size_t)P->K * rs * rs * sizeof(double));
  if (st == BL_OK) st = dalloc((void**)&P->lcs, (size_t)P->K * rs * sizeof(double));
  if (st == BL_OK) st = dalloc((void**)&P->lcy, (size_t)P->K * rs * sizeof(double));
  return st;
}

}  // namespace

namespace bl {

bl_status load_theta(bl_problem* P, const double* theta) {
  BL_CUDA_TRY(cudaMemcpyAsync(P->theta, theta, P->p * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
  k_theta<<<std::max(1, (P->p + 255) / 256), 256, 0, P->stream>>>(P->theta, P->N, P->F, P->reg.kind, P->taps_f,
                                                                  P->taps_d, P->ealpha);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

}  // namespace bl

extern "C" {

const char* bl_last_error(void) {
  static thread_local std::string copy;
  copy = error_copy();
  return copy.c_str();
}

int64_t bl_launch_count(const bl_problem* P) { return P ? P->launches : 0; }

int32_t bl_hvp_tma(const bl_problem* P) { return (P && P->tma) ? 1 : 0; }

int32_t bl_hvp_tile(const bl_problem* P, int32_t pair) { return P ? hvp_tma_tile(P, pair) : 0; }

bl_status bl_set_hvp_tile(bl_problem* P, int32_t pair, int32_t side) {
  if (!P) return fail(BL_EINVAL, "null problem");
  return hvp_tma_force_tile(P, pair, side);
}

int32_t bl_graph_used(const bl_problem* P) { return (P && P->graph_used) ? 1 : 0; }

static bl_status prof_collect(bl_problem* P) {
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  for (size_t i = 0; i < P->prof_used; ++i) {
    float ms = 0.f;
    BL_CUDA_TRY(cudaEventElapsedTime(&ms, P->prof_ev[i].a, P->prof_ev[i].b));
    P->prof_ms[P->prof_ev[i].cls] += ms;
    P->prof_n[P->prof_ev[i].cls] += 1;
  }
  P->prof_used = 0;
  return BL_OK;
}

bl_status bl_profile_enable(bl_problem* P, int32_t enable) {
  if (!P) return fail(BL_EINVAL, "null problem");
  bl_status st = prof_collect(P);
  if (st != BL_OK) return st;
  for (int c = 0; c < BL_KC_COUNT; ++c) {
    P->prof_ms[c] = 0.0;
    P->prof_n[c] = 0;
  }
  BL_CUDA_TRY(cudaMemsetAsync(P->d_pix, 0, BL_KC_COUNT * sizeof(unsigned long long), P->stream));
  BL_CUDA_TRY(cudaMemsetAsync(P->d_bytes, 0, BL_KC_COUNT * sizeof(unsigned long long), P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  P->prof = enable != 0;
  return BL_OK;
}

bl_status bl_profile_read(bl_problem* P, int32_t cls, double* total_ms, int64_t* launches, int64_t* pixels) {
  if (!P) return fail(BL_EINVAL, "null problem");
  if (cls < 0 || cls >= BL_KC_COUNT) return fail(BL_EINVAL, "unknown kernel class");
  bl_status st = prof_collect(P);
  if (st != BL_OK) return st;
  unsigned long long pix[BL_KC_COUNT];
  BL_CUDA_TRY(cudaMemcpy(pix, P->d_pix, sizeof(pix), cudaMemcpyDeviceToHost));
  if (total_ms) *total_ms = P->prof_ms[cls];
  if (launches) *launches = P->prof_n[cls];
  if (pixels) *pixels = (int64_t)pix[cls];
  return BL_OK;
}

bl_status bl_profile_read_bytes(bl_problem* P, int32_t cls, int64_t* bytes) {
  if (!P || !bytes) return fail(BL_EINVAL, "null argument");
  if (cls < 0 || cls >= BL_KC_COUNT) return fail(BL_EINVAL, "unknown kernel class");
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  unsigned long long b[BL_KC_COUNT];
  BL_CUDA_TRY(cudaMemcpy(b, P->d_bytes, sizeof(b), cudaMemcpyDeviceToHost));
  *bytes = (int64_t)b[cls];
  return BL_OK;
}

int32_t bl_num_params(const bl_problem* P) { return P ? P->p : 0; }

int64_t bl_num_pixels(const bl_problem* P, const int32_t* pairs, int32_t npairs) {
  if (!P || !pairs) return 0;
  int64_t n = 0;
  for (int i = 0; i < npairs; ++i)
    if (pairs[i] >= 0 && pairs[i] < P->K) n += P->ph[pairs[i]].n;
  return n;
}

int32_t bl_recycle_dim(const bl_problem* P, int32_t pair) {
  return (P && pair >= 0 && pair < P->K) ? P->s_k[pair] : 0;
}

int32_t bl_basis_size(const bl_problem* P, int32_t pair) {
  return (P && pair >= 0 && pair < P->K) ? P->kb_k[pair] : 0;
}

bl_status bl_set_stream(bl_problem* P, void* s) {
  if (!P) return fail(BL_EINVAL, "null problem");
  P->stream = (cudaStream_t)s;
  return BL_OK;
}

void bl_problem_destroy(bl_problem* P) {
  if (!P) return;
  cudaStreamSynchronize(P->stream);
  destroy_krylov_graph(P);
  if (P->cstream) cudaStreamDestroy(P->cstream);
  void* bufs[] = {P->d_pairs, P->d_tiles, P->d_jtiles, P->d_chunks, P->y, P->xstar, P->xhat, P->fu, P->fd, P->theta,
                  P->taps_f, P->taps_d, P->ealpha, P->r, P->pv, P->q, P->w, P->g, P->tmp, P->U, P->C, P->Z,
                  P->V, P->W, P->Wt, P->HWt, P->st, P->c, P->zc, P->e, P->ztr, P->ztc, P->d_s, P->d_hasz,
                  P->d_active, P->d_cols, P->d_flag, P->dG, P->dT, P->dJ, P->dY, P->dY2, P->dY3, P->d_tk,
                  P->lx, P->lg, P->ld, P->lxt, P->lgt, P->lq, P->S, P->Yh, P->lsy, P->lyy, P->lcs, P->lcy,
                  P->lst, P->tpart, P->cpart, P->vals,
                  P->d_pix, P->d_zero, P->d_loop, P->mv_prev, P->my1, P->my2, P->mrs, P->d_opmask, P->lz_alpha, P->lz_rho, P->lz_c,
                  P->d_tmaps, P->d_kerr, P->d_bytes, P->d_htiles};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (P->h_flag) cudaFreeHost(P->h_flag);
  for (auto& e : P->prof_ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  delete P;
}

bl_status bl_problem_create(const bl_pair_desc* pairs, int32_t K, const bl_reg_desc* reg, const void* y_packed,
                            const void* xstar_packed, void* cuda_stream, bl_problem** out) {
  if (!out) return fail(BL_EINVAL, "null output handle");
  *out = nullptr;
  if (!pairs || !reg || !y_packed || !xstar_packed) return fail(BL_EINVAL, "null argument");
  if (K < 1) return fail(BL_EINVAL, "K must be >= 1");
  if (reg->kind != BL_REG_TV && reg->kind != BL_REG_FOE) return fail(BL_EINVAL, "unknown regulariser kind");
  if (reg->precision != BL_FP32 && reg->precision != BL_FP64) return fail(BL_EINVAL, "unknown precision");
  if (reg->kind == BL_REG_FOE) {
    if (reg->n_filters < 1 || reg->n_filters > kMaxFilters) return fail(BL_EINVAL, "n_filters must be in 1..64");
    if (reg->filter_size < 1 || reg->filter_size > BL_MAX_FILTER_SIZE || reg->filter_size % 2 == 0)
      return fail(BL_EINVAL, "filter_size must be odd and <= 7");
    if (reg->phi < BL_PHI_CHARBONNIER || reg->phi > BL_PHI_LOG1P) return fail(BL_EINVAL, "unknown phi");
  }
  if (!(reg->phi_eps > 0.0) && !(reg->kind == BL_REG_FOE && reg->phi != BL_PHI_CHARBONNIER))
    return fail(BL_EINVAL, "phi_eps must be > 0");
  if (!(reg->l2_eps >= 0.0)) return fail(BL_EINVAL, "l2_eps must be >= 0");
  if (reg->max_recycle < 0 || reg->max_recycle > 64) return fail(BL_EINVAL, "max_recycle must be in 0..64");
  if (reg->max_basis < 0 || reg->max_recycle + reg->max_basis > kMaxTM)
    return fail(BL_EINVAL, "max_recycle + max_basis must be <= 96");
  for (int k = 0; k < K; ++k) {
    if (pairs[k].height < 1 || pairs[k].width < 1) return fail(BL_EINVAL, "image sizes must be >= 1");
    if (pairs[k].mask) continue;   // inpainting pair: the blur fields are ignored
    if (pairs[k].blur_radius < 0 || pairs[k].blur_radius > BL_MAX_BLUR_RADIUS)
      return fail(BL_EINVAL, "blur_radius must be in 0..4");
    if (!(pairs[k].blur_sigma > 0.0)) return fail(BL_EINVAL, "blur_sigma must be > 0");
  }
  bl_problem* P = new bl_problem();
  P->K = K;
  P->reg = *reg;
  P->prec = reg->precision;
  P->esz = P->prec == BL_FP32 ? 4 : 8;
  P->stream = (cudaStream_t)cuda_stream;
  if (reg->kind == BL_REG_FOE) {
    P->N = reg->n_filters;
    P->F = reg->filter_size;
    P->p = P->N * (P->F * P->F + 1);
  } else {
    P->N = 0;
    P->F = 1;
    P->p = 1;
  }
  P->rf = P->F / 2;
  P->SMAX = std::max(1, reg->max_recycle);
  P->KMAX = reg->max_basis;
  P->TM = std::max(1, reg->max_recycle + reg->max_basis);

  // pair geometry, tiles and chunks
  const int TILE = tile_out(P->F);
  const int TILEJ = P->prec == BL_FP32 ? jw_tile_out<float>(P->F) : jw_tile_out<double>(P->F);
  std::vector<PairDev> pd(K);
  std::vector<TileDev> tiles, jtiles;
  std::vector<ChunkDev> chunks;
  long long off = 0;
  for (int k = 0; k < K; ++k) {
    PairHost ph{};
    ph.h = pairs[k].height;
    ph.w = pairs[k].width;
    ph.n = (long long)ph.h * ph.w;
    ph.off = off;
    ph.masked = pairs[k].mask != nullptr;
    ph.rb = ph.masked ? 0 : pairs[k].blur_radius;
    ph.sigma = ph.masked ? 1.0 : pairs[k].blur_sigma;
    ph.tbeg = (int)tiles.size();
    for (int ty = 0; ty < ph.h; ty += TILE)
      for (int tx = 0; tx < ph.w; tx += TILE) tiles.push_back(TileDev{k, ty, tx});
    ph.tend = (int)tiles.size();
    ph.jtbeg = (int)jtiles.size();
    for (int ty = 0; ty < ph.h; ty += TILEJ)
      for (int tx = 0; tx < ph.w; tx += TILEJ) jtiles.push_back(TileDev{k, ty, tx});
    ph.jtend = (int)jtiles.size();
    ph.cbeg = (int)chunks.size();
    for (long long s = 0; s < ph.n; s += kChunk)
      chunks.push_back(ChunkDev{k, s, (int)std::min<long long>(kChunk, ph.n - s)});
    ph.cend = (int)chunks.size();
    P->ph.push_back(ph);
    PairDev& d = pd[k];
    memset(&d, 0, sizeof(d));
    d.h = ph.h;
    d.w = ph.w;
    d.n = ph.n;
    d.off = ph.off;
    d.rb = ph.rb;
    d.tbeg = ph.tbeg;
    d.tend = ph.tend;
    d.jtbeg = ph.jtbeg;
    d.jtend = ph.jtend;
    d.cbeg = ph.cbeg;
    d.cend = ph.cend;
    // 1-D normalised Gaussian; the 2-D kernel of Section 5.2 is its outer product
    double gs = 0.0;
    for (int a = -ph.rb; a <= ph.rb; ++a) gs += std::exp(-(double)a * a / (2.0 * ph.sigma * ph.sigma));
    for (int a = -ph.rb; a <= ph.rb; ++a) {
      const double gv = std::exp(-(double)a * a / (2.0 * ph.sigma * ph.sigma)) / gs;
      d.gd[a + ph.rb] = gv;
      d.gf[a + ph.rb] = (float)gv;
    }
    off += ph.n;
  }
  P->n_tot = off;
  P->n_tiles = (int)tiles.size();
  P->n_jtiles = (int)jtiles.size();
  P->n_chunks = (int)chunks.size();
  P->vec4 = true;
  for (const auto& ph : P->ph) P->vec4 = P->vec4 && (ph.n % 4 == 0);
  P->s_k.assign(K, 0);
  P->kb_k.assign(K, 0);
  P->hz_k.assign(K, 0);
  P->head_k.assign(K, 0);
  P->lz_k.assign(K, 0);
  P->lz_u.assign(K, 0);

  bl_status st = BL_OK;
#define BL_ALLOC(expr)              \
  do {                              \
    st = (expr);                    \
    if (st != BL_OK) {              \
      bl_problem_destroy(P);        \
      return st;                    \
    }                               \
  } while (0)
  const size_t n = (size_t)P->n_tot;
  BL_ALLOC(dalloc((void**)&P->d_pairs, K * sizeof(PairDev)));
  BL_ALLOC(dalloc((void**)&P->d_tiles, tiles.size() * sizeof(TileDev)));
  BL_ALLOC(dalloc((void**)&P->d_jtiles, jtiles.size() * sizeof(TileDev)));
  BL_ALLOC(dalloc((void**)&P->d_chunks, chunks.size() * sizeof(ChunkDev)));
  for (void** b : {&P->y, &P->xstar, &P->xhat, &P->r, &P->pv, &P->q, &P->w, &P->g, &P->lx, &P->lg, &P->ld,
                   &P->lxt, &P->lgt})
    BL_ALLOC(alloc_vec(P, b, n));
  // inpainting masks: one byte per pixel of every pair (0 / 1), pointed to by the pair descriptors
  std::vector<unsigned char> hmask;
  for (int k = 0; k < K; ++k)
    if (pairs[k].mask) {
      if (hmask.empty()) {
        BL_ALLOC(dalloc((void**)&P->d_opmask, n));
        hmask.assign(n, 0);
      }
      const PairHost& ph = P->ph[k];
      for (long long i = 0; i < ph.n; ++i) hmask[ph.off + i] = pairs[k].mask[i] ? 1 : 0;
      pd[k].opm = P->d_opmask + ph.off;
    }
  BL_ALLOC(alloc_vec(P, &P->tmp, 3 * n));
  if (P->N > 0) {
    BL_ALLOC(alloc_vec(P, &P->fu, (size_t)P->N * n));
    BL_ALLOC(alloc_vec(P, &P->fd, (size_t)P->N * n));
  }
  BL_ALLOC(alloc_vec(P, &P->U, n * P->SMAX));
  BL_ALLOC(alloc_vec(P, &P->C, n * P->SMAX));
  BL_ALLOC(alloc_vec(P, &P->Z, n * P->SMAX));
  BL_ALLOC(alloc_vec(P, &P->V, n * std::max(1, P->KMAX)));
  BL_ALLOC(alloc_vec(P, &P->W, n * P->TM));
  BL_ALLOC(alloc_vec(P, &P->Wt, n * P->TM));
  BL_ALLOC(alloc_vec(P, &P->HWt, n * P->TM));
  BL_ALLOC(dalloc((void**)&P->theta, P->p * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->taps_f, std::max(1, P->N * P->F * P->F) * sizeof(float)));
  BL_ALLOC(dalloc((void**)&P->taps_d, std::max(1, P->N * P->F * P->F) * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->ealpha, std::max(1, P->N) * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->st, K * sizeof(SolveState)));
  BL_ALLOC(dalloc((void**)&P->lst, K * sizeof(LbfgsState)));
  for (double** b : {&P->c, &P->zc, &P->e, &P->ztr})
    BL_ALLOC(dalloc((void**)b, (size_t)K * P->SMAX * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->ztc, (size_t)K * P->SMAX * P->SMAX * sizeof(double)));
  {
    const size_t kk = (size_t)K * std::max(1, P->KMAX);
    BL_ALLOC(dalloc((void**)&P->lz_alpha, kk * sizeof(double)));
    BL_ALLOC(dalloc((void**)&P->lz_rho, kk * sizeof(double)));
    BL_ALLOC(dalloc((void**)&P->lz_c, kk * P->SMAX * sizeof(double)));
  }
  BL_ALLOC(dalloc((void**)&P->d_s, K * sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_hasz, K * sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_active, 3 * K * sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_cols, 2 * K * sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_tk, 3 * K * sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_flag, sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_zero, K * sizeof(int)));
  BL_ALLOC(dalloc((void**)&P->d_loop, 2 * sizeof(int)));
  const size_t tm2 = (size_t)K * P->TM * P->TM;
  BL_ALLOC(dalloc((void**)&P->dG, tm2 * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->dT, 2 * tm2 * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->dJ, (size_t)K * P->TM * P->p * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->dY, tm2 * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->dY2, tm2 * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->dY3, std::max(4 * tm2, (size_t)K * kMaxHistory) * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->vals, 8 * (size_t)K * sizeof(double)));
  BL_ALLOC(dalloc((void**)&P->d_pix, BL_KC_COUNT * sizeof(unsigned long long)));
  BL_ALLOC(dalloc((void**)&P->d_bytes, BL_KC_COUNT * sizeof(unsigned long long)));
  BL_ALLOC(dalloc((void**)&P->d_kerr, sizeof(int)));
  if (cudaMallocHost((void**)&P->h_flag, sizeof(int)) != cudaSuccess) {
    bl_problem_destroy(P);
    return fail(BL_ENOMEM, "cudaMallocHost failed");
  }
#undef BL_ALLOC
  auto cpy = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    return cudaMemcpyAsync(dst, src, bytes, kind, P->stream);
  };
  cudaError_t e = cudaSuccess;
  P->pd_host = pd;
  e = e == cudaSuccess ? cpy(P->d_pairs, pd.data(), K * sizeof(PairDev), cudaMemcpyHostToDevice) : e;
  if (!hmask.empty()) e = e == cudaSuccess ? cpy(P->d_opmask, hmask.data(), n, cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cpy(P->d_tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cpy(P->d_jtiles, jtiles.data(), jtiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cpy(P->d_chunks, chunks.data(), chunks.size() * sizeof(ChunkDev), cudaMemcpyHostToDevice) : e;
  e = e == cudaSuccess ? cpy(P->y, y_packed, n * P->esz, cudaMemcpyDeviceToDevice) : e;
  e = e == cudaSuccess ? cpy(P->xstar, xstar_packed, n * P->esz, cudaMemcpyDeviceToDevice) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(P->d_s, 0, K * sizeof(int), P->stream) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(P->d_hasz, 0, K * sizeof(int), P->stream) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(P->d_zero, 0, K * sizeof(int), P->stream) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(P->ztc, 0, (size_t)K * P->SMAX * P->SMAX * sizeof(double), P->stream) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(P->xhat, 0, n * P->esz, P->stream) : e;
  e = e == cudaSuccess ? cudaMemsetAsync(P->d_kerr, 0, sizeof(int), P->stream) : e;
  e = e == cudaSuccess ? cudaStreamSynchronize(P->stream) : e;
  if (e != cudaSuccess) {
    bl_problem_destroy(P);
    return fail(BL_ECUDA, std::string("problem set-up: ") + cudaGetErrorString(e));
  }
  if ((st = prepare_kernels(P)) != BL_OK || (st = hvp_tma_setup(P)) != BL_OK || (st = prepare_hvp_tma(P)) != BL_OK) {
    bl_problem_destroy(P);
    return st;
  }
  *out = P;
  return BL_OK;
}

bl_status bl_set_data(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* y, const void* xstar) {
  if (!P || !y || !xstar) return fail(BL_EINVAL, "null argument");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if ((st = gather_packed(P, pairs, npairs, y, P->y)) != BL_OK) return st;
  return gather_packed(P, pairs, npairs, xstar, P->xstar);
}

bl_status bl_forward(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* x, void* out) {
  if (!P || !x || !out) return fail(BL_EINVAL, "null argument");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if ((st = gather_packed(P, pairs, npairs, x, P->r)) != BL_OK) return st;
  if ((st = launch_forward(P, P->r, P->q, P->d_active)) != BL_OK) return st;
  return scatter_packed(P, pairs, npairs, P->q, out);
}

bl_status bl_set_point(bl_problem* P, const int32_t* pairs, int32_t npairs, const double* theta, const void* xhat) {
  if (!P || !theta || !xhat) return fail(BL_EINVAL, "null argument");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if ((st = load_theta(P, theta)) != BL_OK) return st;
  if ((st = gather_packed(P, pairs, npairs, xhat, P->xhat)) != BL_OK) return st;
  if ((st = launch_fields(P, P->d_active)) != BL_OK) return st;
  P->point_set = true;
  return BL_OK;
}

bl_status bl_gradient(bl_problem* P, const int32_t* pairs, int32_t npairs, const double* theta, const void* x,
                      void* grad, double* values) {
  if (!P || !theta || !x || !grad) return fail(BL_EINVAL, "null argument");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if ((st = load_theta(P, theta)) != BL_OK) return st;
  P->point_set = false;   // the current theta changed; the stored fields no longer match
  if ((st = gather_packed(P, pairs, npairs, x, P->lx)) != BL_OK) return st;
  if ((st = launch_grad(P, P->lx, P->lg, P->d_active, P->vals)) != BL_OK) return st;
  if ((st = scatter_packed(P, pairs, npairs, P->lg, grad)) != BL_OK) return st;
  if (values) {
    std::vector<double> hv(3 * P->K);
    BL_CUDA_TRY(cudaMemcpyAsync(hv.data(), P->vals, 3 * P->K * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    std::vector<double> out(npairs);
    for (int i = 0; i < npairs; ++i) {
      const int k = pairs[i];
      out[i] = hv[3 * k] + hv[3 * k + 1] + 0.5 * P->reg.l2_eps * hv[3 * k + 2];
    }
    BL_CUDA_TRY(cudaMemcpyAsync(values, out.data(), npairs * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  }
  return BL_OK;
}

bl_status bl_lower_solve(bl_problem* P, const int32_t* pairs, int32_t npairs, const double* theta,
                         const bl_lbfgs_opts* o, void* xhat, bl_solve_info* info) {
  if (!P || !theta || !o || !xhat) return fail(BL_EINVAL, "null argument");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if (o->history < 1 || o->history > kMaxHistory) return fail(BL_EINVAL, "history must be in 1..16");
  if (o->max_iters < 0 || !(o->gtol >= 0.0) || !(o->armijo_slack >= 0.0))
    return fail(BL_EINVAL, "invalid L-BFGS options");
  if ((st = ensure_history(P, o->history)) != BL_OK) return st;
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if ((st = load_theta(P, theta)) != BL_OK) return st;
  if ((st = gather_packed(P, pairs, npairs, xhat, P->lx)) != BL_OK) return st;
  std::vector<int> mh = host_mask(P, pairs, npairs);
  std::vector<bl_solve_info> inf;
  if ((st = run_lower_solve(P, mh, o, inf)) != BL_OK) return st;
  // the solution becomes the current point
  for (int i = 0; i < npairs; ++i) {
    const PairHost& ph = P->ph[pairs[i]];
    BL_CUDA_TRY(cudaMemcpyAsync((char*)P->xhat + ph.off * P->esz, (const char*)P->lx + ph.off * P->esz, ph.n * P->esz,
                                cudaMemcpyDeviceToDevice, P->stream));
  }
  if ((st = scatter_packed(P, pairs, npairs, P->lx, xhat)) != BL_OK) return st;
  if ((st = launch_fields(P, P->d_active)) != BL_OK) return st;
  P->point_set = true;
  bl_status ret = BL_OK;
  for (int i = 0; i < npairs; ++i) {
    const bl_solve_info& s = inf[pairs[i]];
    if (info) info[i] = s;
    if (s.status == BL_EBREAKDOWN) ret = BL_EBREAKDOWN;
    else if (s.status == BL_ENOCONV && ret == BL_OK) ret = BL_ENOCONV;
  }
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  return ret;
}

bl_status bl_hvp(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* v, void* out) {
  if (!P || !v || !out) return fail(BL_EINVAL, "null argument");
  if (!P->point_set) return fail(BL_ESTATE, "no point set: call bl_set_point or bl_lower_solve first");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if ((st = gather_packed(P, pairs, npairs, v, P->r)) != BL_OK) return st;
  if ((st = launch_hvp(P, P->r, P->q, 0, 0, P->d_active, nullptr, nullptr)) != BL_OK) return st;
  return scatter_packed(P, pairs, npairs, P->q, out);
}

bl_status bl_ritz_update(bl_problem* P, const int32_t* pairs, int32_t npairs, const bl_recycle_opts* o) {
  if (!P || !o) return fail(BL_EINVAL, "null argument");
  if (!P->point_set) return fail(BL_ESTATE, "no point set: call bl_set_point or bl_lower_solve first");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if (o->kind < BL_RECYCLE_RITZ || o->kind > BL_RECYCLE_RGSV || o->size < BL_SIZE_SMALL ||
      o->size > BL_SIZE_MIXED || o->side < BL_SIDE_RIGHT || o->side > BL_SIDE_MIXED)
    return fail(BL_EINVAL, "unknown recycle option");
  if (o->s < 1 || o->s > P->reg.max_recycle) return fail(BL_EINVAL, "s must be in 1..max_recycle");
  if (o->kind == BL_RECYCLE_RGSV && o->s > P->p) return fail(BL_EINVAL, "RGSV needs s <= p");
  if (o->variant != BL_REFRESH_OUTER && o->variant != BL_REFRESH_INNER) return fail(BL_EINVAL, "unknown refresh variant");
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  return run_ritz_update(P, host_mask(P, pairs, npairs), o);
}

bl_status bl_hessian_solve(bl_problem* P, const int32_t* pairs, int32_t npairs, const bl_krylov_opts* o,
                           const void* g, void* w, const double* nsc_scale, bl_solve_info* info) {
  if (!P || !o || !w) return fail(BL_EINVAL, "null argument");
  if (!P->point_set) return fail(BL_ESTATE, "no point set: call bl_set_point or bl_lower_solve first");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if (o->method < BL_SOLVE_CG || o->method > BL_SOLVE_RMINRES) return fail(BL_EINVAL, "unknown solve method");
  if (o->stop != BL_STOP_RESID && o->stop != BL_STOP_NSC) return fail(BL_EINVAL, "unknown stop rule");
  if (o->maxit < 0 || !(o->tol >= 0.0)) return fail(BL_EINVAL, "invalid Krylov options");
  if (o->store_basis < BL_STORE_NONE || o->store_basis > BL_STORE_LANCZOS)
    return fail(BL_EINVAL, "unknown store mode");
  if (o->store_basis == BL_STORE_LANCZOS && (o->method == BL_SOLVE_MINRES || o->method == BL_SOLVE_RMINRES))
    return fail(BL_EINVAL, "BL_STORE_LANCZOS records CG steps; MINRES keeps BL_STORE_RECENT");
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if (o->warm_start && (st = gather_packed(P, pairs, npairs, w, P->w)) != BL_OK) return st;
  if (g) {
    if ((st = gather_packed(P, pairs, npairs, g, P->g)) != BL_OK) return st;
  } else {
    if (P->prec == BL_FP32)
      k_sub<float><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const float*)P->xhat,
                                                                  (const float*)P->xstar, (float*)P->g, P->d_active);
    else
      k_sub<double><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const double*)P->xhat,
                                                                   (const double*)P->xstar, (double*)P->g, P->d_active);
    BL_LAUNCH_CHECK(P);
  }
  std::vector<double> scale(P->K, 1.0);
  if (nsc_scale)
    for (int i = 0; i < npairs; ++i) scale[pairs[i]] = nsc_scale[i];
  std::vector<int> mh = host_mask(P, pairs, npairs);
  std::vector<bl_solve_info> inf;
  if ((st = run_hessian_solve(P, mh.data(), o, P->g, nsc_scale ? scale.data() : nullptr, inf)) != BL_OK) return st;
  if ((st = scatter_packed(P, pairs, npairs, P->w, w)) != BL_OK) return st;
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  bl_status ret = BL_OK;
  for (int i = 0; i < npairs; ++i) {
    const bl_solve_info& s = inf[pairs[i]];
    if (info) info[i] = s;
    if (s.status == BL_EBREAKDOWN) ret = BL_EBREAKDOWN;
    else if (s.status == BL_ENOCONV && ret == BL_OK) ret = BL_ENOCONV;
  }
  return ret;
}

bl_status bl_hypergrad(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* w, double* grads,
                       double* mean_grad, double* loss) {
  if (!P || !w) return fail(BL_EINVAL, "null argument");
  if (!P->point_set) return fail(BL_ESTATE, "no point set: call bl_set_point or bl_lower_solve first");
  bl_status st = check_pairs(P, pairs, npairs);
  if (st != BL_OK) return st;
  if ((st = set_active_pairs(P, pairs, npairs)) != BL_OK) return st;
  if ((st = gather_packed(P, pairs, npairs, w, P->r)) != BL_OK) return st;
  double* all = P->dJ;    // K x p per-pair results (dJ holds K x TM x p doubles)
  if ((st = launch_jw(P, P->r, 0, 1, P->d_active, all)) != BL_OK) return st;
  if (grads || mean_grad) {
    int* dlist = P->d_tk;   // 2K ints of scratch
    BL_CUDA_TRY(cudaMemcpyAsync(dlist, pairs, npairs * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    k_pick_rows<<<(P->p + 127) / 128, 128, 0, P->stream>>>(all, dlist, npairs, P->p, grads, mean_grad);
    BL_LAUNCH_CHECK(P);
  }
  if (loss) {
    if (P->prec == BL_FP32)
      k_sub<float><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const float*)P->xhat,
                                                                  (const float*)P->xstar, (float*)P->q, P->d_active);
    else
      k_sub<double><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const double*)P->xhat,
                                                                   (const double*)P->xstar, (double*)P->q, P->d_active);
    BL_LAUNCH_CHECK(P);
    if ((st = batched_dot(P, P->q, P->q, P->d_active, P->vals)) != BL_OK) return st;
    std::vector<double> hv(P->K);
    BL_CUDA_TRY(cudaMemcpyAsync(hv.data(), P->vals, P->K * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
    double s = 0.0;
    for (int i = 0; i < npairs; ++i) s += 0.5 * hv[pairs[i]];
    *loss = s / npairs;
  }
  return BL_OK;
}

// ---- recycle checkpoint: header + U, C, Z (s columns each, problem precision) + Z^T C (FP64) ----
struct RecycleHeader {
  uint32_t magic, version;
  int32_t prec, height, width, s, hasz, smax;
};
static const uint32_t kMagic = 0x424c5243u;   // "BLRC"

// Stored Krylov basis of a pair (what the next bl_ritz_update reads): its columns in storage order and,
// for a Lanczos record, the CG coefficients of the steps it holds.
struct BasisHeader {
  int32_t kb, lz, lzu, head, ncols, kmax;
};

static size_t basis_bytes(const bl_problem* P, int pair) {
  const int kb = P->kb_k[pair];
  const int ncols = P->lz_k[pair] ? std::min(kb + 1, P->KMAX) : kb;
  size_t b = sizeof(BasisHeader) + (size_t)ncols * P->ph[pair].n * P->esz;
  if (P->lz_k[pair]) b += (size_t)P->KMAX * (2 + P->SMAX) * sizeof(double);
  return b;
}

bl_status bl_recycle_export(bl_problem* P, int32_t pair, void* buf, size_t* bytes) {
  if (!P || !bytes) return fail(BL_EINVAL, "null argument");
  if (pair < 0 || pair >= P->K) return fail(BL_EINVAL, "pair index out of range");
  const PairHost& ph = P->ph[pair];
  const int s = P->s_k[pair];
  const size_t vec = (size_t)s * ph.n * P->esz;
  const size_t need = sizeof(RecycleHeader) + 3 * vec + (size_t)s * s * sizeof(double) + basis_bytes(P, pair);
  if (!buf) {
    *bytes = need;
    return BL_OK;
  }
  if (*bytes < need) return fail(BL_EINVAL, "checkpoint buffer too small");
  RecycleHeader hd{kMagic, 2, P->prec, ph.h, ph.w, s, P->hz_k[pair], P->SMAX};
  char* o = (char*)buf;
  memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  const size_t base = (size_t)ph.off * P->SMAX * P->esz;
  BL_CUDA_TRY(cudaMemcpyAsync(o, (const char*)P->U + base, vec, cudaMemcpyDeviceToHost, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync(o + vec, (const char*)P->C + base, vec, cudaMemcpyDeviceToHost, P->stream));
  if (P->hz_k[pair])
    BL_CUDA_TRY(cudaMemcpyAsync(o + 2 * vec, (const char*)P->Z + base, vec, cudaMemcpyDeviceToHost, P->stream));
  else
    memset(o + 2 * vec, 0, vec);   // no Ritz-GSV operator for this pair: Z is written as zeros
  std::vector<double> ztc((size_t)P->SMAX * P->SMAX);
  BL_CUDA_TRY(cudaMemcpyAsync(ztc.data(), P->ztc + (size_t)pair * P->SMAX * P->SMAX, ztc.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, P->stream));
  // the stored basis (and Lanczos record) that the next refresh reads
  char* ob = o + 3 * vec + (size_t)s * s * sizeof(double);
  const int kb = P->kb_k[pair];
  BasisHeader bh{kb, P->lz_k[pair], P->lz_u[pair], P->head_k[pair], P->lz_k[pair] ? std::min(kb + 1, P->KMAX) : kb,
                 P->KMAX};
  memcpy(ob, &bh, sizeof(bh));
  char* ov = ob + sizeof(bh);
  const size_t bvec = (size_t)bh.ncols * ph.n * P->esz;
  if (bvec)
    BL_CUDA_TRY(cudaMemcpyAsync(ov, (const char*)P->V + (size_t)ph.off * P->KMAX * P->esz, bvec,
                                cudaMemcpyDeviceToHost, P->stream));
  if (bh.lz) {
    char* oc = ov + bvec;
    const size_t km = (size_t)P->KMAX;
    BL_CUDA_TRY(cudaMemcpyAsync(oc, P->lz_alpha + pair * km, km * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    BL_CUDA_TRY(cudaMemcpyAsync(oc + km * sizeof(double), P->lz_rho + pair * km, km * sizeof(double),
                                cudaMemcpyDeviceToHost, P->stream));
    BL_CUDA_TRY(cudaMemcpyAsync(oc + 2 * km * sizeof(double), P->lz_c + pair * km * P->SMAX,
                                km * P->SMAX * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  }
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  double* zo = (double*)(o + 3 * vec);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) zo[i * s + j] = P->hz_k[pair] ? ztc[(size_t)i * P->SMAX + j] : 0.0;
  *bytes = need;
  return BL_OK;
}

bl_status bl_recycle_import(bl_problem* P, int32_t pair, const void* buf, size_t bytes) {
  if (!P || !buf) return fail(BL_EINVAL, "null argument");
  if (pair < 0 || pair >= P->K) return fail(BL_EINVAL, "pair index out of range");
  if (bytes < sizeof(RecycleHeader)) return fail(BL_EINVAL, "checkpoint truncated");
  RecycleHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  const PairHost& ph = P->ph[pair];
  if (hd.magic != kMagic || (hd.version != 1 && hd.version != 2)) return fail(BL_EINVAL, "not a recycle checkpoint");
  if (hd.prec != P->prec || hd.height != ph.h || hd.width != ph.w)
    return fail(BL_EINVAL, "checkpoint does not match this pair's size or precision");
  if (hd.s < 0 || hd.s > P->reg.max_recycle || hd.hasz < 0 || hd.hasz > 1)
    return fail(BL_EINVAL, "checkpoint recycle dimension out of range");
  const int s = hd.s;
  const size_t vec = (size_t)s * ph.n * P->esz;
  const size_t need1 = sizeof(RecycleHeader) + 3 * vec + (size_t)s * s * sizeof(double);
  if (bytes < need1) return fail(BL_EINVAL, "checkpoint truncated");
  const char* in = (const char*)buf + sizeof(hd);
  BasisHeader bh{0, 0, 0, 0, 0, P->KMAX};
  const char* ib = in + 3 * vec + (size_t)s * s * sizeof(double);
  if (hd.version == 2) {
    if (bytes < need1 + sizeof(BasisHeader)) return fail(BL_EINVAL, "checkpoint truncated");
    memcpy(&bh, ib, sizeof(bh));
    if (bh.kmax != P->KMAX || hd.smax != P->SMAX)
      return fail(BL_EINVAL, "checkpoint basis needs the same max_basis and max_recycle");
    if (bh.kb < 0 || bh.ncols < 0 || bh.ncols > P->KMAX || bh.lz < 0 || bh.lz > 1 ||
        bh.ncols != (bh.lz ? std::min(bh.kb + 1, P->KMAX) : bh.kb))
      return fail(BL_EINVAL, "checkpoint basis out of range");
    size_t nb = sizeof(BasisHeader) + (size_t)bh.ncols * ph.n * P->esz;
    if (bh.lz) nb += (size_t)P->KMAX * (2 + P->SMAX) * sizeof(double);
    if (bytes < need1 + nb) return fail(BL_EINVAL, "checkpoint truncated");
  }
  const size_t base = (size_t)ph.off * P->SMAX * P->esz;
  BL_CUDA_TRY(cudaMemcpyAsync((char*)P->U + base, in, vec, cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync((char*)P->C + base, in + vec, vec, cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync((char*)P->Z + base, in + 2 * vec, vec, cudaMemcpyHostToDevice, P->stream));
  std::vector<double> ztc((size_t)P->SMAX * P->SMAX, 0.0);
  const double* zi = (const double*)(in + 3 * vec);
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) {
      double v;
      memcpy(&v, zi + i * s + j, sizeof(double));
      ztc[(size_t)i * P->SMAX + j] = v;
    }
  BL_CUDA_TRY(cudaMemcpyAsync(P->ztc + (size_t)pair * P->SMAX * P->SMAX, ztc.data(), ztc.size() * sizeof(double),
                              cudaMemcpyHostToDevice, P->stream));
  if (bh.ncols) {
    const char* iv = ib + sizeof(BasisHeader);
    const size_t bvec = (size_t)bh.ncols * ph.n * P->esz;
    BL_CUDA_TRY(cudaMemcpyAsync((char*)P->V + (size_t)ph.off * P->KMAX * P->esz, iv, bvec, cudaMemcpyHostToDevice,
                                P->stream));
    if (bh.lz) {
      const char* ic = iv + bvec;
      const size_t km = (size_t)P->KMAX;
      BL_CUDA_TRY(cudaMemcpyAsync(P->lz_alpha + pair * km, ic, km * sizeof(double), cudaMemcpyHostToDevice, P->stream));
      BL_CUDA_TRY(cudaMemcpyAsync(P->lz_rho + pair * km, ic + km * sizeof(double), km * sizeof(double),
                                  cudaMemcpyHostToDevice, P->stream));
      BL_CUDA_TRY(cudaMemcpyAsync(P->lz_c + pair * km * P->SMAX, ic + 2 * km * sizeof(double),
                                  km * P->SMAX * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    }
  }
  P->s_k[pair] = s;
  P->hz_k[pair] = hd.hasz;
  P->kb_k[pair] = bh.kb;
  P->lz_k[pair] = bh.lz;
  P->lz_u[pair] = bh.lzu;
  P->head_k[pair] = bh.head;
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_s, P->s_k.data(), P->K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_hasz, P->hz_k.data(), P->K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  return BL_OK;
}

}  // extern "C"
