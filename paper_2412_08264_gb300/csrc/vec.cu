// Batched-vector helpers: partial-sum reductions, dot products, buffer management.
#include <cstring>

#include "common.cuh"
#include "device.cuh"

namespace bl {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

std::string error_copy() { return g_err; }

bl_status fail(bl_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

ProfScope::ProfScope(bl_problem* p, int cls) : P(p), slot(-1) {
  if (!P->prof) return;
  if (P->prof_used == P->prof_ev.size()) {
    ProfEvent e{};
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return;
    P->prof_ev.push_back(e);
  }
  slot = (int)P->prof_used++;
  P->prof_ev[slot].cls = cls;
  cudaEventRecord(P->prof_ev[slot].a, P->stream);
}

ProfScope::~ProfScope() {
  if (slot >= 0) cudaEventRecord(P->prof_ev[slot].b, P->stream);
}

unsigned long long* pix_counter(bl_problem* P, int cls) { return P->prof ? P->d_pix + cls : nullptr; }
unsigned long long* bytes_counter(bl_problem* P, int cls) { return P->prof ? P->d_bytes + cls : nullptr; }

bl_status check_kernel_error(bl_problem* P) {
  int code = 0;
  BL_CUDA_TRY(cudaMemcpyAsync(&code, P->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  BL_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (code == 0) return BL_OK;
  BL_CUDA_TRY(cudaMemsetAsync(P->d_kerr, 0, sizeof(int), P->stream));
  return fail(BL_ECUDA, "a Hessian-action kernel gave up waiting for its tile copies (code " + std::to_string(code) +
                            "); its results are invalid");
}

bl_status dalloc(void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(BL_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return BL_OK;
}

bl_status ensure_tpart(bl_problem* P, size_t doubles) {
  if (doubles <= P->tpart_cap) return BL_OK;
  destroy_krylov_graph(P);
  if (P->tpart) {
    cudaStreamSynchronize(P->stream);
    cudaFree(P->tpart);
    P->tpart = nullptr;
  }
  bl_status st = dalloc((void**)&P->tpart, doubles * sizeof(double));
  P->tpart_cap = st == BL_OK ? doubles : 0;
  return st;
}

bl_status ensure_cpart(bl_problem* P, size_t doubles) {
  if (doubles <= P->cpart_cap) return BL_OK;
  destroy_krylov_graph(P);
  if (P->cpart) {
    cudaStreamSynchronize(P->stream);
    cudaFree(P->cpart);
    P->cpart = nullptr;
  }
  bl_status st = dalloc((void**)&P->cpart, doubles * sizeof(double));
  P->cpart_cap = st == BL_OK ? doubles : 0;
  return st;
}

bl_status check_pairs(const bl_problem* P, const int32_t* pairs, int32_t npairs) {
  if (!pairs || npairs < 1 || npairs > P->K) return fail(BL_EINVAL, "pair list must hold 1..K indices");
  std::vector<char> seen(P->K, 0);
  for (int i = 0; i < npairs; ++i) {
    if (pairs[i] < 0 || pairs[i] >= P->K) return fail(BL_EINVAL, "pair index out of range");
    if (seen[pairs[i]]) return fail(BL_EINVAL, "pair listed twice");
    seen[pairs[i]] = 1;
  }
  return BL_OK;
}

bl_status set_active_pairs(bl_problem* P, const int32_t* pairs, int32_t npairs) {
  std::vector<int> m(P->K, 0);
  for (int i = 0; i < npairs; ++i) m[pairs[i]] = 1;
  BL_CUDA_TRY(cudaMemcpyAsync(P->d_active, m.data(), P->K * sizeof(int), cudaMemcpyHostToDevice, P->stream));
  return BL_OK;
}

bl_status gather_packed(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* packed,
                        void* batched) {
  size_t pos = 0;
  for (int i = 0; i < npairs; ++i) {
    const PairHost& ph = P->ph[pairs[i]];
    BL_CUDA_TRY(cudaMemcpyAsync((char*)batched + ph.off * P->esz, (const char*)packed + pos * P->esz,
                                ph.n * P->esz, cudaMemcpyDeviceToDevice, P->stream));
    pos += ph.n;
  }
  return BL_OK;
}

bl_status scatter_packed(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* batched,
                         void* packed) {
  size_t pos = 0;
  for (int i = 0; i < npairs; ++i) {
    const PairHost& ph = P->ph[pairs[i]];
    BL_CUDA_TRY(cudaMemcpyAsync((char*)packed + pos * P->esz, (const char*)batched + ph.off * P->esz,
                                ph.n * P->esz, cudaMemcpyDeviceToDevice, P->stream));
    pos += ph.n;
  }
  return BL_OK;
}

// out[(k * cols + col) * ncomp + m] = sum_{u in pair k} part[(col * n_units + u) * ncomp + m]; the
// units are the chunks, the stencil tiles or the J w tiles (kUnit*).
__global__ void k_reduce_units(const PairDev* pairs, const double* part, int n_units, int ncomp, int cols,
                               int units, const int* mask, const int* colcnt, double* out) {
  const int k = blockIdx.x, col = blockIdx.y;
  if (mask && !mask[k]) return;
  if (colcnt && col >= colcnt[k]) return;
  const PairDev pr = pairs[k];
  const int beg = units == kUnitTiles ? pr.tbeg : units == kUnitJwTiles ? pr.jtbeg : units == kUnitHTiles ? pr.htbeg : pr.cbeg;
  const int end = units == kUnitTiles ? pr.tend : units == kUnitJwTiles ? pr.jtend : units == kUnitHTiles ? pr.htend : pr.cend;
  const double* pc = part + (size_t)col * n_units * ncomp;
  if (ncomp < 32) {
    // few values: a warp per value, its lanes over the units
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int m = wid; m < ncomp; m += nwarp) {
      double s = 0.0;
      for (int u = beg + lane; u < end; u += 32) s += pc[(size_t)u * ncomp + m];
      s = warp_sum(s);
      if (lane == 0) out[((size_t)k * cols + col) * ncomp + m] = s;
    }
    return;
  }
  for (int m = threadIdx.x; m < ncomp; m += blockDim.x) {
    double s = 0.0;
    for (int u = beg; u < end; ++u) s += pc[(size_t)u * ncomp + m];
    out[((size_t)k * cols + col) * ncomp + m] = s;
  }
}

bl_status reduce_units(bl_problem* P, const double* part, int ncomp, int cols, int units, const int* mask,
                       const int* colcnt, double* out) {
  const int n_units = units == kUnitTiles    ? P->n_tiles
                      : units == kUnitJwTiles ? P->n_jtiles
                      : units == kUnitHTiles  ? P->n_htiles
                                              : P->n_chunks;
  k_reduce_units<<<dim3(P->K, cols), 128, 0, P->stream>>>(P->d_pairs, part, n_units, ncomp, cols, units, mask,
                                                          colcnt, out);
  BL_LAUNCH_CHECK(P);
  return BL_OK;
}

bl_status reduce_chunk_partials(bl_problem* P, int ncomp, const int* mask, double* out) {
  return reduce_units(P, P->cpart, ncomp, 1, kUnitChunks, mask, nullptr, out);
}

bl_status reduce_tile_partials(bl_problem* P, int ncomp, int cols, const int* mask, double* out) {
  return reduce_units(P, P->tpart, ncomp, cols, kUnitTiles, mask, nullptr, out);
}

template <typename T>
__global__ void k_dot(const PairDev* pairs, const ChunkDev* chunks, const T* a, const T* b, const int* mask,
                      double* cpart) {
  __shared__ double red[40];
  const ChunkDev ch = chunks[blockIdx.x];
  if (mask && !mask[ch.pair]) return;
  const PairDev pr = pairs[ch.pair];
  Accum<T> acc;
  for (int t = threadIdx.x; t < ch.len; t += blockDim.x) {
    const long long i = pr.off + ch.start + t;
    acc.add(a[i] * b[i]);
  }
  const double s = block_total<kChunkThreads>(acc, red);
  if (threadIdx.x == 0) cpart[blockIdx.x] = s;
}

bl_status batched_dot(bl_problem* P, const void* a, const void* b, const int* mask, double* out) {
  bl_status st = ensure_cpart(P, P->n_chunks);
  if (st != BL_OK) return st;
  if (P->prec == BL_FP32)
    k_dot<float><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const float*)a,
                                                                (const float*)b, mask, P->cpart);
  else
    k_dot<double><<<P->n_chunks, kChunkThreads, 0, P->stream>>>(P->d_pairs, P->d_chunks, (const double*)a,
                                                                 (const double*)b, mask, P->cpart);
  BL_LAUNCH_CHECK(P);
  return reduce_chunk_partials(P, 1, mask, out);
}

}  // namespace bl
