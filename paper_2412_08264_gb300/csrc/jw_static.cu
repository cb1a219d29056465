// Allocation-free J w for one FP32 image: the scratch lives in a fixed device array.
//
// Some callers cannot allocate device memory: code that runs inside a host framework which owns
// the whole device heap (a serving process or a plugin whose pool forbids cudaMalloc after
// start-up), or any caller under a no-allocation rule once it is running.  Creating a bl_problem
// allocates, so those callers use this entry point instead: it computes the same contraction as
// bl_hypergrad for one image, with every intermediate (exp(alpha_j), the taps and the per-tile
// partial sums) held in `g_jw_scratch`, a file-scope __device__ array of fixed size that each GPU
// loading the library keeps until the process exits.
//
// In host code the name g_jw_scratch stands for a host-side shadow, not a device address, so the
// device address is looked up once per device with cudaGetSymbolAddress (with that device
// current) and cached; kernels receive that address.  All calls share the array: calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on it.
#include <mutex>

#include "common.cuh"
#include "device.cuh"

namespace {

constexpr int kTile = 32;                        // output tile side
constexpr size_t kHead = 4096;                   // doubles: exp(alpha_j) at [0, 64), taps at [64, 64 + N f^2)
constexpr size_t kPartials = 524288;             // doubles of per-tile partial sums (4 MiB)

static __device__ __align__(256) double g_jw_scratch[kHead + kPartials];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
double* g_addr[kMaxDevices] = {};

bl_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bl::fail(BL_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return bl::fail(BL_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_jw_scratch);
    if (e != cudaSuccess || !p)
      return bl::fail(BL_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return BL_OK;
}

__global__ void k_static_theta(const double* theta, int N, int FF, double* scratch) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * (FF + 1); i += gridDim.x * blockDim.x) {
    const int j = i / (FF + 1), t = i - j * (FF + 1);
    if (t == 0) scratch[j] = exp(theta[i]);
    else scratch[64 + j * FF + t - 1] = theta[i];
  }
}

// Per tile and filter j, with u = k_j * x^, e = phi'(u), d = phi''(u) (k_j * w):
//   alpha_j part  -e^{alpha_j} sum_p e_p (k_j * w)_p
//   tap (a, b)    -e^{alpha_j} sum_p [ e_p w_{p+o} + d_p x^_{p+o} ],  o = (a - r, b - r)
template <int F>
__global__ void __launch_bounds__(256) k_static_jw(const float* __restrict__ xhat, const float* __restrict__ w,
                                                   int h, int wd, int N, float eps, int phi, int p,
                                                   double* scratch) {
  constexpr int R = F / 2, RS = kTile + 2 * R, FF = F * F;
  __shared__ float xs[RS * RS], ws[RS * RS];
  __shared__ double red[8][FF + 1];
  const int ntx = (wd + kTile - 1) / kTile;
  const int oy = (blockIdx.x / ntx) * kTile, ox = (blockIdx.x % ntx) * kTile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int idx = tid; idx < RS * RS; idx += blockDim.x) {
    const int i = idx / RS, j = idx - (idx / RS) * RS;
    const int iy = oy - R + i, ix = ox - R + j;
    const bool in = iy >= 0 && iy < h && ix >= 0 && ix < wd;
    xs[idx] = in ? xhat[(long long)iy * wd + ix] : 0.f;
    ws[idx] = in ? w[(long long)iy * wd + ix] : 0.f;
  }
  __syncthreads();
  const double* ealpha = scratch;
  const double* taps = scratch + 64;
  double* part = scratch + kHead + (size_t)blockIdx.x * p;
  for (int jf = 0; jf < N; ++jf) {
    float k[FF], gt[FF];
#pragma unroll
    for (int t = 0; t < FF; ++t) {
      k[t] = (float)taps[jf * FF + t];
      gt[t] = 0.f;
    }
    double ga = 0.0;
    for (int q = tid; q < kTile * kTile; q += blockDim.x) {
      const int yy = q / kTile, xx = q - (q / kTile) * kTile;
      if (oy + yy >= h || ox + xx >= wd) continue;
      float u = 0.f, kw = 0.f;
#pragma unroll
      for (int a = 0; a < F; ++a)
#pragma unroll
        for (int b = 0; b < F; ++b) {
          u = fmaf(k[a * F + b], xs[(yy + a) * RS + xx + b], u);
          kw = fmaf(k[a * F + b], ws[(yy + a) * RS + xx + b], kw);
        }
      const float e = bl::phi_d1(u, eps, phi);
      const float d = bl::phi_d2(u, eps, phi) * kw;
      ga += (double)(e * kw);
#pragma unroll
      for (int a = 0; a < F; ++a)
#pragma unroll
        for (int b = 0; b < F; ++b)
          gt[a * F + b] = fmaf(e, ws[(yy + a) * RS + xx + b], fmaf(d, xs[(yy + a) * RS + xx + b], gt[a * F + b]));
    }
    double v = bl::warp_sum(ga);
    if (lane == 0) red[wid][0] = v;
#pragma unroll
    for (int t = 0; t < FF; ++t) {
      const double s = bl::warp_sum((double)gt[t]);
      if (lane == 0) red[wid][1 + t] = s;
    }
    __syncthreads();
    if (tid < FF + 1) {
      double s = 0.0;
      for (int q = 0; q < 8; ++q) s += red[q][tid];
      part[jf * (FF + 1) + tid] = -ealpha[jf] * s;
    }
    __syncthreads();
  }
}

__global__ void k_static_reduce(const double* scratch, int n_tiles, int p, double* out) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < p; m += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < n_tiles; ++t) s += scratch[kHead + (size_t)t * p + m];
    out[m] = s;
  }
}

}  // namespace

extern "C" bl_status bl_jw_fp32_static(const float* xhat, const float* w, int32_t height, int32_t width,
                                       const double* theta, int32_t n_filters, int32_t filter_size, int32_t phi,
                                       double phi_eps, double* out, void* cuda_stream) {
  if (!xhat || !w || !theta || !out) return bl::fail(BL_EINVAL, "null argument");
  if (height < 1 || width < 1) return bl::fail(BL_EINVAL, "image sizes must be >= 1");
  if (filter_size < 1 || filter_size > BL_MAX_FILTER_SIZE || filter_size % 2 == 0)
    return bl::fail(BL_EINVAL, "filter_size must be odd and <= 7");
  if (n_filters < 1 || n_filters > 64) return bl::fail(BL_EINVAL, "n_filters must be in 1..64");
  if (phi < BL_PHI_CHARBONNIER || phi > BL_PHI_LOG1P) return bl::fail(BL_EINVAL, "unknown phi");
  if (phi == BL_PHI_CHARBONNIER && !(phi_eps > 0.0)) return bl::fail(BL_EINVAL, "phi_eps must be > 0");
  const int FF = filter_size * filter_size;
  const int p = n_filters * (FF + 1);
  const long long n_tiles = (long long)((height + kTile - 1) / kTile) * ((width + kTile - 1) / kTile);
  if ((unsigned long long)n_tiles * (unsigned long long)p > kPartials)
    return bl::fail(BL_EINVAL, "image too large for the static scratch: ceil(H/32) * ceil(W/32) * p must be <= " +
                                   std::to_string(kPartials) + ", got " + std::to_string(n_tiles * p));
  // An error left on this thread by earlier, unrelated work would otherwise surface as this call's
  // launch failure (and be cleared by the check): report it untouched instead.
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return bl::fail(BL_ECUDA, std::string("a CUDA error was pending before this call (left untouched): ") +
                                  cudaGetErrorString(pending));
  double* s = nullptr;
  bl_status st = scratch_address(&s);
  if (st != BL_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  auto launched = [](const char* what) -> bl_status {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bl::fail(BL_ECUDA, std::string(what) + " launch: " + cudaGetErrorString(e));
    return BL_OK;
  };
  k_static_theta<<<(p + 255) / 256, 256, 0, stream>>>(theta, n_filters, FF, s);
  if ((st = launched("k_static_theta")) != BL_OK) return st;
  switch (filter_size) {
    case 1: k_static_jw<1><<<(unsigned)n_tiles, 256, 0, stream>>>(xhat, w, height, width, n_filters, (float)phi_eps, phi, p, s); break;
    case 3: k_static_jw<3><<<(unsigned)n_tiles, 256, 0, stream>>>(xhat, w, height, width, n_filters, (float)phi_eps, phi, p, s); break;
    case 5: k_static_jw<5><<<(unsigned)n_tiles, 256, 0, stream>>>(xhat, w, height, width, n_filters, (float)phi_eps, phi, p, s); break;
    default: k_static_jw<7><<<(unsigned)n_tiles, 256, 0, stream>>>(xhat, w, height, width, n_filters, (float)phi_eps, phi, p, s); break;
  }
  if ((st = launched("k_static_jw")) != BL_OK) return st;
  k_static_reduce<<<(p + 255) / 256, 256, 0, stream>>>(s, (int)n_tiles, p, out);
  if ((st = launched("k_static_reduce")) != BL_OK) return st;
  return BL_OK;
}
