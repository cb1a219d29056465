// Internal declarations shared by the translation units of libbl.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bl.h"

namespace bl {

// ---------------------------------------------------------------------------------------------
// Error handling: a thread-local message, set by fail(); every entry point returns a status.
void set_error(const std::string& msg);
std::string error_copy();
bl_status fail(bl_status st, const std::string& msg);

#define BL_CUDA_TRY(expr)                                                                  \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess)                                                                 \
      return ::bl::fail(BL_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));     \
  } while (0)

#define BL_LAUNCH_CHECK(prob)                                                              \
  do {                                                                                     \
    (prob)->launches++;                                                                    \
    cudaError_t _e = cudaGetLastError();                                                   \
    if (_e != cudaSuccess)                                                                 \
      return ::bl::fail(BL_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(_e));\
  } while (0)

// ---------------------------------------------------------------------------------------------
// Geometry.  Every batched n-vector is the concatenation of the pairs' images (pair k at
// pixel offset off_k).  A batched n x M matrix keeps, for pair k, a column-major n_k x M
// block starting at off_k * M (column j of pair k at off_k * M + j * n_k).

constexpr int kTileRegion = 64;           // side of the step-1 region of the fused stencil
constexpr int kHalo = 8;                  // staged halo: covers 2 r_b (r_b <= 4) and 2 r_f (r_f <= 3)
constexpr int kStencilThreads = 256;
constexpr int kChunk = 4096;              // pixels per block of the elementwise kernels
constexpr int kChunkThreads = 256;
constexpr int kMaxFilters = 64;
constexpr int kMaxTM = 96;                // max columns of W (recycle + basis)
constexpr int kMaxHistory = 16;           // L-BFGS memory

__host__ __device__ constexpr int tile_out(int F) { return (kTileRegion - 2 * (F / 2)) & ~3; }
// Output side of the J w tiles.  J w has no step-1 region to fit in 64 x 64 (its K_j w is computed
// per 4 x 4 block straight from the staged tile), so FP32 takes the full 16 x 16 grid of 4 x 4
// blocks: one tile covers a 64 x 64 image.  FP64 keeps the stencil's tile (its 7 x 7 shared-memory
// budget has no room for a wider staged region).
template <typename T>
__host__ __device__ constexpr int jw_tile_out(int F) { return sizeof(T) == 4 ? 64 : tile_out(F); }
// Which work-list a per-pair reduction of unit partials walks.
constexpr int kUnitChunks = 0;
constexpr int kUnitTiles = 1;
constexpr int kUnitJwTiles = 2;
constexpr int kUnitHTiles = 3;

struct PairDev {
  int h, w;
  long long n, off;
  const unsigned char* opm;   // inpainting: this pair's measured-pixel mask (A = diag(opm != 0)); null: blur
  int rb;
  int tbeg, tend;      // tiles [tbeg, tend) of this pair
  int jtbeg, jtend;    // J w tiles [jtbeg, jtend)
  int cbeg, cend;      // chunks [cbeg, cend)
  int htbeg, htend;    // tiles [htbeg, htend) of the TMA-staged kernels' list
  float gf[2 * BL_MAX_BLUR_RADIUS + 1];
  double gd[2 * BL_MAX_BLUR_RADIUS + 1];
};

struct TileDev { int pair, oy, ox; };
// Tile of the TMA-staged Hessian action: var selects the tile geometry (0: tile_out(F), 1: 64 x 64)
struct HTileDev { int pair, oy, ox, var; };
struct ChunkDev { int pair; long long start; int len; };

// Per-pair scalar state of a Krylov solve (FP64 recurrences).
struct SolveState {
  double rho, rho_new, alpha, beta, pq, est, tol, gnorm2;
  // MINRES: Lanczos beta_k, zeta_k, the last two Givens rotations, and the step coefficients
  // (gamma_k, delta_k, 1 / eps~_k, c_k zeta_{k-1}, 1 / beta_{k+1}) handed to the update pass
  double beta_l, zeta, cm1, sm1, cm2, sm2, gam, del, inv_et, coef, inv_bn;
  int active, iters, status, maxit;
};

// Per-pair L-BFGS state.
// The (s, y) history is a ring of m + 1 slots: the newest `hist_count` <= m pairs are valid and
// `hist_head` (the next slot written) never holds one of them.
struct LbfgsState {
  double f, f_trial, gtd, t, gnorm, gtol, gamma;
  int active, accepted, iters, status, hist_count, hist_head, backtracks;
  int phase;   // kLbDir: needs a direction; kLbTrial: line search running; kLbAccepted: step to take
};
constexpr int kLbDir = 0, kLbTrial = 1, kLbAccepted = 2;

struct ProfEvent {
  cudaEvent_t a, b;
  int cls;
};

// Cached CUDA graph of the recycled-CG loop (a WHILE node around one iteration).
struct KrylovGraphKey {
  bool fused;
  int store, nsc, minres;
  const void *tpart, *cpart, *V;
  bool operator==(const KrylovGraphKey& o) const {
    return fused == o.fused && store == o.store && nsc == o.nsc && minres == o.minres && tpart == o.tpart &&
           cpart == o.cpart && V == o.V;
  }
};
// The L-BFGS loop as one graph launch: its body bakes these options into its kernels.
struct LbfgsGraphKey {
  const void *cpart, *tpart, *S;
  int MH, max_bt, maxit;
  double slack;
  bool operator==(const LbfgsGraphKey& o) const {
    return cpart == o.cpart && tpart == o.tpart && S == o.S && MH == o.MH && max_bt == o.max_bt && maxit == o.maxit &&
           slack == o.slack;
  }
};
struct KrylovGraph {
  KrylovGraphKey key{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int body_kernels = 0;
};

struct PairHost {
  int h, w;
  long long n, off;
  int rb;
  double sigma;
  bool masked;
  int tbeg, tend, cbeg, cend, jtbeg, jtend;
};

}  // namespace bl

struct bl_problem {
  int K = 0;
  int prec = BL_FP32;
  size_t esz = 4;
  bl_reg_desc reg{};
  int p = 0, N = 0, F = 1, rf = 0;
  int SMAX = 0, KMAX = 0, TM = 0;
  std::vector<bl::PairHost> ph;
  long long n_tot = 0;
  cudaStream_t stream = nullptr;
  int64_t launches = 0;
  int n_tiles = 0, n_chunks = 0, n_jtiles = 0;
  bool vec4 = false;                // every pair's n is a multiple of 4 (16-byte column starts)
  // TMA-staged FP32 Hessian action: tensor maps per pair for the fields (slot 0) and for each input
  // buffer the Hessian action is launched on (slots 1..tma_slots), encoded at creation
  bool tma = false;
  void* d_tmaps = nullptr;
  const void* tma_in_ptr[8] = {};
  int tma_in_mult[8] = {};
  int tma_slots = 0;
  int tma_nvar = 0;                 // tile variants with encoded maps
  bl::HTileDev* d_htiles = nullptr; // tile list of the TMA-staged Hessian action
  int n_htiles = 0, htiles_cap = 0;
  std::vector<int> hvar;            // per pair: its tile variant
  std::vector<bl::PairDev> pd_host; // host copy of d_pairs (the H tile ranges change after tuning)
  int* d_kerr = nullptr;            // error word of bounded device waits (0: none)

  bl::PairDev* d_pairs = nullptr;
  bl::TileDev* d_tiles = nullptr;
  bl::TileDev* d_jtiles = nullptr;         // the J w work-list (tiles of jw_tile_out)
  bl::ChunkDev* d_chunks = nullptr;

  void *y = nullptr, *xstar = nullptr, *xhat = nullptr;
  void *fu = nullptr, *fd = nullptr;       // FoE fields u_j = k_j * x^, d_j = e^{alpha_j} phi''(u_j)
  double* theta = nullptr;                 // p
  float* taps_f = nullptr;                 // N * F * F
  double* taps_d = nullptr;
  double* ealpha = nullptr;                // N: exp(alpha_j)  (TV: [exp(theta_0)])
  bool point_set = false;

  // Krylov vectors and recycle state
  void *r = nullptr, *pv = nullptr, *q = nullptr, *w = nullptr, *g = nullptr, *tmp = nullptr;
  // MINRES vectors (v_{k-1}, vt_{k-1}, vt_{k-2}) and s-vectors (beta~_{k-1,k-2}, Z^T Hvt_{k-1,k-2}),
  // allocated on the first MINRES solve
  void *mv_prev = nullptr, *my1 = nullptr, *my2 = nullptr;
  double* mrs = nullptr;
  unsigned char* d_opmask = nullptr;   // inpainting masks of all pairs (n_tot bytes), if any pair has one
  // Lanczos-relation record of the last CG solve (BL_STORE_LANCZOS): per pair and step j < KMAX,
  // alpha_j, rho_j = ||r_j||^2 and C^T H p_j; lz_k[k] = 1 when pair k's stored basis is such a record
  // (a refresh or a checkpoint import consumes it); lz_u[k] = 1 when that solve deflated with the
  // recycle space the pair holds now, so its C^T H p_j complete the relation for [U, V]
  double *lz_alpha = nullptr, *lz_rho = nullptr, *lz_c = nullptr;
  std::vector<int> lz_k, lz_u;
  void *U = nullptr, *C = nullptr, *Z = nullptr, *V = nullptr;
  void *W = nullptr, *Wt = nullptr, *HWt = nullptr;
  bl::SolveState* st = nullptr;
  double *c = nullptr, *zc = nullptr, *e = nullptr, *ztr = nullptr, *ztc = nullptr;
  int* d_s = nullptr;       // recycle dimension per pair
  int* d_hasz = nullptr;    // pair has an NSC operator Z
  int* d_active = nullptr;  // generic per-pair mask
  int* d_cols = nullptr;    // per-pair column counts for multi-column kernels
  int* d_flag = nullptr;    // any-active flag (device)
  int* d_zero = nullptr;    // K zeros (per-pair "none" flags)
  int* d_loop = nullptr;    // graph loop counter and cap
  cudaStream_t cstream = nullptr;   // private stream used only to capture graphs
  bl::KrylovGraph* kgraph = nullptr;
  bl::KrylovGraph* lgraph = nullptr;     // the L-BFGS loop (its key: lgraph_key)
  bl::LbfgsGraphKey lgraph_key{};
  bool graph_failed = false;        // graph capture unavailable: the stream path is used
  bool graph_used = false;          // the last solve ran as a graph launch
  bool capturing = false;           // a graph capture is recording the launches
  std::string graph_error;          // why the graph capture failed, if it did
  int* h_flag = nullptr;    // pinned host mirror
  std::vector<int> s_k, kb_k, hz_k, head_k;

  // dense small-matrix workspace (FP64)
  double *dG = nullptr, *dT = nullptr, *dJ = nullptr, *dY = nullptr, *dY2 = nullptr, *dY3 = nullptr;
  int* d_tk = nullptr;      // 3K ints: reduced basis size t' per pair, selected s, previous s in W

  // L-BFGS
  void *lx = nullptr, *lg = nullptr, *ld = nullptr, *lxt = nullptr, *lgt = nullptr, *lq = nullptr;
  void *S = nullptr, *Yh = nullptr;    // n x (MH + 1) ring of s and y columns
  double *lsy = nullptr, *lyy = nullptr; // K x (MH + 1)^2: s_i^T y_j and y_i^T y_j by slot
  double *lcs = nullptr, *lcy = nullptr; // K x (MH + 1): direction coefficients by slot
  bl::LbfgsState* lst = nullptr;
  int MH = 0;

  // profiling: events per launch and device pixel counters per kernel class
  bool prof = false;
  std::vector<bl::ProfEvent> prof_ev;
  size_t prof_used = 0;
  double prof_ms[BL_KC_COUNT] = {};
  int64_t prof_n[BL_KC_COUNT] = {};
  unsigned long long* d_pix = nullptr;   // BL_KC_COUNT counters
  unsigned long long* d_bytes = nullptr; // BL_KC_COUNT algorithmic byte counters

  // partial sums
  double* tpart = nullptr;
  size_t tpart_cap = 0;
  double* cpart = nullptr;
  size_t cpart_cap = 0;
  double* vals = nullptr;   // per-pair reduced values (K * 8)
};

namespace bl {

// Profiling scope: records a CUDA event pair around the launches it encloses when enabled.
struct ProfScope {
  bl_problem* P;
  int slot;
  ProfScope(bl_problem* p, int cls);
  ~ProfScope();
};
unsigned long long* pix_counter(bl_problem* P, int cls);   // null when profiling is off
unsigned long long* bytes_counter(bl_problem* P, int cls); // null when profiling is off

// Allocation helper (tracks nothing; caller frees in bl_problem_destroy).
bl_status dalloc(void** ptr, size_t bytes);
bl_status ensure_tpart(bl_problem* P, size_t doubles);
bl_status ensure_cpart(bl_problem* P, size_t doubles);
bl_status set_active_pairs(bl_problem* P, const int32_t* pairs, int32_t npairs);
bl_status gather_packed(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* packed,
                        void* batched);
bl_status scatter_packed(bl_problem* P, const int32_t* pairs, int32_t npairs, const void* batched,
                         void* packed);
bl_status check_pairs(const bl_problem* P, const int32_t* pairs, int32_t npairs);

// ---- stencil.cu ----
// out = H v for `cols` columns of a batched matrix (mult = 0: plain batched vector).
// With dots_s != null (FoE only) the tile partials of p^T q, C^T q (dots_s[k] columns) and Z^T q
// (if dots_hz[k]) are written to tpart, layout [tile][1 + 2 SMAX].
bl_status launch_hvp(bl_problem* P, const void* in, void* out, int mult, int cols, const int* mask,
                     const int* dots_s, const int* dots_hz);
bl_status launch_grad(bl_problem* P, const void* x, void* grad, const int* mask, double* values);
bl_status launch_fields(bl_problem* P, const int* mask);
bl_status launch_forward(bl_problem* P, const void* x, void* out, const int* mask);
// J w for `cols` columns: per-pair results (K x cols x p doubles, [k][col][m]) in out.
bl_status launch_jw(bl_problem* P, const void* in, int mult, int cols, const int* mask, double* out);
bl_status load_theta(bl_problem* P, const double* theta);
// Raise the dynamic shared-memory limits of the stencil kernels this problem launches (done once at
// creation, so that graph capture never has to change function attributes).
bl_status prepare_kernels(bl_problem* P);

// ---- hvp_tma.cu ----
// Encode the tensor maps of the TMA-staged FP32 Hessian action (sets P->tma when the problem
// qualifies: FP32 FoE, every width a multiple of 4); prepare its shared-memory limit.
bl_status hvp_tma_setup(bl_problem* P);
bl_status prepare_hvp_tma(bl_problem* P);
// Slot of an input buffer whose tensor maps exist, or -1.
int hvp_tma_slot(const bl_problem* P, const void* in, int mult);
bl_status launch_hvp_tma(bl_problem* P, int slot, const void* in, void* out, int mult, int cols, const int* mask);
// Gradient and value partials of Phi (eq. (5.1)) by the TMA-staged kernel; false-free: returns -1 from
// hvp_tma_grad_slot when the input buffer has no tensor maps (the generic kernel runs then).
int hvp_tma_grad_slot(const bl_problem* P, const void* x);
bl_status launch_grad_tma(bl_problem* P, int slot, void* grad, const int* mask, double* tpart);
// Output tile side of the TMA-staged Hessian action for one pair (0 when the generic kernel runs), and
// forcing a pair's tile variant (tests check every variant).
int hvp_tma_tile(const bl_problem* P, int pair);
bl_status hvp_tma_force_tile(bl_problem* P, int pair, int side);
// Whether the Krylov loop takes its dot products from the Hessian action's epilogue (tile partials)
// or from the separate chunk pass (the TMA-staged kernel computes q only).
inline bool hvp_fused_dots(const bl_problem* P) { return P->reg.kind == BL_REG_FOE && !P->tma; }
// Read and clear the device error word of bounded waits (synchronises the stream).
bl_status check_kernel_error(bl_problem* P);

// ---- krylov.cu ----
bl_status run_hessian_solve(bl_problem* P, const int* mask_host, const bl_krylov_opts* o,
                            const void* g_batched, const double* nsc_scale_batched,
                            std::vector<bl_solve_info>& info);

void destroy_krylov_graph(bl_problem* P);   // also drops the L-BFGS loop graph
void destroy_lbfgs_graph(bl_problem* P);

// ---- recycle.cu ----
bl_status run_ritz_update(bl_problem* P, const std::vector<int>& mask_host,
                          const bl_recycle_opts* o);

// ---- lbfgs.cu ----
bl_status run_lower_solve(bl_problem* P, const std::vector<int>& mask_host, const bl_lbfgs_opts* o,
                          std::vector<bl_solve_info>& info);

// ---- vec.cu: batched vector helpers ----
// Sum per-unit partials (units = tiles or chunks; layout part[(col * n_units + u) * ncomp + m])
// over the units of each pair: out[(k * cols + col) * ncomp + m].
bl_status reduce_units(bl_problem* P, const double* part, int ncomp, int cols, int units, const int* mask,
                       const int* colcnt, double* out);
// Reduce per-chunk partials: out[k * ncomp + c] = sum over chunks of pair k (masked pairs only).
bl_status reduce_chunk_partials(bl_problem* P, int ncomp, const int* mask, double* out);
bl_status reduce_tile_partials(bl_problem* P, int ncomp, int cols, const int* mask, double* out);
// dot products per pair: out[k] = sum_i a_i b_i (FP64 accumulation).
bl_status batched_dot(bl_problem* P, const void* a, const void* b, const int* mask, double* out);
// Tall-skinny products (tsmm.cu).  ts_gram: out[k] (TM x TM, FP64) = A_k^T B_k over the colsA[k]
// and colsB[k] leading columns (cmaxA, cmaxB: their maxima).  ts_gemm: O1_k = A_k M1_k (cols1[k]
// columns), O2_k = A_k M2_k (optional); M: K x TM x TM FP64; O1 may alias A.
bl_status ts_gram(bl_problem* P, const void* A, int multA, const int* colsA, int cmaxA, const void* B, int multB,
                  const int* colsB, int cmaxB, const int* mask, double* out);
bl_status ts_gemm(bl_problem* P, const void* A, int multA, const int* colsA, int cmaxA, const double* M1, void* O1,
                  int mult1, const int* cols1, int cmax1, const double* M2, void* O2, int mult2, const int* cols2,
                  int cmax2, const int* mask);

}  // namespace bl
