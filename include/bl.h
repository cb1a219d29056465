/*
 * bl.h -- C ABI of the GB300 bilevel-hypergradient library.
 *
 * One call sequence computes the hypergradient of a variational imaging
 * problem for a batch of K training pairs (Ehrhardt, Gazzola, Scott,
 * "Efficient gradient-based methods for bilevel learning via recycling
 * Krylov subspaces"):
 *
 *   bl_problem_create   pairs (y_k, x*_k), operator A_k (blur or inpainting mask), regulariser R(x, theta)
 *   bl_lower_solve      x^_k = argmin_x Phi_k(x, theta)          (eq. (1.1), (5.1); L-BFGS, Section 5.1)
 *   bl_ritz_update      refresh U, C = H U from W = [U, V]       (Section 3, eq. (3.3) outer / (3.4) inner form)
 *   bl_hessian_solve    H_k w_k = grad ell_k by recycled CG or recycled MINRES
 *                       (Section 2.2, eq. (2.5), Algorithm 3, Section 4 stopping)
 *   bl_hypergrad        g_k = J_k w_k = -(D^2_{theta x} Phi_k)^T w_k   (eq. (2.7))
 *
 * Conventions shared by every entry point
 *   - Images are H x W, row-major, pixel p = i * W + j, zero boundary.
 *   - Scalar type of every image buffer is the problem's precision:
 *     float for BL_FP32 (FP32 stencils, FP64 reductions and scalar recurrences),
 *     double for BL_FP64.
 *   - A "packed" buffer holds the images of the listed pairs back to back, in the
 *     order of the `pairs` index array, each H_k * W_k elements.
 *   - Device pointers are CUDA device memory owned by the caller unless stated, on the
 *     device that was current when the problem was created (the library cannot check this:
 *     memory of another device, or host memory, is undefined behaviour on the GPU); the
 *     library reads them during the call's stream work and keeps no reference.
 *   - theta (length p, double, device) is laid out per filter as
 *     [alpha_1, taps_1 (f*f row-major, tap (a, b) at (a + r) * f + (b + r)), alpha_2, ...]
 *     for the Fields-of-Experts regulariser (Section 5), p = N (f*f + 1); p = 1 for TV.
 *   - All work is enqueued on the problem's stream.  Calls that return an info
 *     array or host values synchronise that stream before returning.
 *   - Errors: no exception crosses the ABI.  A call returns a bl_status; on any
 *     status other than BL_OK / BL_ENOCONV, bl_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread).
 */
#ifndef BL_H_
#define BL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BL_MAX_FILTER_SIZE 7   /* f in {1, 3, 5, 7} */
#define BL_MAX_BLUR_RADIUS 4   /* blur support (2 r_b + 1)^2, r_b <= 4 */

typedef enum {
  BL_OK = 0,
  BL_EINVAL = 1,       /* invalid argument: null pointer, size, option out of range */
  BL_ENOMEM = 2,       /* device allocation failed */
  BL_ECUDA = 3,        /* a CUDA runtime call failed (message names it) */
  BL_ENOCONV = 4,      /* a solve hit its iteration cap; results are still written */
  BL_EBREAKDOWN = 5,   /* non-positive curvature or a non-finite value in a solve */
  BL_ESTATE = 6        /* call out of order (e.g. solve before a point was set) */
} bl_status;

typedef enum { BL_REG_TV = 0, BL_REG_FOE = 1 } bl_reg_kind;
typedef enum { BL_PHI_CHARBONNIER = 0, BL_PHI_SQ = 1, BL_PHI_LOG1P = 2 } bl_phi_kind;
typedef enum { BL_FP32 = 0, BL_FP64 = 1 } bl_precision;

/* One training pair: image size and its forward operator A.
 *   mask == NULL: the Gaussian blur of Section 5.2, G[a, b] proportional to
 *                 exp(-(a^2 + b^2) / (2 sigma^2)) on [-r_b, r_b]^2, summing to 1.
 *   mask != NULL: inpainting (Section 5.1): A keeps the measured pixels, A = diag(mask != 0) on
 *                 the image grid (measurements y are zero elsewhere); host, height * width bytes,
 *                 row-major, copied at create; blur_sigma and blur_radius are ignored. */
typedef struct {
  int32_t height, width;
  double blur_sigma;
  int32_t blur_radius;
  const uint8_t* mask;
} bl_pair_desc;

/* Lower-level functional (eq. (1.1) with the eps term of eq. (5.1)):
 *   Phi(x) = ||A x - y||^2 + R(x, theta) + (l2_eps / 2) ||x||^2
 * FoE: R = sum_j exp(alpha_j) sum_p phi((k_j * x)[p]), (k * x)[p] = sum_o k[o] x[p + o].
 * TV:  R = exp(theta_0) sum_p sqrt(|(D x)_p|^2 + phi_eps^2), forward differences. */
typedef struct {
  int32_t kind;          /* bl_reg_kind */
  int32_t n_filters;     /* N (FoE) */
  int32_t filter_size;   /* f, odd, <= BL_MAX_FILTER_SIZE (FoE) */
  int32_t phi;           /* bl_phi_kind (FoE) */
  double phi_eps;        /* Charbonnier / TV smoothing */
  double l2_eps;         /* eps of eq. (5.1) */
  int32_t precision;     /* bl_precision */
  int32_t max_recycle;   /* largest recycle dimension s any later call may ask for */
  int32_t max_basis;     /* Krylov vectors kept per solve for the next refresh (most recent) */
} bl_reg_desc;

typedef struct {
  int32_t max_iters;     /* L-BFGS iteration cap */
  int32_t history;       /* memory m (Section 5.1 uses 10), 1..16 */
  double gtol;           /* stop when ||grad Phi|| <= gtol (absolute) ... */
  int32_t gtol_relative; /* ... or, if non-zero, <= gtol * ||grad Phi(0)|| = gtol * ||2 A^T y|| */
  int32_t max_backtrack; /* Armijo halvings per iteration */
  double armijo_slack;   /* accept Phi(x + t d) <= Phi(x) + 1e-4 t g^T d + armijo_slack |Phi(x)|:
                            0 is the plain Armijo rule; FP32 problems need about 1e-6 because FP32
                            values of Phi cannot resolve decreases below that level */
  int32_t graph;         /* non-zero: run the iteration loop as one CUDA-graph launch (a WHILE node whose
                            condition is set on the device); the host-polled loop is used instead while
                            profiling is enabled */
} bl_lbfgs_opts;

/* CG / recycled CG (augmented CG on P H P, P = I - C C^T: valid for SPD Hessians) and MINRES /
   recycled MINRES (Algorithm 3 with the recurrences of Appendix A: valid for symmetric indefinite
   Hessians, e.g. the non-convex phi = log(1 + s^2) of Section 5.2).  Both store the basis they
   build (normalised CG residuals / Lanczos vectors) for bl_ritz_update. */
typedef enum { BL_SOLVE_CG = 0, BL_SOLVE_RCG = 1, BL_SOLVE_MINRES = 2, BL_SOLVE_RMINRES = 3 } bl_solve_method;
typedef enum { BL_STOP_RESID = 0, BL_STOP_NSC = 1 } bl_stop_rule;
/* Basis kept by bl_hessian_solve for the next refresh:
 *   BL_STORE_NONE
 *   BL_STORE_RECENT   the most recent max_basis basis vectors (CG: normalised residuals; MINRES:
 *                     Lanczos vectors), for the outer refresh (eq. (3.3));
 *   BL_STORE_LANCZOS  (CG only) the first max_basis normalised residuals with the CG coefficients
 *                     alpha_j, rho_j and C^T H p_j, from which the refresh rebuilds H V through the
 *                     Lanczos relation of the projected operator: the inner refresh (eq. (3.4)). */
typedef enum { BL_STORE_NONE = 0, BL_STORE_RECENT = 1, BL_STORE_LANCZOS = 2 } bl_store_mode;

typedef struct {
  int32_t method;        /* BL_SOLVE_CG / BL_SOLVE_MINRES ignore the recycle space; BL_SOLVE_RCG /
                            BL_SOLVE_RMINRES use it (if any) */
  int32_t stop;          /* BL_STOP_RESID: ||r|| < tol * scale;
                            BL_STOP_NSC: ||Z^T r|| < tol * scale (eq. (4.2)); falls back to the
                            residual rule for a pair without a Ritz-GSV recycle space */
  double tol;
  int32_t relative;      /* RESID: scale = ||g_k|| if non-zero, else 1.
                            NSC:   scale = nsc_scale[k] from bl_hessian_solve, else 1. */
  int32_t maxit;
  int32_t store_basis;   /* bl_store_mode: keep the basis for the next bl_ritz_update */
  int32_t warm_start;    /* non-zero: w (in) is the initial guess; zero: start from 0 */
  int32_t graph;         /* non-zero: run the iteration loop as one CUDA-graph launch (a WHILE node whose
                            condition is set on the device), without host round trips; the stream path
                            is used instead while profiling is enabled */
} bl_krylov_opts;

typedef enum { BL_RECYCLE_RITZ = 0, BL_RECYCLE_HRITZ = 1, BL_RECYCLE_RGSV = 2 } bl_recycle_kind;
typedef enum { BL_SIZE_SMALL = 0, BL_SIZE_LARGE = 1, BL_SIZE_MIXED = 2 } bl_recycle_size;
typedef enum { BL_SIDE_RIGHT = 0, BL_SIDE_LEFT = 1, BL_SIDE_MIXED = 2 } bl_recycle_side;

/* Which Hessian projects W = [U, V] (Section 3.1): the current one, W^T H^(i) W (eq. (3.3), t Hessian
 * actions), or the one V was built with, W^T H^(i-1) W (eq. (3.4)), rebuilt from the stored CG
 * coefficients without Hessian actions; the selected U is then paired with C = H^(i) U (s actions). */
typedef enum { BL_REFRESH_OUTER = 0, BL_REFRESH_INNER = 1 } bl_refresh_variant;

/* Table 1 grammar: Ritz-S = {RITZ, SMALL}, RGen-L(R) = {RGSV, LARGE, RIGHT}. */
typedef struct {
  int32_t kind;          /* bl_recycle_kind */
  int32_t size;          /* bl_recycle_size */
  int32_t side;          /* bl_recycle_side (RGSV only) */
  int32_t s;             /* recycle dimension, 1..max_recycle; RGSV also needs s <= p */
  int32_t variant;       /* bl_refresh_variant; INNER needs the last solve's BL_STORE_LANCZOS basis
                            (BL_ESTATE otherwise) */
} bl_recycle_opts;

typedef struct {
  int32_t iters;         /* iterations taken */
  int32_t status;        /* bl_status of this pair */
  double resid;          /* final recursive residual norm ||r|| */
  double nsc_est;        /* final ||Z^T r|| (0 without a Ritz-GSV space) */
  double rhs_norm;       /* ||g|| */
} bl_solve_info;

typedef struct bl_problem bl_problem;

/* Create a problem for K pairs (Section 5, eq. (5.2)).
 * y_packed, xstar_packed: device, packed over pairs 0..K-1, precision's scalar type; copied.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) that all later work runs on.
 * Returns BL_EINVAL for K < 1, sizes < 1, filter size even or > 7, blur radius > 4 (blur pairs),
 * n_filters < 1 (FoE), unknown enum values or a null pointer. */
bl_status bl_problem_create(const bl_pair_desc* pairs, int32_t K, const bl_reg_desc* reg,
                            const void* y_packed, const void* xstar_packed, void* cuda_stream,
                            bl_problem** out);
/* Synchronises the problem's stream, destroys its CUDA graphs and frees all device memory the
 * problem owns; prob may be NULL.  Caller buffers are untouched. */
void bl_problem_destroy(bl_problem* prob);
/* Make cuda_stream (a cudaStream_t, NULL = legacy default stream) the stream of all later calls.
 * The caller orders it after the old stream's pending work; captured CUDA graphs are kept. */
bl_status bl_set_stream(bl_problem* prob, void* cuda_stream);

/* Number of hyperparameters p and total pixels of the listed pairs (host values). */
int32_t bl_num_params(const bl_problem* prob);
int64_t bl_num_pixels(const bl_problem* prob, const int32_t* pairs, int32_t npairs);

/* Replace the measurements and ground truths of the listed pairs (device, packed); same sizes as
 * at creation.  The recycle state and the current point are kept. */
bl_status bl_set_data(bl_problem* prob, const int32_t* pairs, int32_t npairs, const void* y_packed,
                      const void* xstar_packed);

/* y_k = A_k x_k for each listed pair (the blur of Section 5.2, or the inpainting mask of
 * Section 5.1 for pairs created with one); x, out packed, device. */
bl_status bl_forward(bl_problem* prob, const int32_t* pairs, int32_t npairs, const void* x_packed,
                     void* out_packed);

/* Set the point (theta, x^_k) at which H_k and J_k are evaluated (eqs. (2.6), (2.7)) and
 * precompute the per-filter fields u_j = k_j * x^ and exp(alpha_j) phi''(u_j).
 * theta: device, p doubles.  xhat_packed: device, packed over the listed pairs. */
bl_status bl_set_point(bl_problem* prob, const int32_t* pairs, int32_t npairs,
                       const double* theta, const void* xhat_packed);

/* Lower-level solve by L-BFGS with Armijo backtracking (Section 5.1), warm-started from
 * xhat_packed (in), result written back to xhat_packed (out), then bl_set_point.
 * info: host array of npairs (iters = L-BFGS iterations, resid = final ||grad Phi||), or NULL.
 * Returns BL_ENOCONV if a pair reached max_iters. */
bl_status bl_lower_solve(bl_problem* prob, const int32_t* pairs, int32_t npairs, const double* theta,
                         const bl_lbfgs_opts* opts, void* xhat_packed, bl_solve_info* info);

/* Lower-level value and gradient at (x, theta) for the listed pairs (eq. (1.1), (5.1)):
 * grad_packed (device, packed) receives grad Phi_k(x_k); values (device, npairs doubles) Phi_k. */
bl_status bl_gradient(bl_problem* prob, const int32_t* pairs, int32_t npairs, const double* theta,
                      const void* x_packed, void* grad_packed, double* values);

/* out_k = H_k v_k at the current point (matrix-free Hessian action, eq. (2.6)). */
bl_status bl_hvp(bl_problem* prob, const int32_t* pairs, int32_t npairs, const void* v_packed,
                 void* out_packed);

/* Refresh the recycle space of each listed pair (Section 3; opts->variant picks the outer form of
 * eq. (3.3), or the inner form of eq. (3.4), which projects with the Hessian of the last CG solve
 * rebuilt from its Lanczos record):
 * W = [U^(i-1), V^(i-1)] is orthonormalised, projected with H (and J for RGSV),
 * the s selected vectors U~ are QR-normalised so that C = H U, C^T C = I (Section 2.2.2), and
 * for RGSV the estimate operator Z = W~ V~_H diag(mu) of eq. (4.2) is stored.
 * A pair without a stored basis keeps an empty recycle space.  A pair whose projected matrix is not
 * positive definite (T for RGSV, C~^T C~ in the CholeskyQR of C~ = H U~) is left with an empty
 * recycle space (its next solve is plain CG) while the other pairs are refreshed; the call then
 * returns BL_EBREAKDOWN. */
bl_status bl_ritz_update(bl_problem* prob, const int32_t* pairs, int32_t npairs,
                         const bl_recycle_opts* opts);

/* Solve H_k w_k = g_k for the listed pairs in one batched run of (recycled) CG or (recycled)
 * MINRES, as opts->method says (Section 2.2, Algorithm 3):
 *   g_packed: device right-hand sides, or NULL for g_k = x^_k - x*_k (grad of 1/2||x - x*||^2);
 *   w_packed: device, in = warm start (if opts->warm_start), out = solution;
 *   nsc_scale: host, npairs doubles used by a relative NSC rule, or NULL;
 *   info: host, npairs entries, or NULL.
 * The stored Krylov basis V (if opts->store_basis) replaces the previous one.
 * Returns BL_ENOCONV if a pair hit maxit, BL_EBREAKDOWN if a pair broke down. */
bl_status bl_hessian_solve(bl_problem* prob, const int32_t* pairs, int32_t npairs,
                           const bl_krylov_opts* opts, const void* g_packed, void* w_packed,
                           const double* nsc_scale, bl_solve_info* info);

/* Hypergradient contributions g_k = J_k w_k = -(D^2_{theta x} Phi_k)^T w_k (eq. (2.7)):
 *   grads: device, npairs x p doubles (row k for listed pair k), or NULL;
 *   mean_grad: device, p doubles = (1/npairs) sum_k g_k, or NULL;
 *   loss: host, if non-NULL receives (1/npairs) sum_k 1/2 ||x^_k - x*_k||^2 (eq. (5.2)). */
bl_status bl_hypergrad(bl_problem* prob, const int32_t* pairs, int32_t npairs, const void* w_packed,
                       double* grads, double* mean_grad, double* loss);

/* Current recycle dimension and stored basis size of one pair (host values). */
int32_t bl_recycle_dim(const bl_problem* prob, int32_t pair);
int32_t bl_basis_size(const bl_problem* prob, int32_t pair);

/* Checkpoint of one pair's recycle state to a host buffer: U, C, Z, Z^T C and sizes, then the stored
 * Krylov basis the next bl_ritz_update would read (its columns in storage order and, for a
 * BL_STORE_LANCZOS record, the CG coefficients), so that a run resumed from the checkpoint continues
 * exactly as the uninterrupted one (layout version 2; version-1 buffers, without the basis, are
 * still accepted and leave the pair without a stored basis).
 * bl_recycle_export: with buf == NULL sets *bytes to the size needed; otherwise writes
 * at most *bytes (BL_EINVAL if too small) and sets *bytes to the size written.
 * bl_recycle_import: restores a buffer written by bl_recycle_export for a pair of the same
 * size and precision, and (version 2) a problem with the same max_recycle and max_basis
 * (BL_EINVAL on any header mismatch or truncation). */
bl_status bl_recycle_export(bl_problem* prob, int32_t pair, void* buf, size_t* bytes);
bl_status bl_recycle_import(bl_problem* prob, int32_t pair, const void* buf, size_t bytes);

/* 1 if the last bl_hessian_solve ran its loop as a CUDA graph (see bl_krylov_opts.graph), else 0. */
int32_t bl_graph_used(const bl_problem* prob);

/* 1 if the problem's FP32 Hessian action stages its input and field tiles with tensor-memory-access
 * copies (FP32 Fields-of-Experts problem whose every image width is a multiple of 4, on a driver
 * that encodes tensor maps), 0 if it runs the generic kernel.  Both compute eq. (2.6) identically. */
int32_t bl_hvp_tma(const bl_problem* prob);

/* Output tile side of the TMA-staged Hessian action for one pair (0 if the generic kernel runs).
 * At creation the library times its tile variants per image-size class (height, width, blur radius,
 * operator) and keeps the faster: tile_out(f) (60 x 60 for 3 x 3 and 5 x 5 filters, 56 for 7 x 7, 64 for
 * 1 x 1) or, for 3 x 3 and 5 x 5 filters, 64 x 64.  Both compute eq. (2.6) identically. */
int32_t bl_hvp_tile(const bl_problem* prob, int32_t pair);
/* Force a pair's tile variant by its side (one that bl_hvp_tile can return for this filter size);
 * BL_EINVAL otherwise, or when the problem runs the generic kernel.  Synchronises the stream and
 * drops the captured Krylov-loop graph. */
bl_status bl_set_hvp_tile(bl_problem* prob, int32_t pair, int32_t side);

/* Number of this library's kernel launches since the problem was created (host counter). */
int64_t bl_launch_count(const bl_problem* prob);

/* Per-kernel-class timing (CUDA events recorded on the problem's stream around each launch
 * while enabled) and work counters (pixels x columns processed, counted by the kernels).
 * bl_profile_enable(prob, 1) clears the counters and starts recording; 0 stops.
 * bl_profile_read synchronises the stream and returns the totals of one class since enable. */
typedef enum {
  BL_KC_HVP = 0,        /* fused Hessian action in the Krylov loop (one vector) */
  BL_KC_HVP_MULTI = 1,  /* Hessian action on the columns of W~ (recycle refresh) */
  BL_KC_GRAD = 2,       /* fused gradient and value of Phi (lower solve) */
  BL_KC_JW = 3,         /* J w contraction (hypergradient and refresh) */
  BL_KC_KRYLOV = 4,     /* recycled-CG vector updates and scalar kernels */
  BL_KC_LBFGS = 5,      /* L-BFGS vector updates and scalar kernels */
  BL_KC_GRAM = 6,       /* tall-skinny Gram matrices */
  BL_KC_GEMM = 7,       /* tall-skinny basis products */
  BL_KC_DENSE = 8,      /* small FP64 eigen / Cholesky problems */
  BL_KC_OTHER = 9,      /* reductions, fields, copies */
  BL_KC_KRYLOV_VEC = 10,/* recycled-CG vector passes (dot products, updates), bytes counted */
  BL_KC_COUNT = 11
} bl_kernel_class;
bl_status bl_profile_enable(bl_problem* prob, int32_t enable);
bl_status bl_profile_read(bl_problem* prob, int32_t kernel_class, double* total_ms, int64_t* launches,
                          int64_t* pixels);
/* Algorithmic global-memory bytes (each vector read or written once per pass) moved by the kernels of
 * one class since bl_profile_enable, counted by the kernels themselves; 0 for classes that do not
 * count bytes (only BL_KC_KRYLOV_VEC does).  Synchronises the stream. */
bl_status bl_profile_read_bytes(bl_problem* prob, int32_t kernel_class, int64_t* bytes);

const char* bl_last_error(void);

/* J w for one FP32 image without allocating anything (the paper has no counterpart: this is a
 * service for callers that may not allocate device memory, e.g. code running inside a host
 * framework that owns the device heap, or under a no-allocation rule after start-up; such callers
 * cannot create a bl_problem, whose set-up allocates).
 *   xhat, w:  device, height x width FP32, row-major (the point x^ and the vector w);
 *   theta:    device, p = n_filters (filter_size^2 + 1) doubles, layout as for bl_problem;
 *   out:      device, p doubles, receives J w = -(D^2_{theta x} Phi)^T w (the FoE term only,
 *             as in bl_hypergrad);
 *   cuda_stream: the stream all work is enqueued on (asynchronous; no synchronisation).
 * Scratch: a fixed 4 MiB + 32 KiB __device__ array in the library, kept by every GPU that loads
 * it until the process exits.  Limit: ceil(height / 32) * ceil(width / 32) * p <= 524288, else
 * BL_EINVAL (e.g. 1024 x 1024 with p <= 511, 512 x 512 with p <= 2048).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress with that device current);
 * make that first call before any stream capture.  Every call uses the same array and rewrites
 * what it reads, so results never depend on an earlier call, but calls whose GPU work overlaps
 * (unordered streams) race on it: order them on one stream.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  Every argument is validated before the first CUDA call.
 * Returns BL_EINVAL on invalid sizes or options; BL_ECUDA if a launch fails, or if a CUDA error left
 * by earlier work on the calling thread was pending on entry (reported, not cleared; nothing runs). */
bl_status bl_jw_fp32_static(const float* xhat, const float* w, int32_t height, int32_t width,
                            const double* theta, int32_t n_filters, int32_t filter_size, int32_t phi,
                            double phi_eps, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BL_H_ */
