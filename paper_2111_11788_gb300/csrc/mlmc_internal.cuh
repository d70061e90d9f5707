// Internal declarations of libmlmc (device kernels + host launchers).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>

#include "../../include/mlmc.h"

namespace mlmc {

// 2D stencil kernels: CTAs of SWARPS warps, each warp a strip of 30 output
// columns streamed over SROWS rows.
constexpr int SWARPS = 4;
constexpr int SROWS = 32;
// Flat (pointwise) kernels: FLAT_THREADS threads per CTA, FLAT_ELEMS
// elements of one sample per CTA.
constexpr int FLAT_THREADS = 256;
constexpr int FLAT_ELEMS = 4096;
// KLE kernel tiles.
constexpr int TX2 = 32;
constexpr int TY2 = 8;
// 3D tiles: 32 x 4 x 2 threads.
constexpr int TX3 = 32;
constexpr int TY3 = 4;
constexpr int TZ3 = 2;

constexpr int MAX_MODES_1D = 32;

// Kernel identifiers for tracing (mlmc_kernel_stats).
enum KernelId {
  KID_XI = 0,
  KID_TABLE,
  KID_KAPPA,
  KID_COARSEN,
  KID_APPLY,
  KID_PCG_INIT,
  KID_PCG_PQ,
  KID_PCG_XR,
  KID_JACOBI_Z,
  KID_MG_PRE,
  KID_RESTRICT,
  KID_COARSE,
  KID_MG_POST,
  KID_QOI,
  KID_FINALIZE,
  KID_WELFORD,
  KID_ESTIMATE,
  KID_COUNT,
  KID_SETUP,
  KID_REFINE,
  KID_RESID64,
  KID_MG_BOTTOM,
  NUM_KERNELS
};

// Optional per-launch accounting of algorithmic bytes for active samples.
struct Prof {
  double* acc;         // device accumulator (nullptr = off)
  double per_sample;   // algorithmic DRAM bytes per processed sample
};

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

inline int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Geometry of one (multigrid) grid level and its launch shapes.
struct Grid {
  int dim;
  int n;            // cells per side
  int64_t ns;       // node stride (values per sample)
  int64_t es;       // element stride
  double h;
  double c3, c12;   // h / 3 and h / 12 (3D stencil coefficients), computed on the host
  int sx, sy;       // 2D: stencil CTAs per sample (strip groups x row chunks);
                    // 3D: node-tile CTAs per sample of the pointwise kernels (sx)
  int zc;           // 3D: z-planes per CTA of the z-marching stencil kernels
  int zt;           // 3D FP32 z-march tiles: 0 = full width by TMA where possible, 1 = 32 x 16
  int zx;           // 3D: z-marching CTAs per sample
  int64_t tiles_s;  // partials per sample written by stencil kernels
  int fx;           // flat CTAs per sample
  int64_t tiles_f;  // partials per sample written by flat kernels (one per CTA)
  int64_t tiles_q;  // partials per sample written by the QoI kernel
  int64_t tiles() const {
    int64_t t = tiles_s > tiles_f ? tiles_s : tiles_f;
    return t > tiles_q ? t : tiles_q;
  }
};

Grid make_grid(int dim, int n, int z_chunk = 0, int stencil_tile = 0);

// Runs set() once per device of this process (function attributes such as
// the shared-memory opt-in are per device); device ids below 64.
template <class F>
inline cudaError_t once_per_device(std::atomic<uint64_t>& done, F&& set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// The small multigrid levels k0 .. K-1 of a V-cycle fused into one kernel,
// one CTA per sample in shared memory: from b at level k0 (restricted by the
// level above) to the post-smoothed correction out at level k0. Per level:
// the grid, kappa, W and (2D FP64: non-null) operator coefficients; sample
// strides as in the unfused kernels.
constexpr int MAX_BOTTOM = 8;
template <class T>
struct BottomLevels {
  int L;                       // fused levels (the last is the coarsest, n = 2)
  Grid g[MAX_BOTTOM];
  const T* kap[MAX_BOTTOM];
  const T* coef[MAX_BOTTOM];
  const T* w[MAX_BOTTOM];
};
// largest grid (cells per side) whose level is fused: 2D, 3D
constexpr int BOTTOM_MAX_N2 = 64;
constexpr int BOTTOM_MAX_N3 = 16;

// Per-sample scalars of the batched PCG (struct of arrays, B entries each).
struct Scalars {
  double* gamma;
  double* delta;
  double* alpha;
  double* beta;
  double* rho;
  double* tol;      // rtol * ||b||
  int32_t* active;
  int32_t* iters;
  double* scale;    // mixed form: scale of the inner right-hand side (outer scalars only)
  int32_t* total;   // mixed form: inner iterations so far (outer scalars only)
};

enum FinMode { FIN_GAMMA0 = 0, FIN_ALPHA = 1, FIN_CONV = 2, FIN_BETA = 3, FIN_QOI = 4 };

// Mixed form: close one outer refinement step. With rho = ||r|| from the
// partials: converged (rho <= tol) -> inactive, iters = total inner iterations;
// outer_it == outer_max -> inactive, iters = -1; else scale = rho. Inner
// iterations (inner.iters, -1 = hit inner max) are added to the total.
cudaError_t launch_outer_step(cudaStream_t s, const double* part, int64_t tiles,
                              const Scalars& outer, const int32_t* inner_iters, int inner_max,
                              int outer_it, int outer_max, int64_t B,
                              const int32_t* outer_it_dev = nullptr);
// inner.active = outer.active, inner.tol = tol, inner.iters = 0, beta = 0.
cudaError_t launch_inner_init(cudaStream_t s, const Scalars& inner, const Scalars& outer,
                              double tol, int64_t B);

// ---- launchers (return cudaGetLastError()) -----------------------------

cudaError_t launch_draw_xi(cudaStream_t s, uint64_t seed, uint32_t stream_id, int level,
                           int64_t first, int64_t count, int n_modes, double* xi, Prof p);

cudaError_t launch_kle_table(cudaStream_t s, int n, int m, const double* omega,
                             const double* theta, const int32_t* even, double* table);

cudaError_t launch_kappa(cudaStream_t s, const Grid& g, int m, double sqrt_sigma2,
                         const double* table, const double* xi, int M_xi, const int32_t* slot,
                         int64_t B, double* kappa, Prof p);

template <class T>
cudaError_t launch_coarsen(cudaStream_t s, const Grid& fine, const Grid& coarse,
                           const T* kf, T* kc, int64_t B, Prof p);

// kappa32 = (float) kappa64, element arrays.
// the table of the FP64 exp of the kappa kernels, once per device (before any capture)
cudaError_t init_kle_exp();
// kappa32 = exp(Phi xi) on the tensor cores (split BF16, FP32 accumulation); M kept modes
cudaError_t launch_kappa32_tc(cudaStream_t s, const Grid& g, int m, double sqrt_sigma2, const double* table,
                              const double* xi, int M, const int32_t* slot, int64_t B, float* kappa32);
// bounded waits of the tensor-core KLE kernel that gave up since the last call (resets the count)
cudaError_t take_tc_timeouts(cudaStream_t s, unsigned* out);
cudaError_t launch_cast_kappa(cudaStream_t s, const Grid& g, const double* k64, float* k32,
                              int64_t B);

// 2D operator / PCG / multigrid kernels (stencil2d.cu), T = double or float.
namespace d2 {
template <class T>
cudaError_t apply(cudaStream_t s, const Grid& g, const T* kappa, const T* x, T* y, int64_t B, Prof p);
template <class T>
cudaError_t winv(cudaStream_t s, const Grid& g, const T* kappa, double omega, T* w, int64_t B);
// x = 0; if r != nullptr, r = b (b_i = h^2 at interior nodes).
template <class T>
cudaError_t pcg_init(cudaStream_t s, const Grid& g, T* x, T* r, int64_t B, Prof p);
// x = 0 at every node of B samples, 2D or 3D (flat 16-byte stores).
template <class T>
cudaError_t zero_nodes(cudaStream_t s, const Grid& g, T* x, int64_t B, Prof p);
// coef (may be null): the FP64 form's precomputed operator coefficients
// (coef()), used instead of kappa by the stencil kernels
template <class T>
cudaError_t coef(cudaStream_t s, const Grid& g, const T* kappa, T* coef, int64_t B,
                 double omega = 0.0, T* w = nullptr);
template <class T>
cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const T* kappa, const T* z, const T* p_old,
                   T* p_new, T* q, const Scalars& sc, double* part, int64_t B, Prof p, const T* coef);
template <class T>
cudaError_t pcg_xr(cudaStream_t s, const Grid& g, T* x, const T* pv, T* r, const T* q,
                   const Scalars& sc, double* part, int64_t B, Prof p);
template <class T>
cudaError_t jacobi_z(cudaStream_t s, const Grid& g, const T* winv, const T* r, T* z,
                     const Scalars& sc, double* part, int64_t B, Prof p);
template <class T>
cudaError_t mg_pre(cudaStream_t s, const Grid& g, const T* kappa, const T* w, const T* b, T* e,
                   T* r1, const int32_t* active, int64_t B, Prof p, const T* coef);
template <class T>
cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const T* r1, T* bc,
                      const int32_t* active, int64_t B, Prof p);
template <class T>
cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const T* kappa, const T* b, T* e,
                         const int32_t* active, int64_t B);
template <class T>
cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const T* kappa, const T* w,
                    const T* b, const T* e, const T* ec, T* out, const int32_t* active,
                    double* part, int64_t B, Prof p, const T* coef);
template <class T>
cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol, const T* x,
                double* part, int64_t B, Prof p);
// mixed form (FP64 outer refinement around the FP32 inner solve)
cudaError_t resid64(cudaStream_t s, const Grid& g, const double* kappa, const double* u,
                    double* r, const int32_t* active, double* part, int64_t B, Prof p,
                    const double* coef);
cudaError_t to_rhs32(cudaStream_t s, const Grid& g, const double* r, const double* scale,
                     float* r32, const int32_t* active, int64_t B, Prof p);
cudaError_t add_correction(cudaStream_t s, const Grid& g, double* u, const float* d32,
                           const double* scale, const int32_t* active, int64_t B, Prof p);
// nested initial guess: x = P uc (bilinear interpolation from grid `coarse`)
cudaError_t prolong_guess(cudaStream_t s, const Grid& g, const Grid& coarse, const double* uc,
                          double* x, const int32_t* active, int64_t B, Prof p);

template <class T>
cudaError_t mg_bottom(cudaStream_t s, const BottomLevels<T>& lv, const T* b, T* out,
                      const int32_t* active, int64_t B, Prof p);
}  // namespace d2

// iter_dev (may be null) overrides iter with a device-side iteration counter.
// 3D operator / PCG / multigrid kernels (stencil3d.cu); the pointwise PCG
// kernels (pcg_xr, jacobi_z, to_rhs32, add_correction) are the flat d2 ones.
namespace d3 {
template <class T>
cudaError_t apply(cudaStream_t s, const Grid& g, const T* kappa, const T* x, T* y, int64_t B, Prof p);
template <class T>
cudaError_t winv(cudaStream_t s, const Grid& g, const T* kappa, double omega, T* w, int64_t B);
template <class T>
cudaError_t pcg_init(cudaStream_t s, const Grid& g, T* x, T* r, int64_t B, Prof p);
// ks (FP64 only, may be null): the kappa sums of ksum(); with them the
// z-march runs on element sums (k_zm3q)
template <class T>
cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const T* kappa, const T* z, const T* p_old,
                   T* p_new, T* q, const Scalars& sc, double* part, int64_t B, Prof p, const T* ks);
template <class T>
cudaError_t mg_pre(cudaStream_t s, const Grid& g, const T* kappa, const T* w, const T* b, T* e,
                   T* r1, const int32_t* active, int64_t B, Prof p, const T* ks);
template <class T>
cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const T* r1, T* bc,
                      const int32_t* active, int64_t B, Prof p);
template <class T>
cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const T* kappa, const T* b, T* e,
                         const int32_t* active, int64_t B);
// tmp: a node vector of this level used for e + P ec
template <class T>
cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const T* kappa, const T* w,
                    const T* b, const T* e, const T* ec, T* out, T* tmp, const int32_t* active,
                    double* part, int64_t B, Prof p, const T* ks);
template <class T>
cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol, const T* x,
                double* part, int64_t B, Prof p);
// ks (may be null): the kappa sums of ksum(); with them the residual runs
// the element-sum z-march (k_zm3q)
cudaError_t resid64(cudaStream_t s, const Grid& g, const double* kappa, const double* u,
                    double* r, const int32_t* active, double* part, int64_t B, Prof p,
                    const double* ks = nullptr);
// Per-node kappa sums [K_n | K_x | K_y | K_z] (4 node arrays per sample,
// sample stride 4 ns) for the FP64 element-sum z-march.
cudaError_t ksum(cudaStream_t s, const Grid& g, const double* kappa, double* ks, int64_t B);
// nested initial guess: x = P uc (trilinear interpolation from grid `coarse`)
cudaError_t prolong_guess(cudaStream_t s, const Grid& g, const Grid& coarse, const double* uc,
                          double* x, const int32_t* active, int64_t B, Prof p);
template <class T>
cudaError_t mg_bottom(cudaStream_t s, const BottomLevels<T>& lv, const T* b, T* out,
                      const int32_t* active, int64_t B, Prof p);
// bounded waits of the FP32 z-march that gave up (a copy never landed) since
// the last call on this device; resets the count
cudaError_t take_wait_timeouts(cudaStream_t s, unsigned* out);
}  // namespace d3

// Dimension dispatch used by the plan.
namespace op {
template <class T>
inline cudaError_t apply(cudaStream_t s, const Grid& g, const T* kappa, const T* x, T* y, int64_t B, Prof p) {
  return g.dim == 2 ? d2::apply<T>(s, g, kappa, x, y, B, p) : d3::apply<T>(s, g, kappa, x, y, B, p);
}
template <class T>
inline cudaError_t winv(cudaStream_t s, const Grid& g, const T* kappa, double omega, T* w, int64_t B) {
  return g.dim == 2 ? d2::winv<T>(s, g, kappa, omega, w, B) : d3::winv<T>(s, g, kappa, omega, w, B);
}
template <class T>
inline cudaError_t pcg_init(cudaStream_t s, const Grid& g, T* x, T* r, int64_t B, Prof p) {
  return g.dim == 2 ? d2::pcg_init<T>(s, g, x, r, B, p) : d3::pcg_init<T>(s, g, x, r, B, p);
}
template <class T>
inline cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const T* kappa, const T* z, const T* p_old,
                          T* p_new, T* q, const Scalars& sc, double* part, int64_t B, Prof p,
                          const T* coef = nullptr) {
  return g.dim == 2 ? d2::pcg_pq<T>(s, g, kappa, z, p_old, p_new, q, sc, part, B, p, coef)
                    : d3::pcg_pq<T>(s, g, kappa, z, p_old, p_new, q, sc, part, B, p, coef);
}
template <class T>
inline cudaError_t pcg_xr(cudaStream_t s, const Grid& g, T* x, const T* pv, T* r, const T* q,
                          const Scalars& sc, double* part, int64_t B, Prof p) {
  return d2::pcg_xr<T>(s, g, x, pv, r, q, sc, part, B, p);
}
template <class T>
inline cudaError_t jacobi_z(cudaStream_t s, const Grid& g, const T* winv, const T* r, T* z,
                            const Scalars& sc, double* part, int64_t B, Prof p) {
  return d2::jacobi_z<T>(s, g, winv, r, z, sc, part, B, p);
}
template <class T>
inline cudaError_t mg_pre(cudaStream_t s, const Grid& g, const T* kappa, const T* w, const T* b, T* e,
                          T* r1, const int32_t* active, int64_t B, Prof p, const T* coef = nullptr) {
  return g.dim == 2 ? d2::mg_pre<T>(s, g, kappa, w, b, e, r1, active, B, p, coef)
                    : d3::mg_pre<T>(s, g, kappa, w, b, e, r1, active, B, p, coef);
}
template <class T>
inline cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const T* r1, T* bc,
                             const int32_t* active, int64_t B, Prof p) {
  return fine.dim == 2 ? d2::restrict_<T>(s, fine, coarse, r1, bc, active, B, p)
                       : d3::restrict_<T>(s, fine, coarse, r1, bc, active, B, p);
}
template <class T>
inline cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const T* kappa, const T* b, T* e,
                                const int32_t* active, int64_t B) {
  return g.dim == 2 ? d2::coarse_solve<T>(s, g, kappa, b, e, active, B)
                    : d3::coarse_solve<T>(s, g, kappa, b, e, active, B);
}
// tmp: scratch node vector of this level (3D only)
template <class T>
inline cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const T* kappa, const T* w,
                           const T* b, const T* e, const T* ec, T* out, T* tmp, const int32_t* active,
                           double* part, int64_t B, Prof p, const T* coef = nullptr) {
  return g.dim == 2 ? d2::mg_post<T>(s, g, coarse, kappa, w, b, e, ec, out, active, part, B, p, coef)
                    : d3::mg_post<T>(s, g, coarse, kappa, w, b, e, ec, out, tmp, active, part, B, p, coef);
}
template <class T>
inline cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol, const T* x,
                       double* part, int64_t B, Prof p) {
  return g.dim == 2 ? d2::qoi<T>(s, g, box, L, H, inv_vol, x, part, B, p)
                    : d3::qoi<T>(s, g, box, L, H, inv_vol, x, part, B, p);
}
inline cudaError_t resid64(cudaStream_t s, const Grid& g, const double* kappa, const double* u,
                           double* r, const int32_t* active, double* part, int64_t B, Prof p,
                           const double* coef = nullptr) {
  return g.dim == 2 ? d2::resid64(s, g, kappa, u, r, active, part, B, p, coef)
                    : d3::resid64(s, g, kappa, u, r, active, part, B, p, coef);
}
inline cudaError_t to_rhs32(cudaStream_t s, const Grid& g, const double* r, const double* scale,
                            float* r32, const int32_t* active, int64_t B, Prof p) {
  return d2::to_rhs32(s, g, r, scale, r32, active, B, p);
}
inline cudaError_t add_correction(cudaStream_t s, const Grid& g, double* u, const float* d32,
                                  const double* scale, const int32_t* active, int64_t B, Prof p) {
  return d2::add_correction(s, g, u, d32, scale, active, B, p);
}
template <class T>
inline cudaError_t mg_bottom(cudaStream_t s, const BottomLevels<T>& lv, const T* b, T* out,
                             const int32_t* active, int64_t B, Prof p) {
  return lv.g[0].dim == 2 ? d2::mg_bottom<T>(s, lv, b, out, active, B, p)
                          : d3::mg_bottom<T>(s, lv, b, out, active, B, p);
}
inline cudaError_t prolong_guess(cudaStream_t s, const Grid& g, const Grid& coarse, const double* uc,
                                 double* x, const int32_t* active, int64_t B, Prof p) {
  return g.dim == 2 ? d2::prolong_guess(s, g, coarse, uc, x, active, B, p)
                    : d3::prolong_guess(s, g, coarse, uc, x, active, B, p);
}
}  // namespace op

cudaError_t launch_finalize(cudaStream_t s, FinMode mode, const double* part, int64_t tiles,
                            const Scalars& sc, double* out, int iter, int max_iter, int64_t B,
                            const int32_t* iter_dev = nullptr);

// Graph loop control: count = #active; cond = count > 0 && *it_dev < max_iter;
// ++*it_dev; ++*execs (if given).
cudaError_t launch_loop_ctl(cudaStream_t s, const int32_t* active, int64_t B, int32_t* it_dev,
                            int max_iter, int32_t* count, int32_t* execs,
                            cudaGraphConditionalHandle h);
cudaError_t launch_set_int(cudaStream_t s, int32_t* p, int32_t v);
// Sets a graph conditional (re-arms a nested while-node before it is reached).
cudaError_t launch_set_cond(cudaStream_t s, cudaGraphConditionalHandle h, unsigned v);

cudaError_t launch_count_active(cudaStream_t s, const int32_t* active, int64_t B, int32_t* count);

// active = 1, iters = 0, tol = tol, beta = alpha = gamma = 0; total = 0 and
// scale = scale0 when those arrays are present.
cudaError_t launch_scalars_init(cudaStream_t s, const Scalars& sc, double tol, double scale0,
                                int64_t B);

cudaError_t launch_welford(cudaStream_t s, const double* qf, const double* qc, int64_t B,
                           mlmc_level_state* st, double cost);

cudaError_t launch_estimate(cudaStream_t s, const mlmc_level_state* st, int n_levels,
                            const double* cost, double eps, double* out2, int64_t* N);

cudaError_t launch_adapt(cudaStream_t s, const mlmc_level_state* st, int La, int Lmax,
                         const double* cost, double eps, int64_t* N, double* out3);
cudaError_t launch_allocate(cudaStream_t s, const double* V, const double* C, int n_levels,
                            double eps, int64_t* N);

}  // namespace mlmc
