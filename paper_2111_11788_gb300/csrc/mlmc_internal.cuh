// Internal declarations of libmlmc (device kernels + host launchers).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/mlmc.h"

namespace mlmc {

// 2D tiles: 32 x 8 threads, one node per thread.
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

// Geometry of one (multigrid) grid level for a batch.
struct Grid {
  int dim;
  int n;          // cells per side
  int64_t ns;     // node stride (doubles per sample)
  int64_t es;     // element stride
  double h;
  int tiles_x, tiles_y, tiles_z;  // CTA tiles per sample
  int64_t tiles() const { return (int64_t)tiles_x * tiles_y * tiles_z; }
};

Grid make_grid(int dim, int n);

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
};

enum FinMode { FIN_GAMMA0 = 0, FIN_ALPHA = 1, FIN_CONV = 2, FIN_BETA = 3, FIN_QOI = 4 };

// ---- launchers (return cudaGetLastError()) -----------------------------

cudaError_t launch_draw_xi(cudaStream_t s, uint64_t seed, uint32_t stream_id, int level,
                           int64_t first, int64_t count, int n_modes, double* xi, Prof p);

cudaError_t launch_kle_table(cudaStream_t s, int n, int m, const double* omega,
                             const double* theta, const int32_t* even, double* table);

cudaError_t launch_kappa(cudaStream_t s, const Grid& g, int m, double sqrt_sigma2,
                         const double* table, const double* xi, int64_t B, double* kappa, Prof p);

cudaError_t launch_coarsen(cudaStream_t s, const Grid& fine, const Grid& coarse,
                           const double* kf, double* kc, int64_t B, Prof p);

// 2D FP64 operator / PCG / multigrid kernels (stencil2d.cu).
namespace d2 {
cudaError_t apply(cudaStream_t s, const Grid& g, const double* kappa, const double* x, double* y,
                  int64_t B, Prof p);
cudaError_t winv(cudaStream_t s, const Grid& g, const double* kappa, double omega, double* w,
                 int64_t B);
cudaError_t pcg_init(cudaStream_t s, const Grid& g, double* x, double* r, int64_t B, Prof p);
cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const double* kappa, const double* z,
                   const double* p_old, double* p_new, double* q, const Scalars& sc,
                   double* part, int64_t B, Prof p);
cudaError_t pcg_xr(cudaStream_t s, const Grid& g, double* x, const double* pv, double* r,
                   const double* q, const Scalars& sc, double* part, int64_t B, Prof p);
cudaError_t jacobi_z(cudaStream_t s, const Grid& g, const double* winv, const double* r,
                     double* z, const Scalars& sc, double* part, int64_t B, Prof p);
cudaError_t mg_pre(cudaStream_t s, const Grid& g, const double* kappa, const double* w,
                   const double* b, double* e, double* r1, const int32_t* active, int64_t B,
                   Prof p);
cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const double* r1,
                      double* bc, const int32_t* active, int64_t B, Prof p);
cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const double* kappa, const double* b,
                         double* e, const int32_t* active, int64_t B);
cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const double* kappa,
                    const double* w, const double* b, const double* e, const double* ec,
                    double* out, const int32_t* active, double* part, int64_t B, Prof p);
cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol,
                const double* x, double* part, int64_t B, Prof p);
}  // namespace d2

cudaError_t launch_finalize(cudaStream_t s, FinMode mode, const double* part, int64_t tiles,
                            const Scalars& sc, double* out, int iter, int max_iter, int64_t B);

cudaError_t launch_count_active(cudaStream_t s, const int32_t* active, int64_t B, int32_t* count);

cudaError_t launch_scalars_init(cudaStream_t s, const Scalars& sc, double tol, int64_t B);

cudaError_t launch_welford(cudaStream_t s, const double* qf, const double* qc, int64_t B,
                           mlmc_level_state* st, double cost);

cudaError_t launch_estimate(cudaStream_t s, const mlmc_level_state* st, int n_levels,
                            const double* cost, double eps, double* out2, int64_t* N);

cudaError_t launch_allocate(cudaStream_t s, const double* V, const double* C, int n_levels,
                            double eps, int64_t* N);

}  // namespace mlmc
