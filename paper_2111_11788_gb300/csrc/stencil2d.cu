// 2D matrix-free Q1 operator, batched PCG vector kernels and geometric
// multigrid kernels (FP64).
//
// Operator (Eq. (model), Sec. 2.1, Q1 on a uniform grid, kappa constant per
// element, homogeneous Dirichlet): at an interior node c with surrounding
// elements SW, SE, NW, NE (kappa values kSW..kNE) the row of A is
//   diagonal          2/3 (kSW + kSE + kNW + kNE)
//   edge neighbours  -1/6 (sum of kappa of the two elements sharing the edge)
//   corner neighbours -1/3 kappa of the one element shared.
// Node arrays carry the boundary nodes (always 0), so no neighbour needs a
// bounds test. One thread per node, CTA tiles of 32 x 8 nodes; per-sample
// reductions go to one partial per (sample, tile), summed in a fixed order.
#include "mlmc_internal.cuh"

namespace mlmc {
namespace {

constexpr double C23 = 2.0 / 3.0;
constexpr double C16 = 1.0 / 6.0;
constexpr double C13 = 1.0 / 3.0;

struct Node2 {
  int i, j;        // node coordinates in 0..n
  bool valid;      // inside the (n+1)^2 node grid
  bool interior;
  int64_t idx;     // j * (n + 1) + i
};

__device__ __forceinline__ Node2 node2(int n, int tiles_x) {
  Node2 q;
  const int t = blockIdx.x;
  const int ty = t / tiles_x;
  const int tx = t - ty * tiles_x;
  q.i = tx * TX2 + threadIdx.x;
  q.j = ty * TY2 + threadIdx.y;
  q.valid = (q.i <= n) && (q.j <= n);
  q.interior = (q.i > 0) && (q.i < n) && (q.j > 0) && (q.j < n);
  q.idx = (int64_t)q.j * (n + 1) + q.i;
  return q;
}

// Sum over the 256 threads of the CTA; result valid in thread (0, 0).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_w[TY2];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) s_w[threadIdx.y] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int w = 0; w < TY2; ++w) r += s_w[w];
  }
  return r;
}

__device__ __forceinline__ void prof_tick(const Prof& p) {
  if (p.acc && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(p.acc, p.per_sample);
}

// kappa of the four elements around interior node (i, j)
struct K4 {
  double sw, se, nw, ne;
};
__device__ __forceinline__ K4 load_k4(const double* __restrict__ K, int n, int i, int j) {
  K4 k;
  const double* r0 = K + (int64_t)(j - 1) * n + (i - 1);
  k.sw = __ldg(r0);
  k.se = __ldg(r0 + 1);
  k.nw = __ldg(r0 + n);
  k.ne = __ldg(r0 + n + 1);
  return k;
}

__device__ __forceinline__ double diag2(const K4& k) { return C23 * ((k.sw + k.se) + (k.nw + k.ne)); }

// (A v)(c) from the 3x3 values v[dj+1][di+1] around c.
__device__ __forceinline__ double stencil2(const K4& k, const double v[3][3]) {
  const double edge = (k.se + k.ne) * v[1][2] + (k.sw + k.nw) * v[1][0] +
                      (k.nw + k.ne) * v[2][1] + (k.sw + k.se) * v[0][1];
  const double corner = k.ne * v[2][2] + k.nw * v[2][0] + k.se * v[0][2] + k.sw * v[0][0];
  return diag2(k) * v[1][1] - C16 * edge - C13 * corner;
}

__device__ __forceinline__ void load9(const double* __restrict__ X, int n, int64_t idx,
                                      double v[3][3]) {
  const int N1 = n + 1;
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di) v[dj + 1][di + 1] = __ldg(X + idx + dj * N1 + di);
}

__global__ void __launch_bounds__(256) k_apply2d(int n, int tiles_x, int64_t ns, int64_t es,
                                                 const double* __restrict__ K,
                                                 const double* __restrict__ X,
                                                 double* __restrict__ Y, Prof prof) {
  const int b = blockIdx.y;
  const Node2 q = node2(n, tiles_x);
  if (!q.valid) return;
  K += (int64_t)b * es;
  X += (int64_t)b * ns;
  double y = 0.0;
  if (q.interior) {
    double v[3][3];
    load9(X, n, q.idx, v);
    y = stencil2(load_k4(K, n, q.i, q.j), v);
  }
  Y[(int64_t)b * ns + q.idx] = y;
  prof_tick(prof);
}

// W = omega / D at interior nodes, 0 on the boundary.
__global__ void __launch_bounds__(256) k_winv2d(int n, int tiles_x, int64_t ns, int64_t es,
                                                const double* __restrict__ K, double omega,
                                                double* __restrict__ W) {
  const int b = blockIdx.y;
  const Node2 q = node2(n, tiles_x);
  if (!q.valid) return;
  double w = 0.0;
  if (q.interior) w = omega / diag2(load_k4(K + (int64_t)b * es, n, q.i, q.j));
  W[(int64_t)b * ns + q.idx] = w;
}

__global__ void __launch_bounds__(256) k_pcg_init2d(int n, int tiles_x, int64_t ns, double h2,
                                                    double* __restrict__ X,
                                                    double* __restrict__ R, Prof prof) {
  const int b = blockIdx.y;
  const Node2 q = node2(n, tiles_x);
  if (!q.valid) return;
  X[(int64_t)b * ns + q.idx] = 0.0;
  R[(int64_t)b * ns + q.idx] = q.interior ? h2 : 0.0;
  prof_tick(prof);
}

// p_new = z + beta p_old (beta == 0: p_new = z), q = A p_new, partial p.q
__global__ void __launch_bounds__(256) k_pq2d(int n, int tiles_x, int64_t ns, int64_t es,
                                              const double* __restrict__ K,
                                              const double* __restrict__ Z,
                                              const double* __restrict__ Pold,
                                              double* __restrict__ Pnew, double* __restrict__ Q,
                                              const double* __restrict__ beta,
                                              const int32_t* __restrict__ active,
                                              double* __restrict__ part, Prof prof) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const Node2 q = node2(n, tiles_x);
  const double bb = beta[b];
  const int64_t off = (int64_t)b * ns;
  double dot = 0.0;
  if (q.valid) {
    double pv = 0.0, qv = 0.0;
    if (q.interior) {
      const int N1 = n + 1;
      double v[3][3];
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const int64_t o = off + q.idx + dj * N1 + di;
          const double zz = __ldg(Z + o);
          v[dj + 1][di + 1] = (bb == 0.0) ? zz : fma(bb, __ldg(Pold + o), zz);
        }
      pv = v[1][1];
      qv = stencil2(load_k4(K + (int64_t)b * es, n, q.i, q.j), v);
      dot = pv * qv;
    }
    Pnew[off + q.idx] = pv;
    Q[off + q.idx] = qv;
  }
  dot = block_sum(dot);
  if (threadIdx.x == 0 && threadIdx.y == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = dot;
  prof_tick(prof);
}

// x += alpha p, r -= alpha q, partial r.r
__global__ void __launch_bounds__(256) k_xr2d(int n, int tiles_x, int64_t ns,
                                              double* __restrict__ X,
                                              const double* __restrict__ P,
                                              double* __restrict__ R,
                                              const double* __restrict__ Q,
                                              const double* __restrict__ alpha,
                                              const int32_t* __restrict__ active,
                                              double* __restrict__ part, Prof prof) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const Node2 q = node2(n, tiles_x);
  const double a = alpha[b];
  double dot = 0.0;
  if (q.valid) {
    const int64_t o = (int64_t)b * ns + q.idx;
    const double xv = fma(a, P[o], X[o]);
    const double rv = fma(-a, Q[o], R[o]);
    X[o] = xv;
    R[o] = rv;
    dot = rv * rv;
  }
  dot = block_sum(dot);
  if (threadIdx.x == 0 && threadIdx.y == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = dot;
  prof_tick(prof);
}

// z = Dinv r, partial r.z
__global__ void __launch_bounds__(256) k_jz2d(int n, int tiles_x, int64_t ns,
                                              const double* __restrict__ Winv,
                                              const double* __restrict__ R,
                                              double* __restrict__ Z,
                                              const int32_t* __restrict__ active,
                                              double* __restrict__ part, Prof prof) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const Node2 q = node2(n, tiles_x);
  double dot = 0.0;
  if (q.valid) {
    const int64_t o = (int64_t)b * ns + q.idx;
    const double rv = R[o];
    const double zv = Winv[o] * rv;
    Z[o] = zv;
    dot = rv * zv;
  }
  dot = block_sum(dot);
  if (threadIdx.x == 0 && threadIdx.y == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = dot;
  prof_tick(prof);
}

// Pre-smoothing from zero and residual: e = W b, r1 = b - A e.
__global__ void __launch_bounds__(256) k_mgpre2d(int n, int tiles_x, int64_t ns, int64_t es,
                                                 const double* __restrict__ K,
                                                 const double* __restrict__ W,
                                                 const double* __restrict__ Bv,
                                                 double* __restrict__ E,
                                                 double* __restrict__ R1,
                                                 const int32_t* __restrict__ active, Prof prof) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const Node2 q = node2(n, tiles_x);
  if (!q.valid) return;
  const int64_t off = (int64_t)b * ns;
  double ev = 0.0, rv = 0.0;
  if (q.interior) {
    const int N1 = n + 1;
    double v[3][3];
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int64_t o = off + q.idx + dj * N1 + di;
        v[dj + 1][di + 1] = __ldg(W + o) * __ldg(Bv + o);   // W = 0 on the boundary
      }
    ev = v[1][1];
    rv = __ldg(Bv + off + q.idx) - stencil2(load_k4(K + (int64_t)b * es, n, q.i, q.j), v);
  }
  E[off + q.idx] = ev;
  R1[off + q.idx] = rv;
  prof_tick(prof);
}

// Full-weighting restriction (transpose of bilinear prolongation):
// bc(I, J) = sum_{di,dj in -1..1} w(di) w(dj) r1(2I + di, 2J + dj), w(0) = 1, w(+-1) = 1/2.
__global__ void __launch_bounds__(256) k_restrict2d(int nc, int tiles_x, int64_t nsf,
                                                    int64_t nsc,
                                                    const double* __restrict__ R1,
                                                    double* __restrict__ Bc,
                                                    const int32_t* __restrict__ active,
                                                    Prof prof) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const Node2 q = node2(nc, tiles_x);
  if (!q.valid) return;
  double v = 0.0;
  if (q.interior) {
    const int nf = 2 * nc;
    const int N1 = nf + 1;
    const double* r = R1 + (int64_t)b * nsf + (int64_t)(2 * q.j) * N1 + 2 * q.i;
    const double rows0 = 0.5 * __ldg(r - N1 - 1) + __ldg(r - N1) + 0.5 * __ldg(r - N1 + 1);
    const double rows1 = 0.5 * __ldg(r - 1) + __ldg(r) + 0.5 * __ldg(r + 1);
    const double rows2 = 0.5 * __ldg(r + N1 - 1) + __ldg(r + N1) + 0.5 * __ldg(r + N1 + 1);
    v = 0.5 * (rows0 + rows2) + rows1;
  }
  Bc[(int64_t)b * nsc + q.idx] = v;
  prof_tick(prof);
}

// Coarsest grid (n = 2, one unknown): e = b / D exactly.
__global__ void k_coarse2d(int64_t ns, int64_t es, const double* __restrict__ K,
                           const double* __restrict__ Bv, double* __restrict__ E,
                           const int32_t* __restrict__ active, int64_t B) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  const int64_t off = b * ns;
  const double* k = K + b * es;
  const double d = C23 * ((k[0] + k[1]) + (k[2] + k[3]));
  for (int t = 0; t < 9; ++t) E[off + t] = 0.0;
  E[off + 4] = Bv[off + 4] / d;
}

// Bilinear prolongation of the coarse correction at fine node (i, j).
__device__ __forceinline__ double prolong2(const double* __restrict__ Ec, int nc, int i, int j) {
  const int N1c = nc + 1;
  const int I = i >> 1, J = j >> 1;
  const double* e = Ec + (int64_t)J * N1c + I;
  const bool ox = i & 1, oy = j & 1;
  double v0 = __ldg(e);
  if (ox) v0 = 0.5 * (v0 + __ldg(e + 1));
  if (!oy) return v0;
  double v1 = __ldg(e + N1c);
  if (ox) v1 = 0.5 * (v1 + __ldg(e + N1c + 1));
  return 0.5 * (v0 + v1);
}

// out = e' + W (b - A e'), e' = e + P ec; partial b.out when part != nullptr.
__global__ void __launch_bounds__(256) k_mgpost2d(int n, int tiles_x, int64_t ns, int64_t es,
                                                  int64_t nsc, const double* __restrict__ K,
                                                  const double* __restrict__ W,
                                                  const double* __restrict__ Bv,
                                                  const double* __restrict__ E,
                                                  const double* __restrict__ Ec,
                                                  double* __restrict__ Out,
                                                  const int32_t* __restrict__ active,
                                                  double* __restrict__ part, Prof prof) {
  const int b = blockIdx.y;
  if (!active[b]) return;
  const Node2 q = node2(n, tiles_x);
  const int64_t off = (int64_t)b * ns;
  const int nc = n / 2;
  const double* ec = Ec + (int64_t)b * nsc;
  double dot = 0.0;
  if (q.valid) {
    double ov = 0.0;
    if (q.interior) {
      const int N1 = n + 1;
      double v[3][3];
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di)
          v[dj + 1][di + 1] =
              __ldg(E + off + q.idx + dj * N1 + di) + prolong2(ec, nc, q.i + di, q.j + dj);
      const double bv = __ldg(Bv + off + q.idx);
      const double av = stencil2(load_k4(K + (int64_t)b * es, n, q.i, q.j), v);
      ov = fma(__ldg(W + off + q.idx), bv - av, v[1][1]);
      dot = bv * ov;
    }
    Out[off + q.idx] = ov;
  }
  if (part) {
    dot = block_sum(dot);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = dot;
  }
  prof_tick(prof);
}

// Per-tile partial sums of w_i x_i for the QoI weights (exact Q1 integral
// mean): domain: w = h^2 at interior nodes; box [lo, hi]^2 (node indices
// L, H): w = h^2 chi_x chi_y / |box|, chi = 1 strictly inside, 1/2 on a face.
__global__ void __launch_bounds__(256) k_qoi2d(int n, int tiles_x, int64_t ns, double h2,
                                               int box, int L, int H, double inv_vol,
                                               const double* __restrict__ X,
                                               double* __restrict__ part, Prof prof) {
  const int b = blockIdx.y;
  const Node2 q = node2(n, tiles_x);
  double v = 0.0;
  if (q.valid && q.interior) {
    double w = h2;
    if (box) {
      const double cx = (q.i > L && q.i < H) ? 1.0 : ((q.i == L || q.i == H) ? 0.5 : 0.0);
      const double cy = (q.j > L && q.j < H) ? 1.0 : ((q.j == L || q.j == H) ? 0.5 : 0.0);
      w = h2 * cx * cy * inv_vol;
    }
    v = w * X[(int64_t)b * ns + q.idx];
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = v;
  prof_tick(prof);
}

inline dim3 grid2(const Grid& g, int64_t B) { return dim3((unsigned)g.tiles(), (unsigned)B, 1); }
inline dim3 block2() { return dim3(TX2, TY2, 1); }

}  // namespace

namespace d2 {

cudaError_t apply(cudaStream_t s, const Grid& g, const double* kappa, const double* x, double* y,
                  int64_t B, Prof p) {
  k_apply2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.es, kappa, x, y, p);
  return cudaGetLastError();
}

cudaError_t winv(cudaStream_t s, const Grid& g, const double* kappa, double omega, double* w,
                 int64_t B) {
  k_winv2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.es, kappa, omega, w);
  return cudaGetLastError();
}

cudaError_t pcg_init(cudaStream_t s, const Grid& g, double* x, double* r, int64_t B, Prof p) {
  k_pcg_init2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.h * g.h, x, r, p);
  return cudaGetLastError();
}

cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const double* kappa, const double* z,
                   const double* p_old, double* p_new, double* q, const Scalars& sc,
                   double* part, int64_t B, Prof p) {
  k_pq2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.es, kappa, z, p_old, p_new, q,
                                          sc.beta, sc.active, part, p);
  return cudaGetLastError();
}

cudaError_t pcg_xr(cudaStream_t s, const Grid& g, double* x, const double* pv, double* r,
                   const double* q, const Scalars& sc, double* part, int64_t B, Prof p) {
  k_xr2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, x, pv, r, q, sc.alpha, sc.active,
                                          part, p);
  return cudaGetLastError();
}

cudaError_t jacobi_z(cudaStream_t s, const Grid& g, const double* winv, const double* r,
                     double* z, const Scalars& sc, double* part, int64_t B, Prof p) {
  k_jz2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, winv, r, z, sc.active, part, p);
  return cudaGetLastError();
}

cudaError_t mg_pre(cudaStream_t s, const Grid& g, const double* kappa, const double* w,
                   const double* b, double* e, double* r1, const int32_t* active, int64_t B,
                   Prof p) {
  k_mgpre2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.es, kappa, w, b, e, r1,
                                             active, p);
  return cudaGetLastError();
}

cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const double* r1,
                      double* bc, const int32_t* active, int64_t B, Prof p) {
  k_restrict2d<<<grid2(coarse, B), block2(), 0, s>>>(coarse.n, coarse.tiles_x, fine.ns, coarse.ns,
                                                     r1, bc, active, p);
  return cudaGetLastError();
}

cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const double* kappa, const double* b,
                         double* e, const int32_t* active, int64_t B) {
  k_coarse2d<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(g.ns, g.es, kappa, b, e, active, B);
  return cudaGetLastError();
}

cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const double* kappa,
                    const double* w, const double* b, const double* e, const double* ec,
                    double* out, const int32_t* active, double* part, int64_t B, Prof p) {
  k_mgpost2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.es, coarse.ns, kappa, w, b,
                                              e, ec, out, active, part, p);
  return cudaGetLastError();
}

cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol,
                const double* x, double* part, int64_t B, Prof p) {
  k_qoi2d<<<grid2(g, B), block2(), 0, s>>>(g.n, g.tiles_x, g.ns, g.h * g.h, box, L, H, inv_vol, x,
                                           part, p);
  return cudaGetLastError();
}

}  // namespace d2
}  // namespace mlmc
