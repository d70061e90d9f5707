// 3D matrix-free Q1 operator, PCG and geometric multigrid kernels,
// templated on the value type.
//
// Operator (Eq. (model), Sec. 2.1, trilinear Q1, kappa constant per element,
// homogeneous Dirichlet). The reference element matrix has the entries
// h/3 (diagonal), 0 (vertices differing in one coordinate), -h/12 (two or
// three coordinates). Node c = (x, y, z) is shared by the 8 elements
// (x-1+a, y-1+b, z-1+c'), a, b, c' in {0, 1}; a neighbour at offset
// d in {-1, 0, 1}^3 shares the elements whose index bit is 1 where d = +1,
// 0 where d = -1 and free where d = 0. Hence the row of A at c has
//   diagonal              h/3 * (sum of the 8 kappa)
//   12 edge neighbours    -h/12 * (sum of the 2 shared kappa)
//   8 corner neighbours   -h/12 * (the 1 shared kappa)
// and no face coupling.
//
// One thread per node, CTA tiles of 32 x 8 nodes in one z-plane; neighbour
// values come through the L1 cache. Fields that the stencil acts on (p = z +
// beta p_old, e = W b, e + P e_c) are first formed by a pointwise pass, so
// every stencil kernel gathers one stored vector. Node arrays carry the boundary nodes
// (always 0). Partials: one per CTA (g.tiles_s per sample).
#include "mlmc_internal.cuh"

namespace mlmc {
namespace {

constexpr int BX = 32, BY = 8;

struct Node3 {
  int i, j, k;
  bool valid, interior;
  int64_t idx;  // (k * N1 + j) * N1 + i
};

__device__ __forceinline__ Node3 node3(int n) {
  Node3 q;
  const int N1 = n + 1;
  const int tx = (N1 + BX - 1) / BX, ty = (N1 + BY - 1) / BY;
  int t = blockIdx.x;
  const int kz = t / (tx * ty);
  t -= kz * tx * ty;
  const int ty_ = t / tx;
  const int tx_ = t - ty_ * tx;
  q.i = tx_ * BX + threadIdx.x;
  q.j = ty_ * BY + threadIdx.y;
  q.k = kz;
  q.valid = q.i <= n && q.j <= n && q.k <= n;
  q.interior = q.i > 0 && q.i < n && q.j > 0 && q.j < n && q.k > 0 && q.k < n;
  q.idx = ((int64_t)q.k * N1 + q.j) * N1 + q.i;
  return q;
}

template <class T>
__device__ __forceinline__ T warp_sum3(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of the CTA (256 threads) into part[b * tiles + blockIdx.x].
__device__ __forceinline__ void cta_partial3(double v, double* __restrict__ part, int64_t tiles) {
  __shared__ double s_w[BY];
  v = warp_sum3(v);
  if (threadIdx.x == 0) s_w[threadIdx.y] = v;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double r = 0.0;
#pragma unroll
    for (int w = 0; w < BY; ++w) r += s_w[w];
    part[(int64_t)blockIdx.y * tiles + blockIdx.x] = r;
  }
}

__device__ __forceinline__ void prof_tick3(const Prof& p) {
  if (p.acc && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(p.acc, p.per_sample);
}

// kappa of the 8 elements around interior node q: kk[c'][b][a].
template <class T>
__device__ __forceinline__ void load_k8(const T* __restrict__ K, int n, const Node3& q, T kk[2][2][2]) {
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const T* r = K + ((int64_t)(q.k - 1 + c) * n + (q.j - 1 + b)) * n + (q.i - 1);
      kk[c][b][0] = __ldg(r);
      kk[c][b][1] = __ldg(r + 1);
    }
}

template <class T>
__device__ __forceinline__ T diag3(const T kk[2][2][2], double h) {
  const T s = ((kk[0][0][0] + kk[0][0][1]) + (kk[0][1][0] + kk[0][1][1])) +
              ((kk[1][0][0] + kk[1][0][1]) + (kk[1][1][0] + kk[1][1][1]));
  return T(h / 3.0) * s;
}

// (A v)(c) given v at the 27 nodes around c (v[dz+1][dy+1][dx+1]).
template <class T>
__device__ __forceinline__ T stencil3(const T kk[2][2][2], const T v[3][3][3], double h) {
  T edges = T(0), corners = T(0);
  // edge neighbours: exactly one zero component; sum kappa over the free axis
#pragma unroll
  for (int dy = -1; dy <= 1; dy += 2)
#pragma unroll
    for (int dx = -1; dx <= 1; dx += 2) {
      const int a = dx > 0, b = dy > 0;
      edges += (kk[0][b][a] + kk[1][b][a]) * v[1][dy + 1][dx + 1];            // dz = 0
    }
#pragma unroll
  for (int dz = -1; dz <= 1; dz += 2)
#pragma unroll
    for (int dx = -1; dx <= 1; dx += 2) {
      const int a = dx > 0, c = dz > 0;
      edges += (kk[c][0][a] + kk[c][1][a]) * v[dz + 1][1][dx + 1];            // dy = 0
    }
#pragma unroll
  for (int dz = -1; dz <= 1; dz += 2)
#pragma unroll
    for (int dy = -1; dy <= 1; dy += 2) {
      const int b = dy > 0, c = dz > 0;
      edges += (kk[c][b][0] + kk[c][b][1]) * v[dz + 1][dy + 1][1];            // dx = 0
    }
#pragma unroll
  for (int dz = -1; dz <= 1; dz += 2)
#pragma unroll
    for (int dy = -1; dy <= 1; dy += 2)
#pragma unroll
      for (int dx = -1; dx <= 1; dx += 2)
        corners += kk[dz > 0][dy > 0][dx > 0] * v[dz + 1][dy + 1][dx + 1];
  return diag3(kk, h) * v[1][1][1] - T(h / 12.0) * (edges + corners);
}

template <class T, class F>
__device__ __forceinline__ void gather27(const Node3& q, int n, F&& f, T v[3][3][3]) {
  const int64_t N1 = n + 1, P = N1 * N1;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx)
        v[dz + 1][dy + 1][dx + 1] = f(q.idx + dz * P + dy * N1 + dx, q.i + dx, q.j + dy, q.k + dz);
}

template <class T>
__global__ void __launch_bounds__(256) k_apply3(Grid g, const T* __restrict__ K,
                                                const T* __restrict__ X, T* __restrict__ Y, Prof prof) {
  const int64_t b = blockIdx.y;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  T y = T(0);
  if (q.interior) {
    const T* x = X + b * g.ns;
    const int n = g.n;
    T v[3][3][3], kk[2][2][2];
    // the caller's x may carry boundary values: they are ignored
    gather27<T>(q, n, [&](int64_t o, int i, int j, int k) {
      return (i > 0 && i < n && j > 0 && j < n && k > 0 && k < n) ? __ldg(x + o) : T(0);
    }, v);
    load_k8(K + b * g.es, n, q, kk);
    y = stencil3(kk, v, g.h);
  }
  Y[b * g.ns + q.idx] = y;
  prof_tick3(prof);
}

template <class T>
__global__ void __launch_bounds__(256) k_winv3(Grid g, const T* __restrict__ K, double omega,
                                               T* __restrict__ W) {
  const int64_t b = blockIdx.y;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  T w = T(0);
  if (q.interior) {
    T kk[2][2][2];
    load_k8(K + b * g.es, g.n, q, kk);
    w = T(omega) / diag3(kk, g.h);
  }
  W[b * g.ns + q.idx] = w;
}

template <class T>
__global__ void __launch_bounds__(256) k_init3(Grid g, T* __restrict__ X, T* __restrict__ R, Prof prof) {
  const int64_t b = blockIdx.y;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  X[b * g.ns + q.idx] = T(0);
  if (R) R[b * g.ns + q.idx] = q.interior ? T(g.h * g.h * g.h) : T(0);
  prof_tick3(prof);
}

// Pointwise: p_new = z + beta p_old (beta == 0: p_new = z; p_old unread).
template <class T>
__global__ void __launch_bounds__(256) k_pupd3(Grid g, const T* __restrict__ Z, const T* __restrict__ Pold,
                                               T* __restrict__ Pnew, const double* __restrict__ beta,
                                               const int32_t* __restrict__ active) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  const T bb = (T)beta[b];
  const int64_t o = b * g.ns + q.idx;
  const T zv = Z[o];
  Pnew[o] = (bb == T(0)) ? zv : fma(bb, Pold[o], zv);
}

// q = A p, partials of p.q
template <class T>
__global__ void __launch_bounds__(256) k_aq3(Grid g, const T* __restrict__ K, const T* __restrict__ P,
                                             T* __restrict__ Q, const int32_t* __restrict__ active,
                                             double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  const T* p = P + b * g.ns;
  double dot = 0.0;
  if (q.valid) {
    T qv = T(0);
    if (q.interior) {
      T v[3][3][3], kk[2][2][2];
      gather27<T>(q, g.n, [&](int64_t o, int, int, int) { return __ldg(p + o); }, v);
      load_k8(K + b * g.es, g.n, q, kk);
      qv = stencil3(kk, v, g.h);
      dot = (double)(v[1][1][1] * qv);
    }
    Q[b * g.ns + q.idx] = qv;
  }
  cta_partial3(dot, part, g.tiles_s);
  prof_tick3(prof);
}

// Pointwise: out = W b (the pre-smoothing step from zero).
template <class T>
__global__ void __launch_bounds__(256) k_wb3(Grid g, const T* __restrict__ W, const T* __restrict__ Bv,
                                             T* __restrict__ E, const int32_t* __restrict__ active) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  const int64_t o = b * g.ns + q.idx;
  E[o] = W[o] * Bv[o];
}

// r1 = b - A e
template <class T>
__global__ void __launch_bounds__(256) k_mgres3(Grid g, const T* __restrict__ K, const T* __restrict__ Bv,
                                                const T* __restrict__ E, T* __restrict__ R1,
                                                const int32_t* __restrict__ active, Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  const T* e = E + b * g.ns;
  T rv = T(0);
  if (q.interior) {
    T v[3][3][3], kk[2][2][2];
    gather27<T>(q, g.n, [&](int64_t o, int, int, int) { return __ldg(e + o); }, v);
    load_k8(K + b * g.es, g.n, q, kk);
    rv = __ldg(Bv + b * g.ns + q.idx) - stencil3(kk, v, g.h);
  }
  R1[b * g.ns + q.idx] = rv;
  prof_tick3(prof);
}

// Full weighting: bc(I) = sum_{d in {-1,0,1}^3} w(dx) w(dy) w(dz) r1(2I + d).
template <class T>
__global__ void __launch_bounds__(256) k_restrict3(Grid gc, int64_t nsf, const T* __restrict__ R1,
                                                   T* __restrict__ Bc, const int32_t* __restrict__ active,
                                                   Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(gc.n);
  if (!q.valid) return;
  T v = T(0);
  if (q.interior) {
    const int64_t N1 = 2 * gc.n + 1, P = N1 * N1;
    const T* r = R1 + b * nsf + ((int64_t)(2 * q.k) * N1 + 2 * q.j) * N1 + 2 * q.i;
    const T wt[3] = {T(0.5), T(1), T(0.5)};
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      T pl = T(0);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const T* rr = r + dz * P + dy * N1;
        const T row = T(0.5) * __ldg(rr - 1) + __ldg(rr) + T(0.5) * __ldg(rr + 1);
        pl += wt[dy + 1] * row;
      }
      v += wt[dz + 1] * pl;
    }
  }
  Bc[b * gc.ns + q.idx] = v;
  prof_tick3(prof);
}

// Coarsest grid (n = 2, one unknown at (1,1,1)): e = b / D exactly.
template <class T>
__global__ void k_coarse3(Grid g, const T* __restrict__ K, const T* __restrict__ Bv, T* __restrict__ E,
                          const int32_t* __restrict__ active, int64_t B) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  const T* k = K + b * g.es;
  T s = T(0);
  for (int e = 0; e < 8; ++e) s += k[e];
  const T d = T(g.h / 3.0) * s;
  for (int t = 0; t < 27; ++t) E[b * g.ns + t] = T(0);
  E[b * g.ns + 13] = Bv[b * g.ns + 13] / d;
}

// Trilinear prolongation of the coarse correction at fine node (i, j, k).
template <class T>
__device__ __forceinline__ T prolong3(const T* __restrict__ Ec, int nc, int i, int j, int k) {
  const int64_t N1 = nc + 1;
  const int I = i >> 1, J = j >> 1, Kc = k >> 1;
  const int ox = i & 1, oy = j & 1, oz = k & 1;
  T acc = T(0);
  for (int c = 0; c <= oz; ++c)
    for (int bq = 0; bq <= oy; ++bq)
      for (int a = 0; a <= ox; ++a) acc += __ldg(Ec + ((int64_t)(Kc + c) * N1 + (J + bq)) * N1 + (I + a));
  const T scale = T(1) / T(1 << (ox + oy + oz));
  return acc * scale;
}

// Pointwise: tmp = e + P ec (trilinear prolongation of the coarse correction).
template <class T>
__global__ void __launch_bounds__(256) k_prolong3(Grid g, int64_t nsc, const T* __restrict__ E,
                                                  const T* __restrict__ Ec, T* __restrict__ Tmp,
                                                  const int32_t* __restrict__ active) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  if (!q.valid) return;
  T v = T(0);
  if (q.interior) v = E[b * g.ns + q.idx] + prolong3(Ec + b * nsc, g.n / 2, q.i, q.j, q.k);
  Tmp[b * g.ns + q.idx] = v;
}

// out = e' + W (b - A e') with e' = tmp; partials of b.out when part != nullptr.
template <class T>
__global__ void __launch_bounds__(256) k_mgpost3(Grid g, const T* __restrict__ K,
                                                 const T* __restrict__ W, const T* __restrict__ Bv,
                                                 const T* __restrict__ Tmp, T* __restrict__ Out,
                                                 const int32_t* __restrict__ active,
                                                 double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  const T* e = Tmp + b * g.ns;
  double dot = 0.0;
  if (q.valid) {
    T ov = T(0);
    if (q.interior) {
      T v[3][3][3], kk[2][2][2];
      gather27<T>(q, g.n, [&](int64_t o, int, int, int) { return __ldg(e + o); }, v);
      load_k8(K + b * g.es, g.n, q, kk);
      const T bval = __ldg(Bv + b * g.ns + q.idx);
      ov = fma(__ldg(W + b * g.ns + q.idx), bval - stencil3(kk, v, g.h), v[1][1][1]);
      dot = (double)(bval * ov);
    }
    Out[b * g.ns + q.idx] = ov;
  }
  if (part) cta_partial3(dot, part, g.tiles_s);
  prof_tick3(prof);
}

// QoI partials: domain: w = h^3 at interior nodes; box [L, H]^3 in node
// indices: w = h^3 chi_x chi_y chi_z / |box|, chi = 1 inside, 1/2 on a face.
template <class T>
__global__ void __launch_bounds__(256) k_qoi3(Grid g, int box, int L, int H, double inv_vol,
                                              const T* __restrict__ X, double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  const Node3 q = node3(g.n);
  double v = 0.0;
  if (q.valid && q.interior) {
    double w = g.h * g.h * g.h;
    if (box) {
      auto chi = [&](int c) { return (c > L && c < H) ? 1.0 : ((c == L || c == H) ? 0.5 : 0.0); };
      w *= chi(q.i) * chi(q.j) * chi(q.k) * inv_vol;
    }
    v = w * (double)X[b * g.ns + q.idx];
  }
  cta_partial3(v, part, g.tiles_s);
  prof_tick3(prof);
}

// Mixed form, outer FP64 residual r = b - A u (b_i = h^3), partials of r.r.
__global__ void __launch_bounds__(256) k_resid3(Grid g, const double* __restrict__ K,
                                                const double* __restrict__ U, double* __restrict__ R,
                                                const int32_t* __restrict__ active,
                                                double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const Node3 q = node3(g.n);
  const double* u = U + b * g.ns;
  double dot = 0.0;
  if (q.valid) {
    double rv = 0.0;
    if (q.interior) {
      double v[3][3][3], kk[2][2][2];
      gather27<double>(q, g.n, [&](int64_t o, int, int, int) { return __ldg(u + o); }, v);
      load_k8(K + b * g.es, g.n, q, kk);
      rv = g.h * g.h * g.h - stencil3(kk, v, g.h);
      dot = rv * rv;
    }
    R[b * g.ns + q.idx] = rv;
  }
  cta_partial3(dot, part, g.tiles_s);
  prof_tick3(prof);
}

inline dim3 grid3(const Grid& g, int64_t B) { return dim3((unsigned)g.sx, (unsigned)B, 1); }
inline dim3 block3() { return dim3(BX, BY, 1); }

}  // namespace

namespace d3 {

template <class T>
cudaError_t apply(cudaStream_t s, const Grid& g, const T* kappa, const T* x, T* y, int64_t B, Prof p) {
  k_apply3<T><<<grid3(g, B), block3(), 0, s>>>(g, kappa, x, y, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t winv(cudaStream_t s, const Grid& g, const T* kappa, double omega, T* w, int64_t B) {
  k_winv3<T><<<grid3(g, B), block3(), 0, s>>>(g, kappa, omega, w);
  return cudaGetLastError();
}
template <class T>
cudaError_t pcg_init(cudaStream_t s, const Grid& g, T* x, T* r, int64_t B, Prof p) {
  k_init3<T><<<grid3(g, B), block3(), 0, s>>>(g, x, r, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const T* kappa, const T* z, const T* p_old, T* p_new,
                   T* q, const Scalars& sc, double* part, int64_t B, Prof p) {
  k_pupd3<T><<<grid3(g, B), block3(), 0, s>>>(g, z, p_old, p_new, sc.beta, sc.active);
  k_aq3<T><<<grid3(g, B), block3(), 0, s>>>(g, kappa, p_new, q, sc.active, part, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t mg_pre(cudaStream_t s, const Grid& g, const T* kappa, const T* w, const T* b, T* e, T* r1,
                   const int32_t* active, int64_t B, Prof p) {
  k_wb3<T><<<grid3(g, B), block3(), 0, s>>>(g, w, b, e, active);
  k_mgres3<T><<<grid3(g, B), block3(), 0, s>>>(g, kappa, b, e, r1, active, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const T* r1, T* bc,
                      const int32_t* active, int64_t B, Prof p) {
  k_restrict3<T><<<grid3(coarse, B), block3(), 0, s>>>(coarse, fine.ns, r1, bc, active, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const T* kappa, const T* b, T* e,
                         const int32_t* active, int64_t B) {
  k_coarse3<T><<<(unsigned)((B + 127) / 128), 128, 0, s>>>(g, kappa, b, e, active, B);
  return cudaGetLastError();
}
template <class T>
cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const T* kappa, const T* w,
                    const T* b, const T* e, const T* ec, T* out, T* tmp, const int32_t* active,
                    double* part, int64_t B, Prof p) {
  k_prolong3<T><<<grid3(g, B), block3(), 0, s>>>(g, coarse.ns, e, ec, tmp, active);
  k_mgpost3<T><<<grid3(g, B), block3(), 0, s>>>(g, kappa, w, b, tmp, out, active, part, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol, const T* x,
                double* part, int64_t B, Prof p) {
  k_qoi3<T><<<grid3(g, B), block3(), 0, s>>>(g, box, L, H, inv_vol, x, part, p);
  return cudaGetLastError();
}
cudaError_t resid64(cudaStream_t s, const Grid& g, const double* kappa, const double* u, double* r,
                    const int32_t* active, double* part, int64_t B, Prof p) {
  k_resid3<<<grid3(g, B), block3(), 0, s>>>(g, kappa, u, r, active, part, p);
  return cudaGetLastError();
}

#define MLMC_INST3(T)                                                                              \
  template cudaError_t apply<T>(cudaStream_t, const Grid&, const T*, const T*, T*, int64_t, Prof); \
  template cudaError_t winv<T>(cudaStream_t, const Grid&, const T*, double, T*, int64_t);          \
  template cudaError_t pcg_init<T>(cudaStream_t, const Grid&, T*, T*, int64_t, Prof);              \
  template cudaError_t pcg_pq<T>(cudaStream_t, const Grid&, const T*, const T*, const T*, T*, T*,  \
                                 const Scalars&, double*, int64_t, Prof);                          \
  template cudaError_t mg_pre<T>(cudaStream_t, const Grid&, const T*, const T*, const T*, T*, T*,  \
                                 const int32_t*, int64_t, Prof);                                   \
  template cudaError_t restrict_<T>(cudaStream_t, const Grid&, const Grid&, const T*, T*,          \
                                    const int32_t*, int64_t, Prof);                                \
  template cudaError_t coarse_solve<T>(cudaStream_t, const Grid&, const T*, const T*, T*,          \
                                       const int32_t*, int64_t);                                   \
  template cudaError_t mg_post<T>(cudaStream_t, const Grid&, const Grid&, const T*, const T*,      \
                                  const T*, const T*, const T*, T*, T*, const int32_t*, double*,   \
                                  int64_t, Prof);                                                  \
  template cudaError_t qoi<T>(cudaStream_t, const Grid&, int, int, int, double, const T*, double*, \
                              int64_t, Prof);

MLMC_INST3(double)
MLMC_INST3(float)

}  // namespace d3
}  // namespace mlmc
