// Lognormal coefficient kappa = exp(Phi xi) at element centroids.
//
// Phi is the full tensor basis of the 1D exponential-covariance KLE
// eigenfunctions (Sec. 5.2 "eigenfunctions in each dimension"):
//   Phi[e, k] = sqrt(sigma^2) prod_a sqrt(theta_{k_a}) f_{k_a}(c_a(e)),
// k = (k_z m + k_y) m + k_x. Because Phi is a Kronecker product of per-axis
// tables F[i, k] = sqrt(theta_k) f_k((i + 1/2) h), the contraction Phi xi is
// evaluated axis by axis (sum factorisation) in FP64: for each sample a
// small x-contraction into shared memory, then m FMAs per element and one
// exp. On GB300 the FP64 exp and FMAs bound the kernel (about 20 GB/s of
// kappa per TFLOP/s of FP64), not the write of kappa (8 B per element).
#include <algorithm>
#include <cmath>

#include "mlmc_internal.cuh"

namespace mlmc {
namespace {

// exp in FP64 by the table-driven reduction of P. T. P. Tang ("Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989), written from the mathematics:
//   x = (64 k + j) ln2 / 64 + r,  |r| <= ln2 / 128,  0 <= j < 64,
//   exp(x) = 2^k 2^(j/64) exp(r),  exp(r) = 1 + p(r),
//   p(r) = r + r^2 (1/2 + r (1/6 + r (1/24 + r / 120)))
// (the next Taylor term, r^6 / 720, is below 4e-17). ln2 / 64 is split as
// L1 + L2 with L1 carrying 32 significant bits, so N L1 is exact for the
// |N| < 2^21 of |x| < 2^14; 2^(j/64) comes from a table of 64 doubles made on
// the host. About 1 ulp; |x| < 700 (the log-field of the KLE stays far inside).
__constant__ double c_exp2_tab[64];
constexpr double kInvLn2x64 = 92.332482616893658071;   // 64 / ln 2
// ln 2 / 64 = 0.0108304246962491454596... as L1 (32 significant bits) + L2
constexpr double kLn2d64Hi = 0x1.62e42fee00000p-7;     // 0.01083042469326755963265895843505859375
constexpr double kLn2d64Lo = 2.9815858269852934627254151261796896e-12;

__device__ __forceinline__ double kle_exp(double x) {
  const double t = x * kInvLn2x64;
  const double nf = rint(t);
  const int N = (int)nf;
  const double r = fma(-nf, kLn2d64Lo, fma(-nf, kLn2d64Hi, x));
  const int j = N & 63;
  const int k = (N - j) >> 6;
  const double q = fma(r, fma(r, fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5);
  const double p = fma(r * r, q, r);
  const double T = c_exp2_tab[j];
  return fma(T, p, T) * __longlong_as_double((long long)(k + 1023) << 52);
}

// F[i * m + k] = sqrt(theta_k) f_k(x_i), x_i = (i + 1/2) / n, centred t = x - 1/2:
// even k: cos(w t) / sqrt(1/2 + sin(w) / (2w)); odd k: sin(w t) / sqrt(1/2 - sin(w) / (2w)).
__global__ void k_kle_table(int n, int m, const double* __restrict__ omega,
                            const double* __restrict__ theta, const int32_t* __restrict__ even,
                            double* __restrict__ table) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * m) return;
  const int i = idx / m;
  const int k = idx - i * m;
  const double w = omega[k];
  const double t = ((double)i + 0.5) / (double)n - 0.5;
  const double s2 = sin(w) / (2.0 * w);   // sin(2 w a) / (2 w) with a = 1/2
  double f;
  if (even[k]) {
    f = cos(w * t) / sqrt(0.5 + s2);
  } else {
    f = sin(w * t) / sqrt(0.5 - s2);
  }
  table[idx] = sqrt(theta[k]) * f;
}

// Element rows per thread in 2D: a CTA covers 32 columns x 8 * KAP_ROWS rows,
// so the x-contraction of its columns (m^2 FMAs per column) is shared by 64
// rows of elements (m FMAs and one exp each).
constexpr int KAP_ROWS = 8;

// The sample's KLE coefficients in the full tensor layout (m^dim entries) in
// shared memory: a copy, or under total-order truncation the kept
// coefficients scattered to their full-basis slots and zeros elsewhere.
__device__ __forceinline__ void load_coefs(const double* __restrict__ xs, int M_xi,
                                           const int32_t* __restrict__ slot, int M_full,
                                           double* s_xi, int tid, int nthreads) {
  if (!slot) {
    for (int k = tid; k < M_full; k += nthreads) s_xi[k] = xs[k];
    return;
  }
  for (int k = tid; k < M_full; k += nthreads) s_xi[k] = 0.0;
  __syncthreads();
  for (int t = tid; t < M_xi; t += nthreads) s_xi[slot[t]] = xs[t];
}

// 2D: CTA covers 32 x (8 * KAP_ROWS) elements of one sample.
__global__ void __launch_bounds__(TX2* TY2)
    k_kappa2d(int n, int m, double sqrt_sigma2, const double* __restrict__ table,
              const double* __restrict__ xi, int M_xi, const int32_t* __restrict__ slot,
              int64_t es, double* __restrict__ kappa, Prof prof) {
  __shared__ double s_xi[MAX_MODES_1D * MAX_MODES_1D];
  __shared__ double s_t[TX2][MAX_MODES_1D + 1];          // T[ix][k_y]
  __shared__ double s_fy[TY2 * KAP_ROWS][MAX_MODES_1D + 1];
  const int b = blockIdx.z;
  const int tid = threadIdx.y * TX2 + threadIdx.x;
  const int nthreads = TX2 * TY2;
  const int x0 = blockIdx.x * TX2;
  const int y0 = blockIdx.y * TY2 * KAP_ROWS;
  load_coefs(xi + (int64_t)b * M_xi, M_xi, slot, m * m, s_xi, tid, nthreads);
  for (int idx = tid; idx < TY2 * KAP_ROWS * m; idx += nthreads) {
    const int r = idx / m, k = idx - r * m;
    const int iy = y0 + r;
    s_fy[r][k] = (iy < n) ? table[iy * m + k] : 0.0;
  }
  __syncthreads();
  // T[ix][ky] = sum_kx F[ix][kx] xi[ky * m + kx]
  for (int idx = tid; idx < TX2 * m; idx += nthreads) {
    const int c = idx / m, ky = idx - c * m;
    const int ix = x0 + c;
    double acc = 0.0;
    if (ix < n) {
      const double* fx = table + ix * m;
      for (int kx = 0; kx < m; ++kx) acc = fma(fx[kx], s_xi[ky * m + kx], acc);
    }
    s_t[c][ky] = acc;
  }
  __syncthreads();
  const int ix = x0 + threadIdx.x;
  if (ix < n) {
    double* out = kappa + (int64_t)b * es;
#pragma unroll 4
    for (int r = 0; r < KAP_ROWS; ++r) {
      const int rl = threadIdx.y + TY2 * r;
      const int iy = y0 + rl;
      if (iy >= n) break;
      double g = 0.0;
      for (int ky = 0; ky < m; ++ky) g = fma(s_fy[rl][ky], s_t[threadIdx.x][ky], g);
      out[(int64_t)iy * n + ix] = kle_exp(sqrt_sigma2 * g);
    }
  }
  if (prof.acc && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) atomicAdd(prof.acc, prof.per_sample);
}

// 3D: CTA covers 32 (x) x 4 (y) elements for all z of one sample column
// block; per (ix, iy): T2[kz] = sum_ky F[iy][ky] sum_kx F[ix][kx] xi[kz][ky][kx],
// then g(iz) = sum_kz F[iz][kz] T2[kz].
constexpr int K3_TY = 4;
__global__ void __launch_bounds__(TX2* K3_TY)
    k_kappa3d(int n, int m, double sqrt_sigma2, const double* __restrict__ table,
              const double* __restrict__ xi, int M_xi, const int32_t* __restrict__ slot,
              int64_t es, double* __restrict__ kappa, Prof prof) {
  extern __shared__ double smem[];
  const int M = m * m * m;
  double* s_xi = smem;                              // M
  double* s_t1 = s_xi + M;                          // [TX2][m*m]  T1[ix][kz*m+ky]
  const int b = blockIdx.z;
  const int tid = threadIdx.y * TX2 + threadIdx.x;
  const int nthreads = TX2 * K3_TY;
  const int x0 = blockIdx.x * TX2;
  const int iy = blockIdx.y * K3_TY + threadIdx.y;
  load_coefs(xi + (int64_t)b * M_xi, M_xi, slot, M, s_xi, tid, nthreads);
  __syncthreads();
  const int mm = m * m;
  for (int idx = tid; idx < TX2 * mm; idx += nthreads) {
    const int c = idx / mm, kk = idx - c * mm;     // kk = kz * m + ky
    const int ix = x0 + c;
    double acc = 0.0;
    if (ix < n) {
      const double* fx = table + ix * m;
      for (int kx = 0; kx < m; ++kx) acc = fma(fx[kx], s_xi[kk * m + kx], acc);
    }
    s_t1[c * mm + kk] = acc;
  }
  __syncthreads();
  const int ix = x0 + threadIdx.x;
  if (ix >= n || iy >= n) return;
  double t2[MAX_MODES_1D];
  const double* fy = table + iy * m;
  for (int kz = 0; kz < m; ++kz) {
    double acc = 0.0;
    for (int ky = 0; ky < m; ++ky) acc = fma(fy[ky], s_t1[threadIdx.x * mm + kz * m + ky], acc);
    t2[kz] = acc;
  }
  double* out = kappa + (int64_t)b * es;
  for (int iz = 0; iz < n; ++iz) {
    const double* fz = table + iz * m;
    double g = 0.0;
    for (int kz = 0; kz < m; ++kz) g = fma(fz[kz], t2[kz], g);
    out[((int64_t)iz * n + iy) * n + ix] = kle_exp(sqrt_sigma2 * g);
  }
  if (prof.acc && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) atomicAdd(prof.acc, prof.per_sample);
}

template <class T>
__global__ void k_coarsen2d(int nc, const T* __restrict__ kf, T* __restrict__ kc,
                            int64_t esf, int64_t esc, Prof prof) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  const int b = blockIdx.z;
  if (I >= nc) return;
  const int nf = 2 * nc;
  const T* f = kf + (int64_t)b * esf + (int64_t)(2 * J) * nf + 2 * I;
  kc[(int64_t)b * esc + (int64_t)J * nc + I] = T(0.25) * ((f[0] + f[1]) + (f[nf] + f[nf + 1]));
  if (prof.acc && I == 0 && J == 0) atomicAdd(prof.acc, prof.per_sample);
}

template <class T>
__global__ void k_coarsen3d(int nc, const T* __restrict__ kf, T* __restrict__ kc,
                            int64_t esf, int64_t esc, Prof prof) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y % nc;
  const int K = blockIdx.y / nc;
  const int b = blockIdx.z;
  if (I >= nc) return;
  const int nf = 2 * nc;
  const int64_t pl = (int64_t)nf * nf;
  const T* f = kf + (int64_t)b * esf + (int64_t)(2 * K) * pl + (int64_t)(2 * J) * nf + 2 * I;
  const T s0 = (f[0] + f[1]) + (f[nf] + f[nf + 1]);
  const T s1 = (f[pl] + f[pl + 1]) + (f[pl + nf] + f[pl + nf + 1]);
  kc[(int64_t)b * esc + ((int64_t)K * nc + J) * nc + I] = T(0.125) * (s0 + s1);
  if (prof.acc && I == 0 && J == 0 && K == 0) atomicAdd(prof.acc, prof.per_sample);
}

__global__ void k_cast_kappa(int64_t ne, int64_t es, const double* __restrict__ k64,
                             float* __restrict__ k32) {
  const int64_t b = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x)
    k32[b * es + e] = (float)k64[b * es + e];
}

}  // namespace

// 2^(j/64), j < 64, for kle_exp: set once per device (not under stream capture).
cudaError_t init_kle_exp() {
  static std::atomic<uint64_t> done{0};
  return once_per_device(done, [] {
    double tab[64];
    for (int j = 0; j < 64; ++j) tab[j] = (double)std::exp2((long double)j / 64.0L);
    return cudaMemcpyToSymbol(c_exp2_tab, tab, sizeof(tab));
  });
}

cudaError_t launch_cast_kappa(cudaStream_t s, const Grid& g, const double* k64, float* k32,
                              int64_t B) {
  if (B == 0) return cudaSuccess;
  const int64_t ne = ipow(g.n, g.dim);
  const int64_t blocks = std::min<int64_t>((ne + 255) / 256, 4096);
  k_cast_kappa<<<dim3((unsigned)blocks, (unsigned)B), 256, 0, s>>>(ne, g.es, k64, k32);
  return cudaGetLastError();
}

cudaError_t launch_kle_table(cudaStream_t s, int n, int m, const double* omega,
                             const double* theta, const int32_t* even, double* table) {
  const int total = n * m;
  k_kle_table<<<(total + 255) / 256, 256, 0, s>>>(n, m, omega, theta, even, table);
  return cudaGetLastError();
}

cudaError_t launch_kappa(cudaStream_t s, const Grid& g, int m, double sqrt_sigma2,
                         const double* table, const double* xi, int M_xi, const int32_t* slot,
                         int64_t B, double* kappa, Prof p) {
  if (B == 0) return cudaSuccess;
  if (g.dim == 2) {
    dim3 grid((g.n + TX2 - 1) / TX2, (g.n + TY2 * KAP_ROWS - 1) / (TY2 * KAP_ROWS), (unsigned)B);
    k_kappa2d<<<grid, dim3(TX2, TY2), 0, s>>>(g.n, m, sqrt_sigma2, table, xi, M_xi, slot, g.es, kappa, p);
  } else {
    const int M = m * m * m;
    const size_t smem = sizeof(double) * ((size_t)M + (size_t)TX2 * m * m);
    static std::atomic<uint64_t> opted{0};
    const cudaError_t attr = once_per_device(opted, [] {
      return cudaFuncSetAttribute(k_kappa3d, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (attr != cudaSuccess) return attr;
    dim3 grid((g.n + TX2 - 1) / TX2, (g.n + K3_TY - 1) / K3_TY, (unsigned)B);
    k_kappa3d<<<grid, dim3(TX2, K3_TY), smem, s>>>(g.n, m, sqrt_sigma2, table, xi, M_xi, slot, g.es,
                                                   kappa, p);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_coarsen(cudaStream_t s, const Grid& fine, const Grid& coarse,
                           const T* kf, T* kc, int64_t B, Prof p) {
  if (B == 0) return cudaSuccess;
  const int nc = coarse.n;
  const int threads = nc < 128 ? ((nc + 31) / 32) * 32 : 128;
  if (fine.dim == 2) {
    dim3 grid((nc + threads - 1) / threads, nc, (unsigned)B);
    k_coarsen2d<T><<<grid, threads, 0, s>>>(nc, kf, kc, fine.es, coarse.es, p);
  } else {
    dim3 grid((nc + threads - 1) / threads, nc * nc, (unsigned)B);
    k_coarsen3d<T><<<grid, threads, 0, s>>>(nc, kf, kc, fine.es, coarse.es, p);
  }
  return cudaGetLastError();
}

template cudaError_t launch_coarsen<double>(cudaStream_t, const Grid&, const Grid&, const double*,
                                            double*, int64_t, Prof);
template cudaError_t launch_coarsen<float>(cudaStream_t, const Grid&, const Grid&, const float*,
                                           float*, int64_t, Prof);

}  // namespace mlmc
