// Counter-based KLE coefficients xi_k(l, i) on the device.
//
// The paper does not name a generator; the coupling of Eq. (mlmc_average)
// only needs xi(l, i) to be reproducible from (level, sample). This kernel
// uses Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
// (j, i, l, stream_id) and key (seed mod 2^32, seed >> 32) for normal pair j,
// 52-bit uniforms u = (x + 1/2) 2^-52, and a Box-Muller transform whose
// log, sine and cosine are built from correctly rounded +, -, *, /, sqrt
// (explicit _rn intrinsics, never contracted into FMA) so that the result
// is bit-reproducible by any IEEE binary64 implementation of the same steps.
#include "mlmc_internal.cuh"

namespace mlmc {
namespace {

constexpr uint32_t PH_M0 = 0xD2511F53u;
constexpr uint32_t PH_M1 = 0xCD9E8D57u;
constexpr uint32_t PH_W0 = 0x9E3779B9u;
constexpr uint32_t PH_W1 = 0xBB67AE85u;

// ln 2 = LN2_HI + LN2_LO; LN2_HI keeps 42 significant bits so e * LN2_HI is
// exact for |e| < 2^10.
constexpr double LN2_HI = 0x1.62e42fefa3800p-1;
constexpr double LN2_LO = 0x1.ef35793c76730p-45;
constexpr double SQRT_HALF = 0x1.6a09e667f3bcdp-1;
constexpr double PIO2 = 0x1.921fb54442d18p+0;

// atanh series: ln m = 2 s sum_k s^(2k) / (2k + 1)
__constant__ double c_log[12] = {
    1.0,        1.0 / 3.0,  1.0 / 5.0,  1.0 / 7.0,  1.0 / 9.0,  1.0 / 11.0,
    1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0, 1.0 / 23.0};
// Taylor series of sin x / x and cos x in z = x^2: (-1)^k / (2k+1)!, (-1)^k / (2k)!
__constant__ double c_sin[11] = {
    1.0,
    -1.0 / 6.0,
    1.0 / 120.0,
    -1.0 / 5040.0,
    1.0 / 362880.0,
    -1.0 / 39916800.0,
    1.0 / 6227020800.0,
    -1.0 / 1307674368000.0,
    1.0 / 355687428096000.0,
    -1.0 / 121645100408832000.0,
    1.0 / 51090942171709440000.0};
__constant__ double c_cos[11] = {
    1.0,
    -1.0 / 2.0,
    1.0 / 24.0,
    -1.0 / 720.0,
    1.0 / 40320.0,
    -1.0 / 3628800.0,
    1.0 / 479001600.0,
    -1.0 / 87178291200.0,
    1.0 / 20922789888000.0,
    -1.0 / 6402373705728000.0,
    1.0 / 2432902008176640000.0};

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PH_W0;
      k1 += PH_W1;
    }
    const uint32_t hi0 = __umulhi(PH_M0, c[0]);
    const uint32_t lo0 = PH_M0 * c[0];
    const uint32_t hi1 = __umulhi(PH_M1, c[2]);
    const uint32_t lo1 = PH_M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  const unsigned long long x = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  return __dmul_rn(__dadd_rn(__ull2double_rn(x), 0.5), 0x1p-52);
}

// ln u from the exact exponent split u = m 2^e, m in [sqrt(1/2), sqrt(2)).
__device__ double ln_exact_ops(double u) {
  int e;
  double m = frexp(u, &e);
  if (m < SQRT_HALF) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double t = __dmul_rn(s, s);
  double p = c_log[11];
#pragma unroll
  for (int k = 10; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, t), c_log[k]);
  const double lnm = __dmul_rn(__dmul_rn(s, p), 2.0);
  const double ed = (double)e;
  return __dadd_rn(__dmul_rn(ed, LN2_HI), __dadd_rn(__dmul_rn(ed, LN2_LO), lnm));
}

// (cos 2 pi u, sin 2 pi u) by exact quadrant reduction of 4u.
__device__ void sincos_2pi_exact_ops(double u, double* cs, double* sn) {
  const double t = __dmul_rn(u, 4.0);
  double q = floor(t);
  double f = __dsub_rn(t, q);
  if (f > 0.5) {
    f = __dsub_rn(f, 1.0);
    q = __dadd_rn(q, 1.0);
  }
  const double x = __dmul_rn(f, PIO2);
  const double z = __dmul_rn(x, x);
  double ps = c_sin[10];
  double pc = c_cos[10];
#pragma unroll
  for (int k = 9; k >= 0; --k) {
    ps = __dadd_rn(__dmul_rn(ps, z), c_sin[k]);
    pc = __dadd_rn(__dmul_rn(pc, z), c_cos[k]);
  }
  const double s = __dmul_rn(x, ps);
  const double c = pc;
  switch (((int)q) & 3) {
    case 0: *cs = c; *sn = s; break;
    case 1: *cs = -s; *sn = c; break;
    case 2: *cs = -c; *sn = -s; break;
    default: *cs = s; *sn = -c; break;
  }
}

__global__ void k_draw_xi(uint32_t key0, uint32_t key1, uint32_t stream_id, uint32_t level,
                          int64_t first, int64_t count, int n_modes, double* __restrict__ xi,
                          Prof prof) {
  const int n_pairs = (n_modes + 1) / 2;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= count * n_pairs) return;
  const int64_t s = tid / n_pairs;
  const int j = (int)(tid - s * n_pairs);
  const uint64_t i = (uint64_t)(first + s);
  uint32_t c[4] = {(uint32_t)j, (uint32_t)i, level, stream_id};
  philox4x32_10(c, key0, key1);
  const double u1 = uniform52(c[0], c[1]);
  const double u2 = uniform52(c[2], c[3]);
  const double r = __dsqrt_rn(__dmul_rn(ln_exact_ops(u1), -2.0));
  double cs, sn;
  sincos_2pi_exact_ops(u2, &cs, &sn);
  double* out = xi + s * n_modes + 2 * j;
  out[0] = __dmul_rn(r, cs);
  if (2 * j + 1 < n_modes) out[1] = __dmul_rn(r, sn);
  if (prof.acc && j == 0) atomicAdd(prof.acc, prof.per_sample);
}

}  // namespace

cudaError_t launch_draw_xi(cudaStream_t s, uint64_t seed, uint32_t stream_id, int level,
                           int64_t first, int64_t count, int n_modes, double* xi, Prof p) {
  const int n_pairs = (n_modes + 1) / 2;
  const int64_t total = count * n_pairs;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (total + threads - 1) / threads;
  k_draw_xi<<<(unsigned)blocks, threads, 0, s>>>((uint32_t)(seed & 0xFFFFFFFFull),
                                                  (uint32_t)(seed >> 32), stream_id,
                                                  (uint32_t)level, first, count, n_modes, xi, p);
  return cudaGetLastError();
}

}  // namespace mlmc
