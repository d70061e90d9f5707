// Per-sample reductions of the batched PCG, level statistics and the MLMC
// estimator / allocation.
//
// finalize: one warp per sample sums that sample's per-tile partials in a
//   fixed order (lane-strided, then a shuffle tree), so every per-sample
//   scalar is independent of the batch width and of the other samples.
// welford:  Y = Q_f - Q_c folded into the level state in sample order
//   (Eq. (sample_variance) as (n, mean, M2), V = M2 / n).
// estimate: Eq. (mlmc_average) q = sum_l mean_l, Sec. 2.2 V(Q~) = sum V_l / N_l,
//   and Eq. (mlmc_num_samples) N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum sqrt(V_i C_i)).
#include "mlmc_internal.cuh"

namespace mlmc {
namespace {

__global__ void k_finalize(int mode, const double* __restrict__ part, int64_t tiles, Scalars sc,
                           double* __restrict__ out, int iter, const int32_t* __restrict__ iter_dev,
                           int max_iter, int64_t B) {
  if (iter_dev) iter = *iter_dev;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  if (mode != FIN_QOI && mode != FIN_GAMMA0 && !sc.active[b]) return;
  const double* p = part + b * tiles;
  double v = 0.0;
  for (int64_t t = lane; t < tiles; t += 32) v += p[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane != 0) return;
  switch (mode) {
    case FIN_GAMMA0:
      sc.gamma[b] = v;
      sc.beta[b] = 0.0;
      break;
    case FIN_ALPHA:
      sc.delta[b] = v;
      sc.alpha[b] = (v > 0.0) ? sc.gamma[b] / v : 0.0;
      break;
    case FIN_CONV: {
      const double rho = sqrt(v);
      sc.rho[b] = rho;
      if (rho <= sc.tol[b]) {
        sc.active[b] = 0;
        sc.iters[b] = iter;
      } else if (iter >= max_iter || !(rho == rho)) {
        sc.active[b] = 0;
        sc.iters[b] = -1;
      }
      break;
    }
    case FIN_BETA: {
      const double g = sc.gamma[b];
      sc.beta[b] = (g != 0.0) ? v / g : 0.0;
      sc.gamma[b] = v;
      break;
    }
    case FIN_QOI:
      out[b] = v;
      break;
  }
}

__global__ void k_count_active(const int32_t* __restrict__ active, int64_t B, int32_t* count) {
  __shared__ int32_t s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int32_t c = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) c += active[b] ? 1 : 0;
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) *count = s;
}

// Loop control of a graph-captured iteration: count the active samples,
// advance the device iteration counter and set the while-condition to
// (some sample active and the cap not reached).
__global__ void k_loop_ctl(const int32_t* __restrict__ active, int64_t B, int32_t* it_dev,
                           int max_iter, int32_t* count, int32_t* execs,
                           cudaGraphConditionalHandle h) {
  __shared__ int32_t s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int32_t c = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) c += active[b] ? 1 : 0;
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int32_t it = *it_dev;
    *count = s;
    *it_dev = it + 1;
    if (execs) *execs += 1;
    cudaGraphSetConditional(h, (s > 0 && it < max_iter) ? 1u : 0u);
  }
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, v);
}

__global__ void k_set_int(int32_t* p, int32_t v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void k_scalars_init(Scalars sc, double tol, double scale0, int64_t B) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  sc.tol[b] = tol;
  sc.active[b] = 1;
  sc.iters[b] = 0;
  sc.beta[b] = 0.0;
  sc.alpha[b] = 0.0;
  sc.gamma[b] = 0.0;
  if (sc.total) sc.total[b] = 0;
  if (sc.scale) sc.scale[b] = scale0;
}

__global__ void k_outer_step(const double* __restrict__ part, int64_t tiles, Scalars so,
                             const int32_t* __restrict__ inner_iters, int inner_max, int outer_it,
                             const int32_t* __restrict__ outer_it_dev, int outer_max, int64_t B) {
  if (outer_it_dev) outer_it = *outer_it_dev;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (b >= B || !so.active[b]) return;
  const double* p = part + b * tiles;
  double v = 0.0;
  for (int64_t t = lane; t < tiles; t += 32) v += p[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane != 0) return;
  const double rho = sqrt(v);
  so.rho[b] = rho;
  int32_t tot = so.total[b];
  if (inner_iters) {
    const int32_t it = inner_iters[b];
    tot += (it > 0) ? it : inner_max;
  }
  so.total[b] = tot;
  const double prev = so.scale[b];   // ||r|| before this refinement step
  if (rho <= so.tol[b] || (rho > 0.5 * prev && rho <= 100.0 * so.tol[b])) {
    // converged, or stalled at the rounding floor of the FP64 residual
    so.active[b] = 0;
    so.iters[b] = tot;
  } else if (outer_it >= outer_max || !(rho == rho)) {
    so.active[b] = 0;
    so.iters[b] = -1;
  } else {
    so.scale[b] = rho;
  }
}

__global__ void k_inner_init(Scalars si, Scalars so, double tol, int64_t B) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  si.active[b] = so.active[b];
  si.tol[b] = tol;
  si.iters[b] = 0;
  si.beta[b] = 0.0;
  si.alpha[b] = 0.0;
  si.gamma[b] = 0.0;
}

__global__ void k_welford(const double* __restrict__ qf, const double* __restrict__ qc, int64_t B,
                          mlmc_level_state* st, double cost) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t n = st->n;
  double mean = st->mean, m2 = st->m2, cs = st->cost_sum;
  for (int64_t s = 0; s < B; ++s) {
    const double y = qc ? qf[s] - qc[s] : qf[s];
    n += 1;
    const double d = y - mean;
    mean += d / (double)n;
    m2 += d * (y - mean);
    cs += cost;
  }
  st->n = n;
  st->mean = mean;
  st->m2 = m2;
  st->cost_sum = cs;
}

__device__ void allocate_dev(const double* V, const double* C, int L, double eps, int64_t* N) {
  double s = 0.0;
  for (int l = 0; l < L; ++l) s += sqrt(V[l] * C[l]);
  const double f = 2.0 / (eps * eps);
  for (int l = 0; l < L; ++l) N[l] = (int64_t)ceil(f * sqrt(V[l] / C[l]) * s);
}

__global__ void k_estimate(const mlmc_level_state* st, int L, const double* __restrict__ C,
                           double eps, double* out2, int64_t* N) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double q = 0.0, v = 0.0;
  double V[16];
  for (int l = 0; l < L; ++l) {
    q += st[l].mean;
    V[l] = st[l].n > 0 ? st[l].m2 / (double)st[l].n : 0.0;
    if (st[l].n > 0) v += V[l] / (double)st[l].n;
  }
  out2[0] = q;
  out2[1] = v;
  if (N && eps > 0.0) allocate_dev(V, C, L, eps, N);
}

// One adaptive step over the active levels 0..La (Sec. 2.3): the sample
// counts of Eq. (mlmc_num_samples), and the level of Eq. (mlmc_num_levels)
// from the bias model |E(Q_l - Q)| = c 2^(-alpha l): least squares of
// log2|Ybar_l| on l over the levels l >= 1 with a nonzero mean (rate 2 with
// one such level), alpha clamped to [0.5, 4], intercept mean(y + alpha l),
// c = 2^a / (2^alpha - 1). The new level never drops below La nor exceeds
// Lmax. Products and sums are rounded one by one (no contraction), in the
// order a plain sequential evaluation takes them.
__global__ void k_adapt(const mlmc_level_state* st, int La, int Lmax, const double* __restrict__ C,
                        double eps, int64_t* N, double* out3) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double V[16];
  for (int l = 0; l <= La; ++l) V[l] = st[l].n > 0 ? st[l].m2 / (double)st[l].n : 0.0;
  allocate_dev(V, C, La + 1, eps, N);
  double ls[16], ys[16];
  int np = 0;
  for (int l = 1; l <= La; ++l) {
    if (st[l].mean != 0.0) {
      ls[np] = (double)l;
      ys[np] = log2(fabs(st[l].mean));
      ++np;
    }
  }
  double Lnew = (double)La, alpha = 0.0, c = 0.0;
  if (np > 0) {
    if (np == 1) {
      alpha = 2.0;
    } else {
      double lbar = 0.0, ybar = 0.0;
      for (int k = 0; k < np; ++k) lbar = __dadd_rn(lbar, ls[k]);
      lbar = __ddiv_rn(lbar, (double)np);
      for (int k = 0; k < np; ++k) ybar = __dadd_rn(ybar, ys[k]);
      ybar = __ddiv_rn(ybar, (double)np);
      double sxy = 0.0, sxx = 0.0;
      for (int k = 0; k < np; ++k)
        sxy = __dadd_rn(sxy, __dmul_rn(__dsub_rn(ls[k], lbar), __dsub_rn(ys[k], ybar)));
      for (int k = 0; k < np; ++k)
        sxx = __dadd_rn(sxx, __dmul_rn(__dsub_rn(ls[k], lbar), __dsub_rn(ls[k], lbar)));
      alpha = -__ddiv_rn(sxy, sxx);
    }
    alpha = fmin(fmax(alpha, 0.5), 4.0);
    double a = 0.0;
    for (int k = 0; k < np; ++k) a = __dadd_rn(a, __dadd_rn(ys[k], __dmul_rn(alpha, ls[k])));
    a = __ddiv_rn(a, (double)np);
    c = __ddiv_rn(exp2(a), __dsub_rn(exp2(alpha), 1.0));
    const double Lr = ceil(__ddiv_rn(log2(__ddiv_rn(__dmul_rn(sqrt(2.0), c), eps)), alpha));
    Lnew = fmin(fmax(Lr, (double)La), (double)Lmax);
  }
  out3[0] = Lnew;
  out3[1] = alpha;
  out3[2] = c;
}

__global__ void k_allocate(const double* V, const double* C, int L, double eps, int64_t* N) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  allocate_dev(V, C, L, eps, N);
}

}  // namespace

cudaError_t launch_finalize(cudaStream_t s, FinMode mode, const double* part, int64_t tiles,
                            const Scalars& sc, double* out, int iter, int max_iter, int64_t B,
                            const int32_t* iter_dev) {
  const int warps = 8;
  k_finalize<<<(unsigned)((B + warps - 1) / warps), warps * 32, 0, s>>>(mode, part, tiles, sc, out,
                                                                      iter, iter_dev, max_iter, B);
  return cudaGetLastError();
}

cudaError_t launch_count_active(cudaStream_t s, const int32_t* active, int64_t B, int32_t* count) {
  k_count_active<<<1, 256, 0, s>>>(active, B, count);
  return cudaGetLastError();
}

cudaError_t launch_loop_ctl(cudaStream_t s, const int32_t* active, int64_t B, int32_t* it_dev,
                            int max_iter, int32_t* count, int32_t* execs,
                            cudaGraphConditionalHandle h) {
  k_loop_ctl<<<1, 256, 0, s>>>(active, B, it_dev, max_iter, count, execs, h);
  return cudaGetLastError();
}

cudaError_t launch_set_cond(cudaStream_t s, cudaGraphConditionalHandle h, unsigned v) {
  k_set_cond<<<1, 32, 0, s>>>(h, v);
  return cudaGetLastError();
}

cudaError_t launch_set_int(cudaStream_t s, int32_t* p, int32_t v) {
  k_set_int<<<1, 32, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_scalars_init(cudaStream_t s, const Scalars& sc, double tol, double scale0,
                                int64_t B) {
  k_scalars_init<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(sc, tol, scale0, B);
  return cudaGetLastError();
}

cudaError_t launch_outer_step(cudaStream_t s, const double* part, int64_t tiles,
                              const Scalars& outer, const int32_t* inner_iters, int inner_max,
                              int outer_it, int outer_max, int64_t B, const int32_t* outer_it_dev) {
  const int warps = 8;
  k_outer_step<<<(unsigned)((B + warps - 1) / warps), warps * 32, 0, s>>>(
      part, tiles, outer, inner_iters, inner_max, outer_it, outer_it_dev, outer_max, B);
  return cudaGetLastError();
}

cudaError_t launch_inner_init(cudaStream_t s, const Scalars& inner, const Scalars& outer,
                              double tol, int64_t B) {
  k_inner_init<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(inner, outer, tol, B);
  return cudaGetLastError();
}

cudaError_t launch_welford(cudaStream_t s, const double* qf, const double* qc, int64_t B,
                           mlmc_level_state* st, double cost) {
  k_welford<<<1, 32, 0, s>>>(qf, qc, B, st, cost);
  return cudaGetLastError();
}

cudaError_t launch_estimate(cudaStream_t s, const mlmc_level_state* st, int n_levels,
                            const double* cost, double eps, double* out2, int64_t* N) {
  k_estimate<<<1, 32, 0, s>>>(st, n_levels, cost, eps, out2, N);
  return cudaGetLastError();
}

cudaError_t launch_adapt(cudaStream_t s, const mlmc_level_state* st, int La, int Lmax,
                         const double* cost, double eps, int64_t* N, double* out3) {
  k_adapt<<<1, 32, 0, s>>>(st, La, Lmax, cost, eps, N, out3);
  return cudaGetLastError();
}

cudaError_t launch_allocate(cudaStream_t s, const double* V, const double* C, int n_levels,
                            double eps, int64_t* N) {
  k_allocate<<<1, 32, 0, s>>>(V, C, n_levels, eps, N);
  return cudaGetLastError();
}

}  // namespace mlmc
