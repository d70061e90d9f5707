// mlmc_solve_noalloc: the batched PCG solve of mlmc_solve for callers that
// may not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// whose arena already owns all device memory (a raw allocation would fail
// or push the arena out of memory), latency-critical loops where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable,
// and plugin or sandbox hosts that forbid device allocation outright. For
// them this entry point runs the same kernels with its scratch in a static
// device array that is part of the loaded library, so the call itself
// allocates nothing (no cudaMalloc/cudaFree, no pinned host memory).
//
// The array holds MLMC_NOALLOC_SCRATCH_BYTES on every GPU that loads the
// library, until the process exits. Its name is only a host-side stand-in in
// host code; the device address is looked up once per device with
// cudaGetSymbolAddress (on the first call made with that device current).
#include <cmath>
#include <mutex>

#include "mlmc_internal.cuh"

namespace {

using namespace mlmc;

static __device__ __align__(256) unsigned char g_noalloc_scratch[MLMC_NOALLOC_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
constexpr int NA_MAX_MG = 16;
std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (set up once).
cudaError_t na_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

struct NaWs {
  double *x, *r, *p0, *p1, *q, *z;
  double* kap[NA_MAX_MG];
  double* w[NA_MAX_MG];
  double *e[NA_MAX_MG], *r1[NA_MAX_MG], *bk[NA_MAX_MG], *eo[NA_MAX_MG];
  double* part;
  Scalars sc;
  int32_t* count;
};

// Lays the scratch out from `base` (nullptr: size only); returns the bytes used.
size_t na_layout(char* base, const Grid* g, int K, int64_t B, NaWs& w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = (off + 255) / 256 * 256;
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  auto dv = [&](int64_t n) { return (double*)take(sizeof(double) * (size_t)n); };
  const int64_t ns0 = g[0].ns;
  w.x = dv(B * ns0);
  w.r = dv(B * ns0);
  w.p0 = dv(B * ns0);
  w.p1 = dv(B * ns0);
  w.q = dv(B * ns0);
  w.z = dv(B * ns0);
  for (int k = 0; k < K; ++k) {
    w.kap[k] = (k == 0) ? nullptr : dv(B * g[k].es);
    w.w[k] = dv(B * g[k].ns);
    if (K > 1) {
      w.e[k] = dv(B * g[k].ns);
      w.r1[k] = (k < K - 1) ? dv(B * g[k].ns) : nullptr;
      w.bk[k] = (k == 0) ? w.r : dv(B * g[k].ns);
      w.eo[k] = (k == 0) ? w.z : ((k < K - 1) ? dv(B * g[k].ns) : w.e[k]);
    }
  }
  w.part = dv(B * g[0].tiles());
  w.sc.gamma = dv(B);
  w.sc.delta = dv(B);
  w.sc.alpha = dv(B);
  w.sc.beta = dv(B);
  w.sc.rho = dv(B);
  w.sc.tol = dv(B);
  w.sc.active = (int32_t*)take(sizeof(int32_t) * (size_t)B);
  w.sc.iters = (int32_t*)take(sizeof(int32_t) * (size_t)B);
  w.count = (int32_t*)take(sizeof(int32_t));
  w.sc.scale = nullptr;
  w.sc.total = nullptr;
  return off;
}

__global__ void k_na_count_failed(const int32_t* __restrict__ iters, int64_t B, int32_t* count) {
  __shared__ int32_t sc;
  if (threadIdx.x == 0) sc = 0;
  __syncthreads();
  int32_t c = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) c += iters[b] < 0 ? 1 : 0;
  atomicAdd(&sc, c);
  __syncthreads();
  if (threadIdx.x == 0) *count = sc;
}

#define NA_CK(call)                              \
  do {                                           \
    if ((call) != cudaSuccess) return MLMC_ERR_CUDA; \
  } while (0)

mlmc_status na_precondition(cudaStream_t s, const Grid* g, int K, NaWs& w, int64_t B,
                            int64_t* tiles) {
  const Prof off{nullptr, 0.0};
  if (K == 1) {
    NA_CK(d2::jacobi_z(s, g[0], w.w[0], w.r, w.z, w.sc, w.part, B, off));
    *tiles = g[0].tiles_f;
    return MLMC_OK;
  }
  for (int k = 0; k < K - 1; ++k) {
    NA_CK(d2::mg_pre(s, g[k], w.kap[k], w.w[k], w.bk[k], w.e[k], w.r1[k], w.sc.active, B, off,
                     (const double*)nullptr));
    NA_CK(d2::restrict_(s, g[k], g[k + 1], w.r1[k], w.bk[k + 1], w.sc.active, B, off));
  }
  NA_CK(d2::coarse_solve(s, g[K - 1], w.kap[K - 1], w.bk[K - 1], w.e[K - 1], w.sc.active, B));
  for (int k = K - 2; k >= 0; --k)
    NA_CK(d2::mg_post(s, g[k], g[k + 1], w.kap[k], w.w[k], w.bk[k], w.e[k], w.eo[k + 1], w.eo[k],
                      w.sc.active, k == 0 ? w.part : nullptr, B, off, (const double*)nullptr));
  *tiles = g[0].tiles_s;
  return MLMC_OK;
}

}  // namespace

extern "C" mlmc_status mlmc_solve_noalloc(const mlmc_config* c, int mesh, const double* kappa,
                                          int64_t count, double* q, int32_t* iters,
                                          void* stream) {
  if (!c || c->dim != 2 || c->precision != MLMC_FP64) return c ? MLMC_ERR_UNIMPLEMENTED : MLMC_ERR_INVALID;
  if (c->n_levels < 1 || c->n_levels > 16 || c->coarse_cells < 2 || mesh < 0 ||
      mesh >= c->n_levels || count < 0 || count > 65535 || !(c->rtol > 0.0) || c->max_iter < 1 ||
      (c->solver != MLMC_JACOBI_PCG && c->solver != MLMC_GMG_PCG) ||
      (c->qoi != MLMC_QOI_DOMAIN_MEAN && c->qoi != MLMC_QOI_BOX_MEAN))
    return MLMC_ERR_INVALID;
  if (count > 0 && (!kappa || !q)) return MLMC_ERR_INVALID;
  const int64_t n = (int64_t)c->coarse_cells << mesh;
  if (n > 16384) return MLMC_ERR_INVALID;
  if (c->solver == MLMC_GMG_PCG &&
      ((c->coarse_cells & (c->coarse_cells - 1)) != 0 || !(c->mg_omega > 0.0 && c->mg_omega < 2.0)))
    return MLMC_ERR_INVALID;
  if (count == 0) return MLMC_OK;

  Grid g[NA_MAX_MG];
  int K = 1;
  g[0] = make_grid(2, (int)n);
  if (c->solver == MLMC_GMG_PCG) {
    int nn = (int)n;
    while (nn > 2 && K < NA_MAX_MG) {
      nn /= 2;
      g[K++] = make_grid(2, nn);
    }
  }
  NaWs w;
  if (na_layout(nullptr, g, K, count, w) > (size_t)MLMC_NOALLOC_SCRATCH_BYTES)
    return MLMC_ERR_INVALID;   // the batch does not fit the static scratch
  void* base = nullptr;
  NA_CK(na_scratch(&base));
  na_layout((char*)base, g, K, count, w);
  w.kap[0] = const_cast<double*>(kappa);

  cudaStream_t s = (cudaStream_t)stream;
  const Prof off{nullptr, 0.0};
  for (int k = 1; k < K; ++k) NA_CK(launch_coarsen(s, g[k - 1], g[k], w.kap[k - 1], w.kap[k], count, off));
  const double omega = (K > 1) ? c->mg_omega : 1.0;
  for (int k = 0; k < (K > 1 ? K - 1 : 1); ++k) NA_CK(d2::winv(s, g[k], w.kap[k], omega, w.w[k], count));
  const double bnorm = g[0].h * g[0].h * (double)(n - 1);
  NA_CK(launch_scalars_init(s, w.sc, c->rtol * bnorm, 0.0, count));
  NA_CK(d2::pcg_init(s, g[0], w.x, w.r, count, off));
  int64_t Tp = 0;
  mlmc_status st = na_precondition(s, g, K, w, count, &Tp);
  if (st != MLMC_OK) return st;
  NA_CK(launch_finalize(s, FIN_GAMMA0, w.part, Tp, w.sc, nullptr, 0, c->max_iter, count));
  const int check = c->check_every > 0 ? c->check_every : 4;
  double* pold = w.p0;
  double* pnew = w.p1;
  int32_t h_count = 0;
  for (int it = 1; it <= c->max_iter; ++it) {
    NA_CK(d2::pcg_pq(s, g[0], w.kap[0], w.z, pold, pnew, w.q, w.sc, w.part, count, off,
                     (const double*)nullptr));
    NA_CK(launch_finalize(s, FIN_ALPHA, w.part, g[0].tiles_s, w.sc, nullptr, it, c->max_iter, count));
    NA_CK(d2::pcg_xr(s, g[0], w.x, pnew, w.r, w.q, w.sc, w.part, count, off));
    NA_CK(launch_finalize(s, FIN_CONV, w.part, g[0].tiles_f, w.sc, nullptr, it, c->max_iter, count));
    if (it % check == 0 || it == c->max_iter) {
      NA_CK(launch_count_active(s, w.sc.active, count, w.count));
      NA_CK(cudaMemcpyAsync(&h_count, w.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      NA_CK(cudaStreamSynchronize(s));
      if (h_count == 0) break;
    }
    st = na_precondition(s, g, K, w, count, &Tp);
    if (st != MLMC_OK) return st;
    NA_CK(launch_finalize(s, FIN_BETA, w.part, Tp, w.sc, nullptr, it, c->max_iter, count));
    double* t = pold;
    pold = pnew;
    pnew = t;
  }
  const int L = (int)std::lround(c->box_lo * (double)n), H = (int)std::lround(c->box_hi * (double)n);
  const int box = (c->qoi == MLMC_QOI_BOX_MEAN) ? 1 : 0;
  const double vol = (c->box_hi - c->box_lo) * (c->box_hi - c->box_lo);
  NA_CK(d2::qoi(s, g[0], box, L, H, box ? 1.0 / vol : 1.0, w.x, w.part, count, off));
  NA_CK(launch_finalize(s, FIN_QOI, w.part, g[0].tiles_f, w.sc, q, 0, c->max_iter, count));
  if (iters) NA_CK(cudaMemcpyAsync(iters, w.sc.iters, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, s));
  // number of samples that hit max_iter (iteration count -1)
  k_na_count_failed<<<1, 256, 0, s>>>(w.sc.iters, count, w.count);
  NA_CK(cudaGetLastError());
  NA_CK(cudaMemcpyAsync(&h_count, w.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  const int32_t bad = h_count;
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}
