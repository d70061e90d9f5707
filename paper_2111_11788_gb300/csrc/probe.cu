// Measured FP64 FMA rate of the device (the peak the FP64-bound stencil
// kernels are reported against): a kernel of independent FMA chains that
// keeps every SM's FP64 pipe busy, timed with CUDA events.
#include "mlmc_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 16;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma64_chains(int iters, double seed) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 0.9999999, add = 1e-9;
#pragma unroll 4
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = fma(a[c], m, add);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
  if (s == -1.0) g_probe_sink = s;   // never true (the chains stay positive): keeps them live
}

}  // namespace

extern "C" mlmc_status mlmc_probe_fp64_rate(void* stream, double* tflops, double* ms_out) {
  if (!tflops) return MLMC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MLMC_ERR_CUDA;
  const int blocks = sms * 4;   // 32 warps per SM, 16 chains each
  const int iters = 1 << 14;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MLMC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MLMC_ERR_CUDA;
  }
  mlmc_status st = MLMC_OK;
  float best = 0.f;
  for (int rep = 0; rep < 4 && st == MLMC_OK; ++rep) {   // first launch is a warm-up
    cudaEventRecord(e0, s);
    k_fma64_chains<<<blocks, PROBE_THREADS, 0, s>>>(iters, 1.0 + rep);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = MLMC_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MLMC_OK) return st;
  const double flops = 2.0 * PROBE_CHAINS * (double)iters * blocks * PROBE_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return MLMC_OK;
}
