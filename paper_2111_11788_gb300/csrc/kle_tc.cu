// KLE contraction on the tensor cores (tcgen05, TMEM accumulators) for the
// FP32 kappa of the mixed form.
//
// The log-field at the element centroids of one mesh is the dense product
// (Sec. 5.2 KLE, the full tensor basis or its total-order truncation)
//   G[e, b] = sum_k Phi[e, k] Xi[b, k],
//   Phi[e, k] = sqrt(sigma^2) F[ix(e), kx(k)] F[iy(e), ky(k)] (F[iz(e), kz(k)]),
// F the per-axis table sqrt(theta) f(centroid); kappa32[b, e] = exp(G[e, b]).
// Both operands are split into two BF16 terms (v = hi + lo, hi = bf16(v),
// lo = bf16(v - hi)) and G = Ph Xh + Ph Xl + Pl Xh is accumulated in FP32 in
// tensor memory (the lo x lo term is below FP32 resolution of the sum): about
// 16 significant bits per product, far below the inner solve's tolerance.
// The FP64 kappa of the outer residual is not made here.
//
// A CTA (16 warps) owns N_t samples (N_t a multiple of 16, <= 256) and walks
// 128-element tiles of the mesh. Xi of its samples stays in shared memory for
// the whole launch; Phi is generated a 64-mode chunk at a time (four threads
// per tile row, 16 modes each, the per-axis factors of the tile's rows in
// shared memory, the log2(e) of the epilogue folded into them) into one of
// two stages while the MMAs of the other stage run. Shared operands use the
// 128-byte swizzled K-major layout (rows of 64 BF16, 8-row atoms of 1 KB);
// thread 0 issues tcgen05.mma (M = 128, N = N_t, K = 16) and commits each
// stage to an mbarrier. The accumulators are double-buffered in tensor
// memory: while the MMAs of tile t run, the CTA loads the factors of its
// next tile and runs the epilogue of tile t - 1, which reads that buffer
// with tcgen05.ld (warp w: lanes 32 (w mod 4) .. 32 (w mod 4) + 31, i.e.
// elements, and every fourth 16-column chunk starting at w / 4) and stores
// kappa32 = 2^(G log2 e) coalesced along the elements. Waits on mbarriers
// are bounded: a CTA whose wait gives up counts a timeout in g_tc_timeouts,
// lets its MMAs land (bounded), frees its tensor memory and ends.
#include "mlmc_internal.cuh"

#include <cuda_bf16.h>

namespace mlmc {
namespace {

constexpr int TC_THREADS = 512;
constexpr int TC_ROW_THREADS = TC_THREADS / 128;   // threads per tile row
constexpr int TC_TILE = 128;                       // elements per tile (MMA M)
constexpr int TC_KC = 64;                          // modes per chunk (one 128-byte row of BF16)
constexpr int TC_CHUNK_BYTES = TC_TILE * TC_KC * 2;  // one BF16 operand chunk of Phi: 16 KB
constexpr int TC_WAIT_TRIES = 1 << 22;
constexpr long long TC_WAIT_CYCLES = 1ll << 32;

__device__ unsigned int g_tc_timeouts;

// ---- PTX wrappers --------------------------------------------------------

__device__ __forceinline__ void tc_mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool tc_mbar_wait(unsigned addr, unsigned parity) {
  if (tc_mbar_try(addr, parity)) return true;
  const long long t0 = clock64();
  for (int k = 0; k < TC_WAIT_TRIES; ++k) {
    if (tc_mbar_try(addr, parity)) return true;
    if (clock64() - t0 > TC_WAIT_CYCLES) break;
  }
  return false;
}
__device__ __forceinline__ void tmem_alloc(unsigned smem_dst, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_dst),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// D (tensor memory) (+)= A * B, A and B BF16 from shared-memory descriptors.
__device__ __forceinline__ void umma_bf16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier completes one phase when the MMAs issued so far by this thread have completed.
__device__ __forceinline__ void umma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// 2^x by the hardware approximation (ex2.approx.ftz.f32, relative error
// about 2^-22): kappa32 = exp(G) = 2^(G log2 e), the log2(e) folded into Phi.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Shared-memory matrix descriptor: 128-byte swizzled K-major tile whose
// 8-row atoms are 1024 bytes apart (start at `addr`, advanced by 32 bytes per
// K step of 16 BF16 inside the swizzle row).
__device__ __forceinline__ uint64_t sw128_desc(unsigned addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                        // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}
// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major, M x N.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) (k < 64) in a 128-byte swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)row * 128u + ((uint32_t)(((k >> 3) ^ (row & 7)) << 4)) + (uint32_t)((k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

struct TcArgs {
  int dim, n, m;
  int M;                 // kept modes (columns of Phi)
  int nch;               // 64-mode chunks (K padded to nch * 64)
  int Nt;                // samples per CTA (multiple of 16, <= 256)
  int tmem_cols;         // two buffers of the power of two >= max(32, Nt) columns
  int64_t ne;            // elements of the mesh
  int64_t es;            // element stride of kappa32
  int64_t B;             // samples
  float scale;           // sqrt(sigma^2) log2(e): the accumulators hold G log2(e)
  const double* table;   // F[i * m + k], i < n, k < m
  const double* xi;      // Xi[b * M + k]
  const int32_t* slot;   // kept mode t -> full index (null: t itself)
  float* kappa32;
  // shared-memory layout (bytes from the 1024-aligned base)
  uint32_t off_a, off_b, off_modes, off_fac, off_bar;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_kappa32_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  const uint32_t raw0 = (uint32_t)__cvta_generic_to_shared(tc_raw);
  const uint32_t base = (raw0 + 1023u) & ~1023u;
  unsigned char* sm = tc_raw + (base - raw0);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b0 = blockIdx.y * a.Nt;
  const int K = a.nch * TC_KC;
  int4* modes = reinterpret_cast<int4*>(sm + a.off_modes);
  float* fac = reinterpret_cast<float*>(sm + a.off_fac);          // [dim][m][TC_TILE]
  // mbarriers: two stages of Phi, two accumulator buffers; then the TMEM address
  const uint32_t bar_stage0 = base + a.off_bar, bar_acc0 = base + a.off_bar + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + a.off_bar + 32);
  const int m = a.m;

  // kept modes as the fac offsets of their per-axis factors (x, y, z rows of
  // fac; w = 0 for padding columns, whose Phi is 0)
  for (int t = tid; t < K; t += TC_THREADS) {
    int4 code = make_int4(0, 0, 0, 0);
    if (t < a.M) {
      int k = a.slot ? a.slot[t] : t;
      const int kx = k % m;
      k /= m;
      const int ky = k % m;
      const int kz = a.dim == 3 ? k / m : 0;
      code = make_int4(kx * TC_TILE, (m + ky) * TC_TILE, (2 * m + kz) * TC_TILE, 1);
    }
    modes[t] = code;
  }
  // Xi of this CTA's samples, split, in the swizzled K-major layout: chunk c
  // of the hi (lo) part at off_b + (2 c (+1)) * Nt * 128
  for (int idx = tid; idx < a.Nt * K; idx += TC_THREADS) {
    const int r = idx / K, k = idx - r * K;
    const int64_t bb = b0 + r;
    const float v = (bb < a.B && k < a.M) ? (float)a.xi[bb * a.M + k] : 0.f;
    __nv_bfloat16 hi, lo;
    split_bf16(v, hi, lo);
    const int c = k / TC_KC;
    const uint32_t o = sw128_off(r, k - c * TC_KC);
    *reinterpret_cast<__nv_bfloat16*>(sm + a.off_b + (2 * c) * a.Nt * 128 + o) = hi;
    *reinterpret_cast<__nv_bfloat16*>(sm + a.off_b + (2 * c + 1) * a.Nt * 128 + o) = lo;
  }
  if (tid == 0) {
    tc_mbar_init(bar_stage0, 1);
    tc_mbar_init(bar_stage0 + 8, 1);
    tc_mbar_init(bar_acc0, 1);
    tc_mbar_init(bar_acc0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    tmem_alloc(base + a.off_bar + 32, (unsigned)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = bf16_idesc(TC_TILE, a.Nt);

  const int64_t tiles = (a.ne + TC_TILE - 1) / TC_TILE;
  const uint32_t bufcols = (uint32_t)a.tmem_cols / 2;   // two accumulator buffers
  const int row = tid & (TC_TILE - 1), quarter = tid >> 7;
  // per-axis factors of row `row` of tile t into fac (the row's four threads
  // write every fourth mode)
  auto load_fac = [&](int64_t t) {
    const int64_t e = t * TC_TILE + row;
    const bool real = e < a.ne;
    int ix = 0, iy = 0, iz = 0;
    if (real) {
      ix = (int)(e % a.n);
      const int64_t q = e / a.n;
      iy = (int)(q % a.n);
      iz = a.dim == 3 ? (int)(q / a.n) : 0;
    }
    for (int k = quarter; k < m; k += TC_ROW_THREADS) {
      fac[k * TC_TILE + row] = real ? a.scale * (float)a.table[ix * m + k] : 0.f;
      fac[(m + k) * TC_TILE + row] = real ? (float)a.table[iy * m + k] : 0.f;
      if (a.dim == 3) fac[(2 * m + k) * TC_TILE + row] = real ? (float)a.table[iz * m + k] : 0.f;
    }
  };
  // exp of the accumulators of tile t (buffer t mod 2) into kappa32, once its MMAs have completed
  auto epilogue = [&](int64_t t, int nt) -> bool {
    const uint32_t b = (uint32_t)(nt & 1);
    const bool ok = tc_mbar_wait(bar_acc0 + 8u * b, (unsigned)((nt >> 1) & 1));
    tc_fence_after();
    if (ok) {
      // warp w: accumulator lanes (elements) 32 (w mod 4) .., column chunks w / 4, w / 4 + 4, ..
      const int lq = warp & 3, cg = warp >> 2;
      const int64_t ee = t * TC_TILE + 32 * lq + (tid & 31);
      const uint32_t lane_addr = tmem + b * bufcols + ((uint32_t)(lq * 32) << 16);
      for (int c0 = 16 * cg; c0 < a.Nt; c0 += 16 * TC_ROW_THREADS) {
        uint32_t r[16];
        tmem_ld16(lane_addr + (uint32_t)c0, r);
        tmem_ld_wait();
        if (ee < a.ne) {
          float* dst = a.kappa32 + (int64_t)(b0 + c0) * a.es + ee;
          const int64_t left = a.B - (b0 + c0);
#pragma unroll
          for (int j = 0; j < 16; ++j, dst += a.es)
            if (j < left) *dst = ex2_approx(__uint_as_float(r[j]));
        }
      }
    }
    return ok;
  };
  // Per tile t (the CTA's ntile-th): Phi of t and its MMAs into accumulator
  // buffer ntile mod 2; then the factors of the next tile; then the epilogue
  // of the previous tile, whose MMAs ran meanwhile.
  int gc = 0;          // chunks issued by this CTA (stage = gc & 1)
  int ntile = 0;       // tiles whose MMAs were issued by this CTA
  bool failed = false;
  if ((int64_t)blockIdx.x < tiles) load_fac(blockIdx.x);
  __syncthreads();
  int64_t prev = -1;
  for (int64_t tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const uint32_t acc_cols = tmem + (uint32_t)(ntile & 1) * bufcols;
    for (int c = 0; c < a.nch; ++c, ++gc) {
      const int s = gc & 1;
      // the stage's previous MMAs (chunk gc - 2) must have read it
      const bool ok = gc < 2 || tc_mbar_wait(bar_stage0 + 8u * s, (unsigned)(((gc - 2) >> 1) & 1));
      if (ok) {
        unsigned char* ah = sm + a.off_a + s * 2 * TC_CHUNK_BYTES;
        unsigned char* al = ah + TC_CHUNK_BYTES;
#pragma unroll 1
        for (int jj = 0; jj < TC_KC / 8 / TC_ROW_THREADS; ++jj) {   // 8 modes (16 bytes) at a time
          const int j = quarter * (TC_KC / 8 / TC_ROW_THREADS) + jj;
          __align__(16) __nv_bfloat162 hv[4], lv[4];
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int4 code = modes[c * TC_KC + j * 8 + 2 * q2 + h];
              v[h] = 0.f;
              if (code.w) {
                v[h] = fac[code.x + row] * fac[code.y + row];
                if (a.dim == 3) v[h] *= fac[code.z + row];
              }
            }
            // the two modes' hi parts in one paired conversion, then their lo parts
            hv[q2] = __floats2bfloat162_rn(v[0], v[1]);
            const float2 hf = __bfloat1622float2(hv[q2]);
            lv[q2] = __floats2bfloat162_rn(v[0] - hf.x, v[1] - hf.y);
          }
          const uint32_t o = sw128_off(row, j * 8);
          *reinterpret_cast<uint4*>(ah + o) = *reinterpret_cast<const uint4*>(hv);
          *reinterpret_cast<uint4*>(al + o) = *reinterpret_cast<const uint4*>(lv);
        }
      }
      tc_fence_proxy_async();   // generic writes of the stage before the MMAs read it
      tc_fence_before();
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_hi = base + a.off_a + s * 2 * TC_CHUNK_BYTES, a_lo = a_hi + TC_CHUNK_BYTES;
        const uint32_t b_hi = base + a.off_b + (2 * c) * a.Nt * 128, b_lo = b_hi + a.Nt * 128;
#pragma unroll
        for (int kk = 0; kk < TC_KC / 16; ++kk) {
          const uint32_t ko = kk * 32;
          const unsigned acc = (c > 0 || kk > 0) ? 1u : 0u;
          umma_bf16(acc_cols, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), idesc, acc);
          umma_bf16(acc_cols, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), idesc, 1u);
          umma_bf16(acc_cols, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), idesc, 1u);
        }
        umma_commit(bar_stage0 + 8u * s);
        if (c == a.nch - 1) umma_commit(bar_acc0 + 8u * (uint32_t)(ntile & 1));
      }
    }
    if (failed) break;
    // the last chunk's barrier ended every read of fac for this tile
    if (tile + gridDim.x < tiles) load_fac(tile + gridDim.x);
    bool ok = true;
    if (prev >= 0) ok = epilogue(prev, ntile - 1);
    prev = tile;
    ++ntile;
    tc_fence_before();
    // every thread's TMEM reads of the previous buffer precede its next MMAs,
    // and the next tile's factors are complete
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (!failed && prev >= 0) {
    const bool ok = epilogue(prev, ntile - 1);
    tc_fence_before();
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (failed) {
    // record the timeout and let the MMAs in flight land (bounded) before freeing the accumulators
    if (tid == 0) {
      atomicAdd(&g_tc_timeouts, 1u);
      for (int s = 0; s < 2; ++s)
        if (gc - 1 - s >= 0) tc_mbar_wait(bar_stage0 + 8u * ((gc - 1 - s) & 1), (unsigned)(((gc - 1 - s) >> 1) & 1));
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (unsigned)a.tmem_cols);
  }
}

}  // namespace

// Shared-memory plan of the kernel for Nt samples; returns the dynamic bytes.
static size_t tc_layout(int dim, int m, int nch, int Nt, TcArgs* out) {
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    const size_t o = off;
    off += bytes;
    return (uint32_t)o;
  };
  TcArgs& a = *out;
  a.off_a = take(4 * (size_t)TC_CHUNK_BYTES, 1024);                 // two stages of hi + lo
  a.off_b = take((size_t)nch * 2 * Nt * 128, 1024);                 // Xi hi/lo, every chunk
  a.off_modes = take(sizeof(int4) * (size_t)nch * TC_KC, 16);
  a.off_fac = take(sizeof(float) * (size_t)dim * m * TC_TILE, 16);
  a.off_bar = take(48, 16);
  return off + 1024;   // slack for aligning the dynamic base to 1 KB
}

cudaError_t launch_kappa32_tc(cudaStream_t s, const Grid& g, int m, double sqrt_sigma2, const double* table,
                              const double* xi, int M, const int32_t* slot, int64_t B, float* kappa32) {
  if (B <= 0) return cudaSuccess;
  if (M < 1 || m < 1 || m > 255 || (g.dim != 2 && g.dim != 3)) return cudaErrorInvalidValue;
  const int nch = (M + TC_KC - 1) / TC_KC;
  // samples per CTA: a multiple of 16 up to 256 whose Xi fits beside the rest
  constexpr size_t kSmemMax = 220 * 1024;
  int Nt = (int)std::min<int64_t>(256, (B + 15) / 16 * 16);
  TcArgs a{};
  size_t bytes = tc_layout(g.dim, m, nch, Nt, &a);
  while (bytes > kSmemMax && Nt > 16) {
    Nt -= 16;
    bytes = tc_layout(g.dim, m, nch, Nt, &a);
  }
  if (bytes > kSmemMax) return cudaErrorInvalidValue;
  // at least 116 KB so that one CTA runs per SM (its tensor memory never waits for another's)
  bytes = std::max<size_t>(bytes, 116 * 1024);
  int cols = 32;
  while (cols < Nt) cols *= 2;
  cols *= 2;   // two accumulator buffers
  a.dim = g.dim;
  a.n = g.n;
  a.m = m;
  a.M = M;
  a.nch = nch;
  a.Nt = Nt;
  a.tmem_cols = cols;
  a.ne = ipow(g.n, g.dim);
  a.es = g.es;
  a.B = B;
  a.scale = (float)(sqrt_sigma2 * 1.4426950408889634074);   // log2(e)
  a.table = table;
  a.xi = xi;
  a.slot = slot;
  a.kappa32 = kappa32;
  static std::atomic<uint64_t> opted{0};
  cudaError_t e = once_per_device(opted, [] {
    return cudaFuncSetAttribute(k_kappa32_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax + 1024);
  });
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t tiles = (a.ne + TC_TILE - 1) / TC_TILE;
  const int64_t ntiles_b = (B + Nt - 1) / Nt;
  // persistent over element tiles: about one CTA per SM in total
  const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(tiles, (sms + ntiles_b - 1) / ntiles_b));
  k_kappa32_tc<<<dim3((unsigned)gx, (unsigned)ntiles_b, 1), TC_THREADS, bytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t take_tc_timeouts(cudaStream_t s, unsigned* out) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_tc_timeouts, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h != 0) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_timeouts, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  *out = h;
  return e;
}

}  // namespace mlmc
