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
// Stencil kernels march along z: a CTA owns a 32 x 16 tile of node columns
// and a chunk of zc planes; a thread owns two rows of one column. Each step
// stages one plane of the input field (with a one-node halo) and one layer
// of kappa (with a one-element halo) in shared memory, double buffered,
// while the next plane is fetched into registers. A plane p feeds three
// outputs of a column: p - 1 (the 8 couplings across layer p - 1, after
// which output p - 1 is complete and goes to the epilogue), p (the centre
// and its 4 in-plane diagonal edge neighbours) and p + 1 (the 8 couplings
// across layer p). So a node costs about one coalesced load of the field and
// of kappa, a few shared-memory reads and one store, instead of 27 + 8
// cached global loads. The field a stencil acts on is formed by a loader
// while its plane is staged (z + beta p for A p, omega D^-1 b for the
// multigrid residual), so those need no pointwise pre-pass. In FP32 the two
// rows of a thread are 8 apart and stored as pairs, so the stencil runs on
// paired FP32 instructions (or, on 32..256 cells per side, on full-width
// tiles staged by TMA bulk copies, k_zm3w). In FP64, where the plan has the
// per-node kappa sums of the level, the same march runs on element sums
// (k_zm3q: about 19 instead of 33 FP64 operations per node). The remaining pointwise kernels run one thread
// per node column of a 32 x 8 tile over 8 z-planes on grids of 64 and more
// cells per side, else over one (the prolongation: one thread per fine
// x-pair over 8 planes); the initialisation and the QoI run
// one CTA per z-plane. Node arrays carry the boundary nodes (always 0).
// Partials: one per CTA (g.tiles_s per sample for the stencil kernels,
// g.tiles_q = N1 for the QoI). The multigrid levels of at most
// 16^3 cells below the finest run as one kernel per V-cycle (k_bottom3, one
// CTA per sample in shared memory).
#include "mlmc_internal.cuh"

#include <type_traits>

namespace mlmc {
namespace {

constexpr int BX = 32, BY = 8;

struct Node3 {
  int i, j, k;
  bool valid, interior;
  int64_t idx;  // (k * N1 + j) * N1 + i
};


// Node tiles with a z-loop: CTA (zg, tile) covers the 32 x 8 node tile in
// planes zg * pz .. zg * pz + pz - 1 (one thread per column, pz planes
// each), so a pointwise kernel on a large grid runs few, large CTAs
// (pz = NODE_PZ) and one on a small grid keeps one plane per thread
// (node_pz).
constexpr int NODE_PZ = 8;
inline int node_pz(int n) { return n >= 64 ? NODE_PZ : 1; }
struct NodeCol {
  int i, j, k0, k1;   // column (i, j), planes [k0, k1)
  bool valid;         // the column lies in the mesh
};
__device__ __forceinline__ NodeCol node_col3(int n, int pz) {
  const int N1 = n + 1;
  const int tx = (N1 + BX - 1) / BX, ty = (N1 + BY - 1) / BY;
  const int tiles = tx * ty;
  const int zg = blockIdx.x / tiles;
  const int t = blockIdx.x - zg * tiles;
  const int ty_ = t / tx;
  NodeCol c;
  c.i = (t - ty_ * tx) * BX + threadIdx.x;
  c.j = ty_ * BY + threadIdx.y;
  c.k0 = zg * pz;
  c.k1 = min(c.k0 + pz, N1);
  c.valid = c.i <= n && c.j <= n;
  return c;
}
inline unsigned node_col3_blocks(int n, int pz) {
  const int N1 = n + 1;
  return (unsigned)(((N1 + BX - 1) / BX) * ((N1 + BY - 1) / BY) * ((N1 + pz - 1) / pz));
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
__device__ __forceinline__ T diag3(const T kk[2][2][2], double c3) {
  const T s = ((kk[0][0][0] + kk[0][0][1]) + (kk[0][1][0] + kk[0][1][1])) +
              ((kk[1][0][0] + kk[1][0][1]) + (kk[1][1][0] + kk[1][1][1]));
  return T(c3) * s;
}

// ---------------------------------------------------------------- z-march

constexpr int ZTX = 32, ZTY = 16;          // node columns per CTA (x, y)
constexpr int ZRY = 2;                     // y-rows per thread
constexpr int ZTHREADS = ZTX * (ZTY / ZRY);
constexpr int ZSX = ZTX + 2, ZSY = ZTY + 2, ZNV = ZSX * ZSY;   // vector plane + halo
constexpr int ZKX = ZTX + 1, ZKY = ZTY + 1, ZNK = ZKX * ZKY;   // kappa layer + halo
constexpr int ZSLOTS = ((ZNV > ZNK ? ZNV : ZNK) + ZTHREADS - 1) / ZTHREADS;
static_assert(ZNV <= ZSLOTS * ZTHREADS && ZNK <= ZSLOTS * ZTHREADS, "staging slots per thread");
static_assert(ZTHREADS == BX * BY, "the z-march CTA has the node-tile thread count");

struct ZTile {
  int tx0, ty0, z0, z1;   // column origin; output planes [z0, z1)
};

__device__ __forceinline__ ZTile ztile(const Grid& g) {
  const int txn = (g.n + ZTX - 1) / ZTX, tyn = (g.n + ZTY - 1) / ZTY;
  int t = blockIdx.x;
  const int zq = t / (txn * tyn);
  t -= zq * txn * tyn;
  const int ty = t / txn;
  ZTile z;
  z.tx0 = (t - ty * txn) * ZTX;
  z.ty0 = ty * ZTY;
  z.z0 = zq * g.zc;
  z.z1 = min(z.z0 + g.zc, g.n + 1);
  return z;
}

// Generic z-marching stencil kernel: y = A(kappa) x at every node of the
// CTA's columns and planes, handed to the epilogue with the centre value of
// x; the epilogue's returned values are summed (in T per thread, in FP64
// across the CTA) into one partial per CTA (part may be null). A thread owns
// two adjacent y-rows of one x-column. The epilogue's own inputs for a node
// are fetched one plane ahead (Epi::Pre). Tiles cover node columns
// [0, 32 ceil(n/32)) x [0, 16 ceil(n/16)); when n is a multiple of the tile
// width, the column n (boundary) is written by the thread of column n - 1
// (epi.zero). Offsets inside one sample fit 32 bits ((n + 1)^3 < 2^31).
template <class T, class Ld, class Epi>
__global__ void __launch_bounds__(ZTHREADS, 2) k_zm3(Grid g, const T* __restrict__ Kap, Ld ld,
                                                  const int32_t* __restrict__ active, Epi epi,
                                                  double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ T sv[2][ZNV];
  __shared__ T sk[2][ZNK];
  const ZTile t = ztile(g);
  const int n = g.n, N1 = n + 1, P = N1 * N1, KP = n * n;
  const int tid = threadIdx.y * ZTX + threadIdx.x;
  const T* __restrict__ kp = Kap + b * g.es;
  ld.bind(b);
  epi.bind(b);
  // staging slots: plane entries tid + q * ZTHREADS, with their in-plane
  // offsets and whether they lie inside (interior nodes for x, whose
  // boundary values are ignored; mesh elements for kappa)
  int vo[ZSLOTS], ko[ZSLOTS];
  bool vok[ZSLOTS], kok[ZSLOTS], vin[ZSLOTS], kin[ZSLOTS];
#pragma unroll
  for (int q = 0; q < ZSLOTS; ++q) {
    const int sidx = tid + q * ZTHREADS;
    vin[q] = sidx < ZNV;
    kin[q] = sidx < ZNK;
    const int vx = t.tx0 - 1 + sidx % ZSX, vy = t.ty0 - 1 + sidx / ZSX;
    vok[q] = vin[q] && vx >= 1 && vx < n && vy >= 1 && vy < n;
    vo[q] = vok[q] ? vy * N1 + vx : 0;
    const int kx = t.tx0 - 1 + sidx % ZKX, ky = t.ty0 - 1 + sidx / ZKX;
    kok[q] = kin[q] && kx >= 0 && kx < n && ky >= 0 && ky < n;
    ko[q] = kok[q] ? ky * n + kx : 0;
  }
  T rv[ZSLOTS], rk[ZSLOTS];
  auto fetch = [&](int pp) {
    const bool pv = pp >= 1 && pp < n, pk = pp >= 0 && pp < n;
#pragma unroll
    for (int q = 0; q < ZSLOTS; ++q) {
      rv[q] = (pv && vok[q]) ? ld(pp * P + vo[q]) : T(0);
      rk[q] = (pk && kok[q]) ? __ldg(kp + pp * KP + ko[q]) : T(0);
    }
  };
  int p = t.z0 - 1;
  fetch(p);

  const int i = t.tx0 + threadIdx.x;
  const int j0 = t.ty0 + ZRY * threadIdx.y;
  bool cvalid[ZRY], cint[ZRY], ey[ZRY];
  int ocol[ZRY];
#pragma unroll
  for (int r = 0; r < ZRY; ++r) {
    const int j = j0 + r;
    cvalid[r] = i <= n && j <= n;
    cint[r] = i >= 1 && i < n && j >= 1 && j < n;
    ey[r] = j == n - 1 && n % ZTY == 0;
    ocol[r] = j * N1 + i;
  }
  const bool ex = i == n - 1 && n % ZTX == 0;
  const T c3 = T(g.c3), c12 = T(g.c12);
  // Per output row: U = unscaled coupling sum and D = (sum of the 8 kappa) x
  // centre of the output of plane p - 1 so far, N = the couplings of the
  // output of plane p with plane p - 1; output = c3 D - c12 U. Pair sums of a
  // kappa layer (X: along x per element row, Y: along y per column, S: the 4
  // elements around an output row) are formed once per layer and reused by
  // both rows and by the next plane; every coupling is one FMA into U.
  T U[ZRY], D[ZRY], N[ZRY], vc[ZRY];
  typename Epi::Pre pre[ZRY];    // epilogue inputs of plane p - 1
#pragma unroll
  for (int r = 0; r < ZRY; ++r) U[r] = D[r] = N[r] = vc[r] = T(0);
  T kb[ZRY + 1][2];              // kappa layer p - 1, element rows j0 - 1 .. j0 + ZRY - 1
  T Xb[ZRY + 1], Yb[ZRY][2], Sb[ZRY];
#pragma unroll
  for (int r = 0; r <= ZRY; ++r) kb[r][0] = kb[r][1] = Xb[r] = T(0);
#pragma unroll
  for (int r = 0; r < ZRY; ++r) Yb[r][0] = Yb[r][1] = Sb[r] = T(0);
  T dot = T(0);
  const int vbase = (ZRY * threadIdx.y + 1) * ZSX + threadIdx.x + 1;
  const int kbase = ZRY * threadIdx.y * ZKX + threadIdx.x;
  int buf = 0;
  for (; p <= t.z1; ++p) {
    T* svb = sv[buf];
    T* skb = sk[buf];
#pragma unroll
    for (int q = 0; q < ZSLOTS; ++q) {
      if (vin[q]) svb[tid + q * ZTHREADS] = rv[q];
      if (kin[q]) skb[tid + q * ZTHREADS] = rk[q];
    }
    __syncthreads();
    if (p < t.z1) fetch(p + 1);   // the next plane is in flight while this one is used
    typename Epi::Pre nxt[ZRY];
#pragma unroll
    for (int r = 0; r < ZRY; ++r)
      if (cint[r] && p >= t.z0 && p < t.z1 && p >= 1 && p < n) nxt[r] = epi.load(p * P + ocol[r]);
    T v[ZRY + 2][3], ka[ZRY + 1][2];
#pragma unroll
    for (int r = 0; r < ZRY + 2; ++r)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) v[r][dx] = svb[vbase + (r - 1) * ZSX + (dx - 1)];
#pragma unroll
    for (int r = 0; r <= ZRY; ++r)
#pragma unroll
      for (int a = 0; a < 2; ++a) ka[r][a] = skb[kbase + r * ZKX + a];
    T Xa[ZRY + 1], Ya[ZRY][2], Sa[ZRY];
#pragma unroll
    for (int r = 0; r <= ZRY; ++r) Xa[r] = ka[r][0] + ka[r][1];
#pragma unroll
    for (int r = 0; r < ZRY; ++r) {
      Ya[r][0] = ka[r][0] + ka[r + 1][0];
      Ya[r][1] = ka[r][1] + ka[r + 1][1];
      Sa[r] = Xa[r] + Xa[r + 1];
    }
    const int m = p - 1;
#pragma unroll
    for (int r = 0; r < ZRY; ++r) {
      const T* v0 = v[r];
      const T* v1 = v[r + 1];
      const T* v2 = v[r + 2];
      // couplings of output p - 1 with plane p across layer p - 1: complete
      T u = U[r];
      u = fma(Yb[r][0], v1[0], u);
      u = fma(Yb[r][1], v1[2], u);
      u = fma(Xb[r], v0[1], u);
      u = fma(Xb[r + 1], v2[1], u);
      u = fma(kb[r][0], v0[0], u);
      u = fma(kb[r][1], v0[2], u);
      u = fma(kb[r + 1][0], v2[0], u);
      u = fma(kb[r + 1][1], v2[2], u);
      // A x = c3 D - c12 U, or f - A x = f - c3 D + c12 U for a residual epilogue
      T done;
      if constexpr (Epi::kRes) done = fma(c12, u, fma(-c3, D[r], T(epi.rhs(pre[r]))));
      else done = fma(-c12, u, c3 * D[r]);
      if (cvalid[r] && m >= t.z0) {
        const int o = m * P + ocol[r];
        dot += epi(o, cint[r] && m >= 1 && m < n, done, vc[r], pre[r]);
        if (ex) epi.zero(o + 1);
        if (ey[r]) epi.zero(o + N1);
        if (ex && ey[r]) epi.zero(o + N1 + 1);
      }
      // output p: couplings with plane p - 1 (N) and the in-plane diagonal
      // edges (free axis z: one kappa of each layer), and the diagonal part
      u = N[r];
      u = fma(kb[r][0] + ka[r][0], v0[0], u);
      u = fma(kb[r][1] + ka[r][1], v0[2], u);
      u = fma(kb[r + 1][0] + ka[r + 1][0], v2[0], u);
      u = fma(kb[r + 1][1] + ka[r + 1][1], v2[2], u);
      U[r] = u;
      D[r] = (Sb[r] + Sa[r]) * v1[1];
      // output p + 1: couplings with plane p across layer p
      u = Ya[r][0] * v1[0];
      u = fma(Ya[r][1], v1[2], u);
      u = fma(Xa[r], v0[1], u);
      u = fma(Xa[r + 1], v2[1], u);
      u = fma(ka[r][0], v0[0], u);
      u = fma(ka[r][1], v0[2], u);
      u = fma(ka[r + 1][0], v2[0], u);
      N[r] = fma(ka[r + 1][1], v2[2], u);
      vc[r] = v1[1];
      pre[r] = nxt[r];
    }
#pragma unroll
    for (int r = 0; r <= ZRY; ++r) {
      kb[r][0] = ka[r][0];
      kb[r][1] = ka[r][1];
      Xb[r] = Xa[r];
    }
#pragma unroll
    for (int r = 0; r < ZRY; ++r) {
      Yb[r][0] = Ya[r][0];
      Yb[r][1] = Ya[r][1];
      Sb[r] = Sa[r];
    }
    buf ^= 1;
  }
  if (part) cta_partial3((double)dot, part, g.tiles_s);
  prof_tick3(prof);
}

// FP64 z-march on precomputed kappa sums (k_zm3q). With K_n the sum of the 8
// kappa around node n and K_{n,n+d} the sum of the 4 elements sharing the
// edge (n, n+d), the Q1 row of node n (element stiffness h/12 (4, 0, -1,
// -1) by the number of differing coordinates, Sec. 5.1 of the FE setting)
// is
//   (A u)_n = h/12 [5 u_n K_n - sum_{e ni n} kappa_e S_e + sum_{6 d} u_{n+d} K_{n,n+d}],
// S_e the sum of u over the 8 nodes of element e. Per plane p a CTA forms,
// for every element position of its tile (33 x 17 with the halo), the sum
// of u over the element's 4 nodes in plane p (PXY), and Q = kappa * S for
// the layer below plane p (S = PXY(p) + PXY(p - 1)), once per element, in
// shared memory; a node takes the 2 x 2 sums of Q of the two layers around
// it (B, one carried from the plane before) and its 6 face neighbours
// weighted by the edge sums. About 19 FP64 operations per node instead of
// the 33 of k_zm3 (the kernel is bound by the FP64 pipe; the 4 node arrays
// of kappa sums, [K_n | K_x | K_y | K_z] per sample, are computed once per
// solve by k_ksum3). Same tiles, chunks, loaders, epilogues and boundary
// rule as k_zm3.
template <class Ld, class Epi>
__global__ void __launch_bounds__(ZTHREADS, 2) k_zm3q(Grid g, const double* __restrict__ Kap,
                                                   const double* __restrict__ Ks, int64_t kss, Ld ld,
                                                   const int32_t* __restrict__ active, Epi epi,
                                                   double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ double sv[3][ZNV];   // field planes with halo (p, p - 1, and the one being refilled)
  __shared__ double sk[2][ZNK];   // kappa layers with halo
  __shared__ double sp[2][ZNK];   // PXY of the plane, per element position
  __shared__ double sq[ZNK];      // Q of the layer below the current plane
  const ZTile t = ztile(g);
  const int n = g.n, N1 = n + 1, P = N1 * N1, KP = n * n;
  const int tid = threadIdx.y * ZTX + threadIdx.x;
  const double* __restrict__ kp = Kap + b * g.es;
  const double* __restrict__ Kn = Ks + b * kss;
  const double* __restrict__ Kx = Kn + g.ns;
  const double* __restrict__ Ky = Kn + 2 * g.ns;
  const double* __restrict__ Kz = Kn + 3 * g.ns;
  ld.bind(b);
  epi.bind(b);
  for (int e = tid; e < ZNK; e += ZTHREADS) sp[1][e] = sk[1][e] = 0.0;
  for (int e = tid; e < ZNV; e += ZTHREADS) sv[2][e] = 0.0;
  int vo[ZSLOTS], ko[ZSLOTS];
  bool vok[ZSLOTS], kok[ZSLOTS], vin[ZSLOTS], kin[ZSLOTS];
#pragma unroll
  for (int q = 0; q < ZSLOTS; ++q) {
    const int sidx = tid + q * ZTHREADS;
    vin[q] = sidx < ZNV;
    kin[q] = sidx < ZNK;
    const int vx = t.tx0 - 1 + sidx % ZSX, vy = t.ty0 - 1 + sidx / ZSX;
    vok[q] = vin[q] && vx >= 1 && vx < n && vy >= 1 && vy < n;
    vo[q] = vok[q] ? vy * N1 + vx : 0;
    const int kx = t.tx0 - 1 + sidx % ZKX, ky = t.ty0 - 1 + sidx / ZKX;
    kok[q] = kin[q] && kx >= 0 && kx < n && ky >= 0 && ky < n;
    ko[q] = kok[q] ? ky * n + kx : 0;
  }
  double rv[ZSLOTS], rk[ZSLOTS];
  auto fetch = [&](int pp) {
    const bool pv = pp >= 1 && pp < n, pk = pp >= 0 && pp < n;
#pragma unroll
    for (int q = 0; q < ZSLOTS; ++q) {
      rv[q] = (pv && vok[q]) ? ld(pp * P + vo[q]) : 0.0;
      rk[q] = (pk && kok[q]) ? __ldg(kp + pp * KP + ko[q]) : 0.0;
    }
  };
  int p = t.z0 - 1;
  fetch(p);

  const int i = t.tx0 + threadIdx.x;
  const int j0 = t.ty0 + ZRY * threadIdx.y;
  bool cvalid[ZRY], cint[ZRY], ey[ZRY];
  int ocol[ZRY];
#pragma unroll
  for (int r = 0; r < ZRY; ++r) {
    const int j = j0 + r;
    cvalid[r] = i <= n && j <= n;
    cint[r] = i >= 1 && i < n && j >= 1 && j < n;
    ey[r] = j == n - 1 && n % ZTY == 0;
    ocol[r] = j * N1 + i;
  }
  const bool ex = i == n - 1 && n % ZTX == 0;
  const double h12 = g.c12;   // h / 12
  // per output row: B of the layer below the current output plane, the
  // centre u and K_z of the plane below it, the kappa sums of the output
  // plane (K_n, K_x(i), K_x(i - 1), K_y(j), K_y(j - 1), K_z) loaded a plane
  // ahead, and the epilogue inputs
  double Bprev[ZRY], ucar[ZRY], kzcar[ZRY], ks[ZRY][6];
  typename Epi::Pre pre[ZRY];
#pragma unroll
  for (int r = 0; r < ZRY; ++r) {
    Bprev[r] = ucar[r] = kzcar[r] = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) ks[r][c] = 0.0;
  }
  double dot = 0.0;
  const int vbase = (ZRY * threadIdx.y + 1) * ZSX + threadIdx.x + 1;   // node (i, j0)
  const int kbase = ZRY * threadIdx.y * ZKX + threadIdx.x;             // element (i - 1, j0 - 1)
  // sv: plane p in sv[cur], plane p - 1 in sv[prv]; a buffer is refilled
  // two steps after its last read, with the barriers of a step between
  int buf = 0, cur = 0, prv = 2;
  for (; p <= t.z1; ++p) {
    double* svb = sv[cur];
    double* skb = sk[buf];
#pragma unroll
    for (int q = 0; q < ZSLOTS; ++q) {
      if (vin[q]) svb[tid + q * ZTHREADS] = rv[q];
      if (kin[q]) skb[tid + q * ZTHREADS] = rk[q];
    }
    __syncthreads();   // plane p and kappa layer p staged
    if (p < t.z1) fetch(p + 1);
    // kappa sums and epilogue inputs of plane p (an output plane at the next step)
    typename Epi::Pre nxt[ZRY];
    double kn[ZRY][6];
#pragma unroll
    for (int r = 0; r < ZRY; ++r) {
      const bool out = cint[r] && p >= 1 && p < n;
      if (out && p >= t.z0 && p < t.z1) nxt[r] = epi.load(p * P + ocol[r]);
      const int o = p * P + ocol[r];
      kn[r][0] = out ? __ldg(Kn + o) : 0.0;
      kn[r][1] = out ? __ldg(Kx + o) : 0.0;
      kn[r][2] = out ? __ldg(Kx + o - 1) : 0.0;
      kn[r][3] = out ? __ldg(Ky + o) : 0.0;
      kn[r][4] = out ? __ldg(Ky + o - N1) : 0.0;
      kn[r][5] = (cint[r] && p >= 0 && p < n) ? __ldg(Kz + o) : 0.0;
    }
    // element sums of plane p and Q of layer p - 1, once per element position
    const double* svo = sv[prv];
    for (int e = tid; e < ZNK; e += ZTHREADS) {
      const int ex_ = e % ZKX, ey_ = e / ZKX;
      const double* v = svb + ey_ * ZSX + ex_;
      const double pxy = (v[0] + v[1]) + (v[ZSX] + v[ZSX + 1]);
      sq[e] = sk[buf ^ 1][e] * (pxy + sp[buf ^ 1][e]);
      sp[buf][e] = pxy;
    }
    __syncthreads();   // Q of layer p - 1 complete
    const int m = p - 1;
    // Q x-pair sums of the element rows j0 - 1 .. j0 + ZRY - 1 at columns i - 1, i
    double qx[ZRY + 1];
#pragma unroll
    for (int r = 0; r <= ZRY; ++r) qx[r] = sq[kbase + r * ZKX] + sq[kbase + r * ZKX + 1];
#pragma unroll
    for (int r = 0; r < ZRY; ++r) {
      const double Bcur = qx[r] + qx[r + 1];
      const double* v = svo + vbase + r * ZSX;   // node (i, j0 + r) of plane m
      const double uc = v[0];
      if (cvalid[r] && m >= t.z0) {
        const int o = m * P + ocol[r];
        const bool in = cint[r] && m >= 1 && m < n;
        double acc = 0.0;
        if (in) {
          // the six face neighbours by their edge sums, then 5 u K_n - sum kappa_e S_e
          double sx = ks[r][1] * v[1];
          sx = fma(ks[r][2], v[-1], sx);
          sx = fma(ks[r][3], v[ZSX], sx);
          sx = fma(ks[r][4], v[-ZSX], sx);
          sx = fma(ks[r][5], svb[vbase + r * ZSX], sx);
          sx = fma(kzcar[r], ucar[r], sx);
          sx = fma(5.0 * uc, ks[r][0], sx);
          acc = sx - (Bprev[r] + Bcur);
        }
        double done;
        if constexpr (Epi::kRes) done = fma(-h12, acc, epi.rhs(pre[r]));
        else done = h12 * acc;
        dot += epi(o, in, done, uc, pre[r]);
        if (ex) epi.zero(o + 1);
        if (ey[r]) epi.zero(o + N1);
        if (ex && ey[r]) epi.zero(o + N1 + 1);
      }
      Bprev[r] = Bcur;
      ucar[r] = uc;
      kzcar[r] = ks[r][5];
#pragma unroll
      for (int c = 0; c < 6; ++c) ks[r][c] = kn[r][c];
      pre[r] = nxt[r];
    }
    buf ^= 1;
    prv = cur;
    cur = cur == 2 ? 0 : cur + 1;
  }
  if (part) cta_partial3(dot, part, g.tiles_s);
  prof_tick3(prof);
}

// Kappa sums of every node (0 outside the mesh), per sample [K_n | K_x | K_y
// | K_z] in node strides: K_n the 8 elements around the node, K_x the 4
// elements sharing the edge to the +x neighbour (element column i, rows j-1
// and j, layers k-1 and k), K_y and K_z likewise. Once per solve.
__global__ void __launch_bounds__(256) k_ksum3(Grid g, const double* __restrict__ K, double* __restrict__ Ks,
                                               int64_t kss, int pz) {
  const int64_t b = blockIdx.y;
  const NodeCol c = node_col3(g.n, pz);
  if (!c.valid) return;
  const int n = g.n, N1 = n + 1;
  const double* k = K + b * g.es;
  double* kn = Ks + b * kss;
  auto el = [&](int z, int y, int x) -> double {
    return (z >= 0 && z < n && y >= 0 && y < n && x >= 0 && x < n) ? __ldg(k + ((int64_t)z * n + y) * n + x) : 0.0;
  };
  // per element layer z, around this node column: L = the 4 elements, X =
  // the 2 elements of row j (x-pair, for K_y), Y = the 2 of column i
  // (y-pair, for K_x); a node adds the sums of the layers below and above
  auto layer = [&](int z, double& L, double& X, double& Y) {
    const double a = el(z, c.j - 1, c.i - 1), bq = el(z, c.j - 1, c.i);
    const double cq = el(z, c.j, c.i - 1), d = el(z, c.j, c.i);
    X = cq + d;
    Y = bq + d;
    L = (a + bq) + X;
  };
  double L0, X0, Y0;
  layer(c.k0 - 1, L0, X0, Y0);
  for (int kz = c.k0; kz < c.k1; ++kz) {
    double L1, X1, Y1;
    layer(kz, L1, X1, Y1);
    const int64_t o = ((int64_t)kz * N1 + c.j) * N1 + c.i;
    kn[o] = L0 + L1;
    kn[g.ns + o] = Y0 + Y1;
    kn[2 * g.ns + o] = X0 + X1;
    kn[3 * g.ns + o] = L1;
    L0 = L1;
    X0 = X1;
    Y0 = Y1;
  }
}

// Loaders: the value the stencil acts on at an interior node, formed while
// the plane is staged (bind(sample) offsets the arrays to the sample), so a
// pointwise pre-pass is not needed.
template <class T>
struct LdX {   // x
  const T* x;
  int64_t ns;
  __device__ void bind(int64_t b) { x += b * ns; }
  __device__ T operator()(int o) const { return __ldg(x + o); }
};

template <class T>
struct LdPupd {   // the new CG direction z + beta p (beta == 0: z)
  const T* z;
  const T* pold;
  const double* beta;
  int64_t ns;
  T bb;
  __device__ void bind(int64_t b) {
    z += b * ns;
    pold += b * ns;
    bb = (T)beta[b];
  }
  __device__ T operator()(int o) const {
    const T zv = __ldg(z + o);
    return bb == T(0) ? zv : fma(bb, __ldg(pold + o), zv);
  }
};

template <class T>
struct LdWb {   // the pre-smoothed iterate from zero: omega D^-1 b
  const T* W;
  const T* Bv;
  int64_t ns;
  __device__ void bind(int64_t b) {
    W += b * ns;
    Bv += b * ns;
  }
  __device__ T operator()(int o) const { return __ldg(W + o) * __ldg(Bv + o); }
};

// Epilogues: bind(sample) offsets their arrays to the sample; load(node)
// fetches the node's own inputs (Pre) one plane ahead; then (node offset,
// interior?, y, x at the node, Pre) -> contribution to the CTA partial;
// zero() writes a boundary node. y is (A x) at the node, or, for an epilogue
// with kRes (the FP64 residual forms, k_zm3 only), f - (A x) with f =
// rhs(Pre): the FP64 kernel then folds f into its last two FMAs instead of a
// multiply, an FMA and a subtraction.
struct NoPre {};


template <class T>
struct EpiApply {   // y = A x
  using Pre = NoPre;
  static constexpr bool kRes = false;
  __device__ T rhs(const Pre&) const { return T(0); }
  T* Y;
  int64_t ns;
  __device__ void bind(int64_t b) { Y += b * ns; }
  __device__ Pre load(int) const { return Pre{}; }
  __device__ T operator()(int o, bool in, T ax, T, const Pre&) const {
    Y[o] = in ? ax : T(0);
    return T(0);
  }
  __device__ void zero(int o) const { Y[o] = T(0); }
};

template <class T>
struct EpiAq {   // q = A p, partial of p.q; p itself stored (Pn) when formed by the loader
  using Pre = NoPre;
  static constexpr bool kRes = false;
  __device__ T rhs(const Pre&) const { return T(0); }
  T* Q;
  T* Pn;
  int64_t ns;
  __device__ void bind(int64_t b) {
    Q += b * ns;
    if (Pn) Pn += b * ns;
  }
  __device__ Pre load(int) const { return Pre{}; }
  __device__ T operator()(int o, bool in, T ax, T xc, const Pre&) const {
    const T qv = in ? ax : T(0);
    Q[o] = qv;
    if (Pn) Pn[o] = in ? xc : T(0);
    return xc * qv;
  }
  __device__ void zero(int o) const {
    Q[o] = T(0);
    if (Pn) Pn[o] = T(0);
  }
};

template <class T>
struct PreB {
  T b;
};

template <class T>
struct EpiMgRes {   // residual of the pre-smoothed iterate: b - A e; e stored (E) when formed by the loader
  using Pre = PreB<T>;
  static constexpr bool kRes = sizeof(T) == 8;
  __device__ T rhs(const Pre& pr) const { return pr.b; }
  const T* Bv;
  T* R1;
  T* E;
  int64_t ns;
  __device__ void bind(int64_t b) {
    Bv += b * ns;
    R1 += b * ns;
    if (E) E += b * ns;
  }
  __device__ Pre load(int o) const { return Pre{__ldg(Bv + o)}; }
  __device__ T operator()(int o, bool in, T y, T xc, const Pre& pr) const {
    R1[o] = in ? (kRes ? y : pr.b - y) : T(0);
    if (E) E[o] = in ? xc : T(0);
    return T(0);
  }
  __device__ void zero(int o) const {
    R1[o] = T(0);
    if (E) E[o] = T(0);
  }
};

template <class T>
struct PreBW {
  T b, w;
};

template <class T>
struct EpiMgPost {   // post-smoothing: e + W (b - A e), partial of b.out
  using Pre = PreBW<T>;
  static constexpr bool kRes = sizeof(T) == 8;
  __device__ T rhs(const Pre& pr) const { return pr.b; }
  const T* W;
  const T* Bv;
  T* Out;
  int64_t ns;
  __device__ void bind(int64_t b) {
    W += b * ns;
    Bv += b * ns;
    Out += b * ns;
  }
  __device__ Pre load(int o) const { return Pre{__ldg(Bv + o), __ldg(W + o)}; }
  __device__ T operator()(int o, bool in, T y, T ec, const Pre& pr) const {
    const T ov = in ? fma(pr.w, kRes ? y : pr.b - y, ec) : T(0);
    Out[o] = ov;
    return in ? pr.b * ov : T(0);
  }
  __device__ void zero(int o) const { Out[o] = T(0); }
};

struct EpiResid {   // outer FP64 residual h^3 - A u, partial of its square
  using Pre = NoPre;
  static constexpr bool kRes = true;
  double* R;
  int64_t ns;
  double h3;
  __device__ double rhs(const Pre&) const { return h3; }
  __device__ void bind(int64_t b) { R += b * ns; }
  __device__ Pre load(int) const { return Pre{}; }
  __device__ double operator()(int o, bool in, double rv_in, double, const Pre&) const {
    const double rv = in ? rv_in : 0.0;
    R[o] = rv;
    return rv * rv;
  }
  __device__ void zero(int o) const { R[o] = 0.0; }
};

// ------------------------------------------------ FP32 z-march, packed pairs
//
// The FP32 form of k_zm3 on Blackwell's paired FP32 instructions (FFMA2 and
// friends, __ffma2_rn / __fadd2_rn / __fmul2_rn): a thread owns rows j and
// j + 8 of one column of the 32 x 16 tile, and shared memory holds each
// staged plane as pairs (value at row r, value at row r + 8), so one 64-bit
// shared load brings the same neighbour of both outputs and every stencil
// operation serves both. Same tile, chunks, boundary rule and epilogues as
// k_zm3.
constexpr int ZPY = ZTY / 2 + 2, ZNVP = ZSX * ZPY;   // 34 x 10 pairs
constexpr int ZKPY = ZTY / 2 + 1, ZNKP = ZKX * ZKPY; // 33 x 9 pairs
static_assert(ZNVP <= 2 * ZTHREADS && ZNKP <= 2 * ZTHREADS, "two paired staging slots per thread");

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Asynchronous 4-byte global -> shared copy to a shared-window address
// (zero-filled when src_bytes = 0).
__device__ __forceinline__ void cp_async4s(unsigned sa, const void* gmem, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int ZSTAGES = 4;   // planes in flight: the current one and ZSTAGES - 1 ahead

// Paired FP32 loaders for k_zm3f: kArrays node arrays are staged per plane
// and combined pairwise into the field once the plane has arrived.
struct LdXf {   // x
  static constexpr int kArrays = 1;
  const float* a0;
  int64_t ns;
  __device__ void bind(int64_t b) { a0 += b * ns; }
  __device__ const float* src(int) const { return a0; }
  __device__ float2 combine(float2 x, float2) const { return x; }
  __device__ float combine1(float x, float) const { return x; }
  bool aligned16() const { return ((uintptr_t)a0 & 15) == 0; }
};

struct LdPupdf {   // z + beta p (beta == 0: z)
  static constexpr int kArrays = 2;
  const float* z;
  const float* pold;
  const double* beta;
  int64_t ns;
  float bb;
  __device__ void bind(int64_t b) {
    z += b * ns;
    pold += b * ns;
    bb = (float)beta[b];
  }
  __device__ const float* src(int k) const { return k ? pold : z; }
  __device__ float2 combine(float2 zv, float2 pv) const {
    return bb == 0.0f ? zv : fma2(make_float2(bb, bb), pv, zv);
  }
  __device__ float combine1(float zv, float pv) const { return bb == 0.0f ? zv : fmaf(bb, pv, zv); }
  bool aligned16() const { return (((uintptr_t)z | (uintptr_t)pold) & 15) == 0; }
};

struct LdWbf {   // omega D^-1 b
  static constexpr int kArrays = 2;
  const float* W;
  const float* Bv;
  int64_t ns;
  __device__ void bind(int64_t b) {
    W += b * ns;
    Bv += b * ns;
  }
  __device__ const float* src(int k) const { return k ? Bv : W; }
  __device__ float2 combine(float2 w, float2 bv) const { return mul2(w, bv); }
  __device__ float combine1(float w, float bv) const { return w * bv; }
  bool aligned16() const { return (((uintptr_t)W | (uintptr_t)Bv) & 15) == 0; }
};

template <class Ld>
struct LdPaired;
template <>
struct LdPaired<LdX<float>> {
  using type = LdXf;
  static LdXf make(const LdX<float>& l) { return LdXf{l.x, l.ns}; }
};
template <>
struct LdPaired<LdPupd<float>> {
  using type = LdPupdf;
  static LdPupdf make(const LdPupd<float>& l) { return LdPupdf{l.z, l.pold, l.beta, l.ns, 0.0f}; }
};
template <>
struct LdPaired<LdWb<float>> {
  using type = LdWbf;
  static LdWbf make(const LdWb<float>& l) { return LdWbf{l.W, l.Bv, l.ns}; }
};

template <class Ld, class Epi>
__global__ void __launch_bounds__(ZTHREADS, 2) k_zm3f(Grid g, const float* __restrict__ Kap, Ld ld,
                                                      const int32_t* __restrict__ active, Epi epi,
                                                      double* __restrict__ part, Prof prof) {
  static_assert(!Epi::kRes, "the FP32 z-march hands A x to its epilogues");
  constexpr int NA = Ld::kArrays;
  const int64_t b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ __align__(16) float2 sv[ZSTAGES][NA][ZNVP];
  __shared__ __align__(16) float2 sk[ZSTAGES][ZNKP];
  const ZTile t = ztile(g);
  const int n = g.n, N1 = n + 1, P = N1 * N1, KP = n * n;
  const int tid = threadIdx.y * ZTX + threadIdx.x;
  const float* __restrict__ kp = Kap + b * g.es;
  ld.bind(b);
  epi.bind(b);
  // copy slots: pair entries tid and tid + 256; entry (xx, yy) holds rows
  // r = ty0 - 1 + yy and r + 8 of column tx0 - 1 + xx
  int vo[2][2], ko[2][2];
  bool vok[2][2], kok[2][2], vin[2], kin[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = tid + q * ZTHREADS;
    vin[q] = e < ZNVP;
    kin[q] = e < ZNKP;
    const int vx = t.tx0 - 1 + e % ZSX, vy = t.ty0 - 1 + e / ZSX;
    const int kx = t.tx0 - 1 + e % ZKX, ky = t.ty0 - 1 + e / ZKX;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ry = vy + 8 * h, rk = ky + 8 * h;
      vok[q][h] = vin[q] && vx >= 1 && vx < n && ry >= 1 && ry < n;
      vo[q][h] = vok[q][h] ? ry * N1 + vx : 0;
      kok[q][h] = kin[q] && kx >= 0 && kx < n && rk >= 0 && rk < n;
      ko[q][h] = kok[q][h] ? rk * n + kx : 0;
    }
  }
  // stage plane pp into ring slot st (one commit group per plane; empty
  // groups past the chunk keep the group count uniform)
  // shared addresses of this thread's copy slots in ring slot 0 (slot st is
  // st * stage bytes further); global reads of masked slots point at a plane
  // inside the sample and copy 0 bytes
  const unsigned sv0 = (unsigned)__cvta_generic_to_shared(&sv[0][0][0]);
  const unsigned sk0 = (unsigned)__cvta_generic_to_shared(&sk[0][0]);
  constexpr unsigned SV_ARR = ZNVP * 8, SV_STAGE = NA * ZNVP * 8, SK_STAGE = ZNKP * 8;
  auto issue = [&](int pp, int st) {
    if (pp <= t.z1) {
      const bool pv = pp >= 1 && pp < n, pk = pp >= 0 && pp < n;
      const int pc = min(max(pp, 0), n - 1);
      const unsigned svs = sv0 + st * SV_STAGE, sks = sk0 + st * SK_STAGE;
      const float* kpl = kp + pc * KP;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const unsigned e8 = (unsigned)(tid + q * ZTHREADS) * 8u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (vin[q]) {
#pragma unroll
            for (int a = 0; a < NA; ++a)
              cp_async4s(svs + a * SV_ARR + e8 + 4u * h, ld.src(a) + pc * P + vo[q][h],
                         (pv && vok[q][h]) ? 4 : 0);
          }
          if (kin[q]) cp_async4s(sks + e8 + 4u * h, kpl + ko[q][h], (pk && kok[q][h]) ? 4 : 0);
        }
      }
    }
    cp_async_commit();
  };
  int p = t.z0 - 1;
#pragma unroll
  for (int j = 0; j < ZSTAGES - 1; ++j) issue(p + j, j);

  const int i = t.tx0 + threadIdx.x;
  const int jr[2] = {t.ty0 + (int)threadIdx.y, t.ty0 + (int)threadIdx.y + 8};
  bool cvalid[2], cint[2], ey[2];
  int ocol[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    cvalid[r] = i <= n && jr[r] <= n;
    cint[r] = i >= 1 && i < n && jr[r] >= 1 && jr[r] < n;
    ey[r] = jr[r] == n - 1 && n % ZTY == 0;
    ocol[r] = jr[r] * N1 + i;
  }
  const bool ex = i == n - 1 && n % ZTX == 0;
  const float c3s = (float)g.c3, c12s = (float)g.c12;
  const float2 c3 = make_float2(c3s, c3s), mc12 = make_float2(-c12s, -c12s);
  // as in k_zm3: U unscaled couplings and D diagonal part of the output of
  // plane p - 1, N couplings of the output of plane p with plane p - 1; the
  // kappa pair sums of a layer (X along x, Y along y, S of the 4 elements)
  // are formed once and reused for the next plane
  const float2 z2 = make_float2(0.f, 0.f);
  float2 U = z2, D = z2, Nn = z2, vc = z2;
  float2 kb[2][2] = {{z2, z2}, {z2, z2}};
  float2 Xb[2] = {z2, z2}, Yb[2] = {z2, z2}, Sb = z2;
  typename Epi::Pre pre[2];
  float dot = 0.0f;
  const int vbase = (threadIdx.y + 1) * ZSX + threadIdx.x + 1;
  const int kbase = threadIdx.y * ZKX + threadIdx.x;
  int st = 0;
  for (; p <= t.z1; ++p) {
    cp_async_wait<ZSTAGES - 2>();   // this thread's copies of plane p have landed
    if (NA > 1) {                   // combine this thread's entries into the field
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (vin[q]) {
          const int e = tid + q * ZTHREADS;
          sv[st][0][e] = ld.combine(sv[st][0][e], sv[st][NA - 1][e]);
        }
    }
    __syncthreads();                // plane p complete; slot of plane p - 1 free
    issue(p + ZSTAGES - 1, (st + ZSTAGES - 1) % ZSTAGES);
    typename Epi::Pre nxt[2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
      if (cint[r] && p >= t.z0 && p < t.z1 && p >= 1 && p < n) nxt[r] = epi.load(p * P + ocol[r]);
    const float2* svb = sv[st][0];
    const float2* skb = sk[st];
    float2 v[3][3], ka[2][2];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) v[dy][dx] = svb[vbase + (dy - 1) * ZSX + (dx - 1)];
#pragma unroll
    for (int bq = 0; bq < 2; ++bq)
#pragma unroll
      for (int a = 0; a < 2; ++a) ka[bq][a] = skb[kbase + bq * ZKX + a];
    float2 Xa[2], Ya[2];
    Xa[0] = add2(ka[0][0], ka[0][1]);
    Xa[1] = add2(ka[1][0], ka[1][1]);
    Ya[0] = add2(ka[0][0], ka[1][0]);
    Ya[1] = add2(ka[0][1], ka[1][1]);
    const float2 Sa = add2(Xa[0], Xa[1]);
    // outputs of plane p - 1 are complete: couplings with plane p across layer p - 1
    float2 u = fma2(Yb[0], v[1][0], U);
    u = fma2(Yb[1], v[1][2], u);
    u = fma2(Xb[0], v[0][1], u);
    u = fma2(Xb[1], v[2][1], u);
    u = fma2(kb[0][0], v[0][0], u);
    u = fma2(kb[0][1], v[0][2], u);
    u = fma2(kb[1][0], v[2][0], u);
    u = fma2(kb[1][1], v[2][2], u);
    const float2 done = fma2(mc12, u, mul2(c3, D));
    const int m = p - 1;
    if (m >= t.z0) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (!cvalid[r]) continue;
        const int o = m * P + ocol[r];
        dot += epi(o, cint[r] && m >= 1 && m < n, r ? done.y : done.x, r ? vc.y : vc.x, pre[r]);
        if (ex) epi.zero(o + 1);
        if (ey[r]) epi.zero(o + N1);
        if (ex && ey[r]) epi.zero(o + N1 + 1);
      }
    }
    // output p: couplings with plane p - 1 and the in-plane diagonal edges
    u = fma2(add2(kb[0][0], ka[0][0]), v[0][0], Nn);
    u = fma2(add2(kb[0][1], ka[0][1]), v[0][2], u);
    u = fma2(add2(kb[1][0], ka[1][0]), v[2][0], u);
    U = fma2(add2(kb[1][1], ka[1][1]), v[2][2], u);
    D = mul2(add2(Sb, Sa), v[1][1]);
    // output p + 1: couplings with plane p across layer p
    u = mul2(Ya[0], v[1][0]);
    u = fma2(Ya[1], v[1][2], u);
    u = fma2(Xa[0], v[0][1], u);
    u = fma2(Xa[1], v[2][1], u);
    u = fma2(ka[0][0], v[0][0], u);
    u = fma2(ka[0][1], v[0][2], u);
    u = fma2(ka[1][0], v[2][0], u);
    Nn = fma2(ka[1][1], v[2][2], u);
#pragma unroll
    for (int bq = 0; bq < 2; ++bq)
#pragma unroll
      for (int a = 0; a < 2; ++a) kb[bq][a] = ka[bq][a];
    Xb[0] = Xa[0];
    Xb[1] = Xa[1];
    Yb[0] = Ya[0];
    Yb[1] = Ya[1];
    Sb = Sa;
    vc = v[1][1];
    pre[0] = nxt[0];
    pre[1] = nxt[1];
    st = (st + 1) % ZSTAGES;
  }
  cp_async_wait<0>();
  if (part) cta_partial3((double)dot, part, g.tiles_s);
  prof_tick3(prof);
}

// ------------------------------------ FP32 z-march, TMA bulk-copy staging
//
// k_zm3w is k_zm3f with its planes staged by the copy engine instead of by
// per-element cp.async, for the meshes with n in {32, 64, 128, 256}: a CTA
// covers the full width of the mesh (n threads across x, one column each)
// and R = 256 RT / n node rows, RT rows per thread (RT = 2: the CTAs per
// sample are those of the 32 x 16 tiles; RT = 4: half as many, each
// covering two of them), so the halo slab of a plane (rows ty0 - 1 ..
// ty0 + R, every column) is one contiguous range of a node array; the kappa
// slab (rows ty0 - 1 .. ty0 + R - 1) is one contiguous range of an element
// array. Each plane of each array is then ONE asynchronous bulk copy
// (cp.async.bulk, global -> shared, completing on the slot's mbarrier),
// issued by one thread: no per-element address, predicate or register work.
// Node rows have an odd pitch n + 1, so a slab starts sh = (offset mod 4)
// floats past a 16-byte boundary; the copy starts at that boundary and lands
// at a slot offset that keeps the destination 16-byte aligned, which shifts
// the slab by OFF (0..3 floats, one value per plane) inside the slot.
// Values that feed only boundary outputs (row -1, column -1, the kappa halo
// and the layers -1 and n) may be stale; planes 0 and n are not copied, and
// the boundary nodes of the field (rows, columns and planes 0 and n) are
// read as 0 by the threads next to them, whatever the array holds there.
// A thread's RT rows are RT / 2 float2 pairs of consecutive rows. Waits are
// bounded: a wait that gives up counts a timeout in g_zt_timeouts (read by
// the host at its sync points), lets the copies still in flight land
// (bounded again) and ends the CTA.
constexpr int ZW_S = 4;                             // ring slots, ZW_S - 1 planes in flight
constexpr int ZW_WAIT_TRIES = 1 << 22;              // bounded waits: tries and SM cycles (~2 s)
constexpr long long ZW_WAIT_CYCLES = 1ll << 32;

// rows per CTA and slot sizes (floats) of a node slab and of a kappa slab
// for cells per side n and rows per thread rt
__host__ __device__ constexpr int zw_rows(int n, int rt) { return 256 * rt / n; }
__host__ __device__ constexpr int zw_vslot(int n, int rt) {
  return (12 + (zw_rows(n, rt) + 2) * (n + 1) + 3) / 4 * 4;
}
__host__ __device__ constexpr int zw_kslot(int n, int rt) { return (8 + (zw_rows(n, rt) + 1) * n + 3) / 4 * 4; }
inline bool zw_mesh(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }

__device__ unsigned int g_zt_timeouts;

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(addr), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of phase `parity`; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity) {
  if (mbar_try_wait(addr, parity)) return true;
  const long long t0 = clock64();
  for (int k = 0; k < ZW_WAIT_TRIES; ++k) {
    if (mbar_try_wait(addr, parity)) return true;
    if (clock64() - t0 > ZW_WAIT_CYCLES) break;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

template <class Ld, class Epi, int RT>
__global__ void __launch_bounds__(ZTHREADS, RT == 2 ? 3 : 2) k_zm3w(Grid g, const float* __restrict__ Kap, Ld ld,
                                                                   const int32_t* __restrict__ active, Epi epi,
                                                                   double* __restrict__ part, Prof prof) {
  static_assert(!Epi::kRes, "the FP32 z-march hands A x to its epilogues");
  static_assert(RT == 2 || RT == 4, "two or four rows per thread");
  constexpr int NA = Ld::kArrays;
  constexpr int NP = RT / 2;   // float2 row pairs per thread
  const int64_t b = blockIdx.y;
  if (active && !active[b]) return;
  extern __shared__ __align__(16) float zw_smem[];
  const int n = g.n, N1 = n + 1, P = N1 * N1, KPn = n * n;
  const int R = zw_rows(n, RT), VS = zw_vslot(n, RT), KS = zw_kslot(n, RT), SS = NA * VS + KS;
  float* ring = zw_smem;                                              // ZW_S slots of SS floats
  unsigned long long* sbar = reinterpret_cast<unsigned long long*>(zw_smem + ZW_S * SS);
  __shared__ double s_w[ZTHREADS / 32];
  const int tyn = n / R;
  int t = blockIdx.x;
  const int zq = t / tyn;
  const int ty0 = (t - zq * tyn) * R;
  const int z0 = zq * g.zc, z1 = min(z0 + g.zc, n + 1);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const float* __restrict__ kp = Kap + b * g.es;
  ld.bind(b);
  epi.bind(b);
  for (int e = tid; e < ZW_S * SS / 4; e += ZTHREADS)
    reinterpret_cast<float4*>(ring)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  const unsigned bar0 = (unsigned)__cvta_generic_to_shared(sbar);
  const unsigned ring0 = (unsigned)__cvta_generic_to_shared(ring);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < ZW_S; ++s) mbar_init(bar0 + 8u * s, 1u);
    fence_mbar_init();
  }
  fence_proxy_async_smem();
  __syncthreads();

  // slabs: node rows ylo..yhi of a plane, kappa rows kylo..ty0 + R - 1 of a layer
  const int ylo = max(ty0 - 1, 0), yhi = min(ty0 + R, n), r0 = ylo - ty0 + 1;
  const int kylo = max(ty0 - 1, 0), kr0 = kylo - ty0 + 1;
  const unsigned kbytes = 4u * (unsigned)((ty0 + R - kylo) * n);
  // shift of plane pp's slab inside its slot (the slab's 16-byte alignment)
  auto voff = [&](int pp) {
    const int sh = (pp * P + ylo * N1) & 3;
    return (sh - r0 * N1) & 3;
  };
  // stage plane pp (field) and layer pp (kappa) into slot st: one bulk copy per array
  auto issue = [&](int pp, int st) {
    if (tid != 0) return;
    const bool pv = pp >= 1 && pp < n, pk = pp >= 0 && pp < n;
    const unsigned bar = bar0 + 8u * st;
    const int G0 = pp * P + ylo * N1, G1 = pp * P + (yhi + 1) * N1;
    const int Ga = G0 & ~3, Gb = (G1 + 3) & ~3;
    const unsigned vbytes = 4u * (unsigned)(Gb - Ga);
    mbar_arrive_tx(bar, (pv ? NA * vbytes : 0u) + (pk ? kbytes : 0u));
    if (pv) {
      const int dst = 4 + voff(pp) + r0 * N1 - (G0 - Ga);
#pragma unroll
      for (int a = 0; a < NA; ++a)
        bulk_g2s(ring0 + 4u * (unsigned)(st * SS + a * VS + dst), ld.src(a) + Ga, vbytes, bar);
    }
    if (pk)
      bulk_g2s(ring0 + 4u * (unsigned)(st * SS + NA * VS + 4 + kr0 * n), kp + (pp * KPn + kylo * n), kbytes,
               bar);
  };

  int p = z0 - 1;
  unsigned pend = 0;   // slots with copies issued and not yet waited for
#pragma unroll
  for (int j = 0; j < ZW_S - 1; ++j)
    if (p + j <= z1) {
      issue(p + j, j);
      pend |= 1u << j;
    }

  const int i = threadIdx.x;
  const int jr0 = ty0 + RT * (int)threadIdx.y;   // this thread's rows jr0 .. jr0 + RT - 1
  bool cint[RT], ey[RT];
  int ocol[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    cint[r] = i >= 1 && i < n && jr0 + r >= 1 && jr0 + r < n;
    ey[r] = jr0 + r == n - 1;
    ocol[r] = (jr0 + r) * N1 + i;
  }
  const bool ex = i == n - 1;
  // field boundary nodes next to this thread's stencils (columns i - 1 .. i + 1,
  // rows jr0 - 1 .. jr0 + RT) read as 0
  bool cok[3], rok[RT + 2];
#pragma unroll
  for (int dx = 0; dx < 3; ++dx) cok[dx] = i - 1 + dx >= 1 && i - 1 + dx <= n - 1;
#pragma unroll
  for (int r = 0; r < RT + 2; ++r) rok[r] = jr0 - 1 + r >= 1 && jr0 - 1 + r <= n - 1;
  const bool edge = !(cok[0] && cok[2] && rok[0] && rok[RT + 1]);
  const float c3s = (float)g.c3, c12s = (float)g.c12;
  const float2 c3 = make_float2(c3s, c3s), mc12 = make_float2(-c12s, -c12s);
  const float2 z2 = make_float2(0.f, 0.f);
  // per row pair q (rows jr0 + 2q, jr0 + 2q + 1), as in k_zm3f: U unscaled
  // couplings and D diagonal part of the output of plane p - 1, N couplings
  // of the output of plane p with plane p - 1, the kappa pair sums of the
  // layer below (X along x, Y along y, S of the 4 elements)
  float2 U[NP], D[NP], Nn[NP], vc[NP], kb[NP][2][2], Xb[NP][2], Yb[NP][2], Sb[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    U[q] = D[q] = Nn[q] = vc[q] = Sb[q] = z2;
    kb[q][0][0] = kb[q][0][1] = kb[q][1][0] = kb[q][1][1] = z2;
    Xb[q][0] = Xb[q][1] = Yb[q][0] = Yb[q][1] = z2;
  }
  typename Epi::Pre pre[RT];
  float dot = 0.0f;
  const int vrow = 4 + RT * (int)threadIdx.y * N1 + i - 1;    // + OFF: row jr0 - 1, column i - 1
  const int krow = 4 + RT * (int)threadIdx.y * n + i - 1;     // row jr0 - 1, element i - 1
  int st = 0;
  unsigned par = 0;    // phase parity of each slot's next completion
  bool timed_out = false;
#pragma unroll 2
  for (; p <= z1; ++p) {
    const bool landed = mbar_wait(bar0 + 8u * st, (par >> st) & 1u);
    if (landed) {
      pend &= ~(1u << st);
      par ^= 1u << st;
    }
    float* slot = ring + st * SS;
    if (NA > 1 && landed && p >= 1 && p < n) {   // combine the arrays into the field
      for (int e = tid; e < VS; e += ZTHREADS) slot[e] = ld.combine1(slot[e], slot[VS + e]);
    }
    fence_proxy_async_smem();       // this thread's shared-memory writes before later copies
    // plane p complete; the slot of plane p - 1 is free (or a wait gave up:
    // every thread leaves the loop together)
    if (__syncthreads_or(!landed)) {
      timed_out = true;
      break;
    }
    if (p + ZW_S - 1 <= z1) {
      const int sn = (st + ZW_S - 1) % ZW_S;
      issue(p + ZW_S - 1, sn);
      pend |= 1u << sn;
    }
    typename Epi::Pre nxt[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r)
      if (cint[r] && p >= z0 && p < z1 && p >= 1 && p < n) nxt[r] = epi.load(p * P + ocol[r]);
    const float* svb = slot + voff(p) + vrow;
    const float* skb = slot + NA * VS + krow;
    float sv[RT + 2][3], kv[RT + 1][2];
#pragma unroll
    for (int r = 0; r < RT + 2; ++r)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) sv[r][dx] = svb[r * N1 + dx];
#pragma unroll
    for (int r = 0; r < RT + 1; ++r)
#pragma unroll
      for (int a = 0; a < 2; ++a) kv[r][a] = skb[r * n + a];
    if (p <= 0 || p >= n) {
#pragma unroll
      for (int r = 0; r < RT + 2; ++r)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) sv[r][dx] = 0.f;
    } else if (edge) {
#pragma unroll
      for (int r = 0; r < RT + 2; ++r)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
          if (!rok[r] || !cok[dx]) sv[r][dx] = 0.f;
    }
    const int m = p - 1;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      float2 v[3][3], ka[2][2];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) v[dy][dx] = make_float2(sv[2 * q + dy][dx], sv[2 * q + dy + 1][dx]);
#pragma unroll
      for (int bq = 0; bq < 2; ++bq)
#pragma unroll
        for (int a = 0; a < 2; ++a) ka[bq][a] = make_float2(kv[2 * q + bq][a], kv[2 * q + bq + 1][a]);
      float2 Xa[2], Ya[2];
      Xa[0] = add2(ka[0][0], ka[0][1]);
      Xa[1] = add2(ka[1][0], ka[1][1]);
      Ya[0] = add2(ka[0][0], ka[1][0]);
      Ya[1] = add2(ka[0][1], ka[1][1]);
      const float2 Sa = add2(Xa[0], Xa[1]);
      // outputs of plane p - 1 are complete: couplings with plane p across layer p - 1
      float2 u = fma2(Yb[q][0], v[1][0], U[q]);
      u = fma2(Yb[q][1], v[1][2], u);
      u = fma2(Xb[q][0], v[0][1], u);
      u = fma2(Xb[q][1], v[2][1], u);
      u = fma2(kb[q][0][0], v[0][0], u);
      u = fma2(kb[q][0][1], v[0][2], u);
      u = fma2(kb[q][1][0], v[2][0], u);
      u = fma2(kb[q][1][1], v[2][2], u);
      const float2 done = fma2(mc12, u, mul2(c3, D[q]));
      if (m >= z0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 2 * q + h;
          const int o = m * P + ocol[r];
          dot += epi(o, cint[r] && m >= 1 && m < n, h ? done.y : done.x, h ? vc[q].y : vc[q].x, pre[r]);
          if (ex) epi.zero(o + 1);
          if (ey[r]) epi.zero(o + N1);
          if (ex && ey[r]) epi.zero(o + N1 + 1);
        }
      }
      // output p: couplings with plane p - 1 and the in-plane diagonal edges
      u = fma2(add2(kb[q][0][0], ka[0][0]), v[0][0], Nn[q]);
      u = fma2(add2(kb[q][0][1], ka[0][1]), v[0][2], u);
      u = fma2(add2(kb[q][1][0], ka[1][0]), v[2][0], u);
      U[q] = fma2(add2(kb[q][1][1], ka[1][1]), v[2][2], u);
      D[q] = mul2(add2(Sb[q], Sa), v[1][1]);
      // output p + 1: couplings with plane p across layer p
      u = mul2(Ya[0], v[1][0]);
      u = fma2(Ya[1], v[1][2], u);
      u = fma2(Xa[0], v[0][1], u);
      u = fma2(Xa[1], v[2][1], u);
      u = fma2(ka[0][0], v[0][0], u);
      u = fma2(ka[0][1], v[0][2], u);
      u = fma2(ka[1][0], v[2][0], u);
      Nn[q] = fma2(ka[1][1], v[2][2], u);
#pragma unroll
      for (int bq = 0; bq < 2; ++bq)
#pragma unroll
        for (int a = 0; a < 2; ++a) kb[q][bq][a] = ka[bq][a];
      Xb[q][0] = Xa[0];
      Xb[q][1] = Xa[1];
      Yb[q][0] = Ya[0];
      Yb[q][1] = Ya[1];
      Sb[q] = Sa;
      vc[q] = v[1][1];
    }
#pragma unroll
    for (int r = 0; r < RT; ++r) pre[r] = nxt[r];
    st = (st + 1) % ZW_S;
  }
  if (timed_out) {
    // record the timeout, let the copies still in flight land (bounded), end the CTA
    if (tid == 0) atomicAdd(&g_zt_timeouts, 1u);
    for (int s2 = 0; s2 < ZW_S; ++s2)
      if (pend & (1u << s2)) mbar_wait(bar0 + 8u * s2, (par >> s2) & 1u);
    return;
  }
  if (part) {
    // the partial sits where the first 32 x 16 tile of this CTA's rows puts
    // it; the other tiles it covers (RT = 4) get 0
    double v = warp_sum3((double)dot);
    if ((tid & 31) == 0) s_w[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double r = 0.0;
#pragma unroll
      for (int w = 0; w < ZTHREADS / 32; ++w) r += s_w[w];
      const int R2 = zw_rows(n, 2);
      double* pt = part + (int64_t)blockIdx.y * g.tiles_s + (int64_t)zq * (n / R2) + ty0 / R2;
      pt[0] = r;
#pragma unroll
      for (int k = 1; k < NP; ++k) pt[k] = 0.0;
    }
  }
  prof_tick3(prof);
}

inline dim3 gridz(const Grid& g, int64_t B) { return dim3((unsigned)g.zx, (unsigned)B, 1); }

// The z-march launch of an epilogue: the paired FP32 kernel for float.
template <class T, class Ld, class Epi>
inline void launch_zm3(cudaStream_t s, const Grid& g, int64_t B, const T* kappa, const Ld& ld,
                       const int32_t* active, const Epi& epi, double* part, Prof p,
                       const T* ks = nullptr) {
  if constexpr (std::is_same<T, double>::value) {
    if (ks) {   // FP64 on the element sums and the per-node kappa sums
      k_zm3q<Ld, Epi><<<gridz(g, B), dim3(ZTX, ZTY / ZRY, 1), 0, s>>>(g, kappa, ks, 4 * g.ns, ld, active, epi,
                                                                        part, p);
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    using LP = LdPaired<Ld>;
    const typename LP::type lp = LP::make(ld);
    // bulk-copy staging: full-width tiles (n in 32..256), 16-byte aligned arrays;
    // stencil_tile 0: four rows per thread, 2: two rows per thread
    if (g.zt != 1 && zw_mesh(g.n) && lp.aligned16() && ((uintptr_t)kappa & 15) == 0 && g.ns % 4 == 0 &&
        g.es % 4 == 0 && (g.zx == (int64_t)(g.n / zw_rows(g.n, 2)) * ((g.n + 1 + g.zc - 1) / g.zc))) {
      constexpr int NA = LP::type::kArrays;
      // four rows per thread: up to 71 KB of ring per CTA (opt-in above 48 KB)
      static std::atomic<uint64_t> opted{0};
      const bool four = g.zt == 0 && once_per_device(opted, [] {
                                       return cudaFuncSetAttribute(k_zm3w<typename LP::type, Epi, 4>,
                                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                   96 * 1024);
                                     }) == cudaSuccess;
      if (four) {
        const size_t smem = sizeof(float) * ZW_S * (NA * zw_vslot(g.n, 4) + zw_kslot(g.n, 4)) + 8 * ZW_S;
        k_zm3w<typename LP::type, Epi, 4><<<dim3((unsigned)(g.zx / 2), (unsigned)B, 1),
                                           dim3(g.n, ZTHREADS / g.n, 1), smem, s>>>(g, kappa, lp, active, epi,
                                                                                   part, p);
      } else {
        const size_t smem = sizeof(float) * ZW_S * (NA * zw_vslot(g.n, 2) + zw_kslot(g.n, 2)) + 8 * ZW_S;
        k_zm3w<typename LP::type, Epi, 2><<<gridz(g, B), dim3(g.n, ZTHREADS / g.n, 1), smem, s>>>(
            g, kappa, lp, active, epi, part, p);
      }
    }
    else
      k_zm3f<typename LP::type, Epi><<<gridz(g, B), dim3(ZTX, ZTY / ZRY, 1), 0, s>>>(g, kappa, lp, active,
                                                                                   epi, part, p);
  }
  else
    k_zm3<T, Ld, Epi><<<gridz(g, B), dim3(ZTX, ZTY / ZRY, 1), 0, s>>>(g, kappa, ld, active, epi, part, p);
}


template <class T>
__global__ void __launch_bounds__(256) k_winv3(Grid g, const T* __restrict__ K, double omega,
                                               T* __restrict__ W, int pz) {
  const int64_t b = blockIdx.y;
  const NodeCol c = node_col3(g.n, pz);
  if (!c.valid) return;
  const int n = g.n, N1 = n + 1;
  for (int k = c.k0; k < c.k1; ++k) {
    Node3 q;
    q.i = c.i;
    q.j = c.j;
    q.k = k;
    q.valid = true;
    q.interior = q.i > 0 && q.i < n && q.j > 0 && q.j < n && k > 0 && k < n;
    q.idx = ((int64_t)k * N1 + q.j) * N1 + q.i;
    T w = T(0);
    if (q.interior) {
      T kk[2][2][2];
      load_k8(K + b * g.es, g.n, q, kk);
      w = T(omega) / diag3(kk, g.c3);
    }
    W[b * g.ns + q.idx] = w;
  }
}

// x = 0 at every node, r = h^3 at interior nodes and 0 on the boundary
// (r may be null): one CTA per z-plane, threads along x, so the stores are
// row-contiguous and the CTA count is N1 per sample.
template <class T>
__global__ void __launch_bounds__(256) k_init3(Grid g, T* __restrict__ X, T* __restrict__ R, Prof prof) {
  const int64_t b = blockIdx.y;
  const int n = g.n, N1 = n + 1, k = blockIdx.x;
  const int64_t plane = b * g.ns + (int64_t)k * N1 * N1;
  const T h3 = T(g.h * g.h * g.h);
  const bool kin = k > 0 && k < n;
  for (int j = threadIdx.y; j <= n; j += blockDim.y) {
    const bool jin = kin && j > 0 && j < n;
    T* x = X + plane + (int64_t)j * N1;
    T* r = R ? R + plane + (int64_t)j * N1 : nullptr;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) {
      x[i] = T(0);
      if (r) r[i] = (jin && i > 0 && i < n) ? h3 : T(0);
    }
  }
  prof_tick3(prof);
}

// Full weighting: bc(I) = sum_{d in {-1,0,1}^3} w(dx) w(dy) w(dz) r1(2I + d).
template <class T>
__global__ void __launch_bounds__(256) k_restrict3(Grid gc, int64_t nsf, const T* __restrict__ R1,
                                                   T* __restrict__ Bc, const int32_t* __restrict__ active,
                                                   Prof prof, int pz) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  prof_tick3(prof);
  const NodeCol c = node_col3(gc.n, pz);
  if (!c.valid) return;
  const int nc = gc.n, C1 = nc + 1;
  const int64_t N1 = 2 * gc.n + 1, P = N1 * N1;
  const T wt[3] = {T(0.5), T(1), T(0.5)};
  const bool col_in = c.i > 0 && c.i < nc && c.j > 0 && c.j < nc;
  for (int k = c.k0; k < c.k1; ++k) {
    T v = T(0);
    if (col_in && k > 0 && k < nc) {
      const T* r = R1 + b * nsf + ((int64_t)(2 * k) * N1 + 2 * c.j) * N1 + 2 * c.i;
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
    Bc[b * gc.ns + ((int64_t)k * C1 + c.j) * C1 + c.i] = v;
  }
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
  const T d = T(g.c3) * s;
  for (int t = 0; t < 27; ++t) E[b * g.ns + t] = T(0);
  E[b * g.ns + 13] = Bv[b * g.ns + 13] / d;
}

// Pointwise: tmp = e + P ec (trilinear prolongation of the coarse
// correction; E == nullptr: tmp = P ec, the nested initial guess). A thread
// takes the fine nodes 2I and 2I + 1 of one fine row y in PROLONG_PZ
// consecutive z-planes: per plane the coarse rows under it (1, 2 or 4 by
// the parity of y and z) are summed at coarse columns I and I + 1 once, the
// even node takes the first sum, the odd node the mean of both, each
// divided by the number of rows. Warps run along I with uniform parities,
// so the gathers do not diverge; several planes per thread keep the CTAs
// few and large.
constexpr int PROLONG_PZ = 8;

template <class T>
__global__ void __launch_bounds__(256) k_prolong3(Grid g, int64_t nsc, const T* __restrict__ E,
                                                  const T* __restrict__ Ec, T* __restrict__ Tmp,
                                                  const int32_t* __restrict__ active, Prof prof) {
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  const int n = g.n, nc = n / 2, N1 = n + 1, C1 = nc + 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int ry = blockIdx.y * blockDim.y + threadIdx.y;   // (z-group, y) index
  const int rows_y = ((N1 + 7) / 8) * 8;
  const int zg = ry / rows_y, y = ry - zg * rows_y;
  if (prof.acc && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    atomicAdd(prof.acc, prof.per_sample);
  if (I > nc || y > n) return;
  const T* ec = Ec + b * nsc;
  const int J = y >> 1, oy = y & 1;
  const int x0 = 2 * I;
  const int z1 = min(zg * PROLONG_PZ + PROLONG_PZ, n + 1);
  for (int z = zg * PROLONG_PZ; z < z1; ++z) {
    const int Kc = z >> 1, oz = z & 1;
    T s0 = T(0), s1 = T(0);
    for (int c = 0; c <= oz; ++c)
      for (int bq = 0; bq <= oy; ++bq) {
        const T* row = ec + ((Kc + c) * C1 + (J + bq)) * C1;
        s0 += __ldg(row + I);
        if (I < nc) s1 += __ldg(row + I + 1);
      }
    const int rows = oy + oz;
    const T inv = rows == 0 ? T(1) : (rows == 1 ? T(0.5) : T(0.25));
    const bool row_in = y >= 1 && y < n && z >= 1 && z < n;
    const int64_t o = b * g.ns + ((int64_t)z * N1 + y) * N1 + x0;
    const T e0 = E ? E[o] : T(0);
    Tmp[o] = (row_in && x0 >= 1 && x0 < n) ? e0 + s0 * inv : T(0);
    if (x0 + 1 <= n) {
      const T e1 = E ? E[o + 1] : T(0);
      Tmp[o + 1] = (row_in && x0 + 1 < n) ? e1 + T(0.5) * (s0 + s1) * inv : T(0);
    }
  }
}

// grid of k_prolong3 for fine mesh g and B samples
inline dim3 prolong3_grid(const Grid& g, int64_t B) {
  const int nc = g.n / 2, rows_y = ((g.n + 1 + 7) / 8) * 8;
  const int zgroups = (g.n + 1 + PROLONG_PZ - 1) / PROLONG_PZ;
  return dim3((unsigned)((nc + 1 + 31) / 32), (unsigned)(rows_y / 8 * zgroups), (unsigned)B);
}

// QoI partials, one per z-plane (g.tiles_q = N1 per sample): domain: w =
// h^3 at interior nodes; box [L, H]^3 in node indices: w = h^3 chi_x chi_y
// chi_z / |box|, chi = 1 inside, 1/2 on a face. A CTA reads only the nodes
// of its plane inside the region, one FP64 add per node: each row is summed
// with its column weights (1, or 1/2 on the two face columns), each row sum
// is added with its row weight and the plane sum is scaled once.
template <class T>
__global__ void __launch_bounds__(256) k_qoi3(Grid g, int box, int L, int H, double inv_vol,
                                              const T* __restrict__ X, double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  const int n = g.n, N1 = n + 1, k = blockIdx.x;
  const int lo = box ? L : 1, hi = box ? H : n - 1;
  double acc = 0.0;
  if (k >= lo && k <= hi) {
    const T* x = X + b * g.ns + (int64_t)k * N1 * N1;
    for (int j = lo + threadIdx.y; j <= hi; j += blockDim.y) {
      double row = 0.0;
      for (int i = lo + threadIdx.x; i <= hi; i += blockDim.x) {
        const double v = (double)x[(int64_t)j * N1 + i];
        row = (box && (i == lo || i == hi)) ? fma(0.5, v, row) : row + v;
      }
      acc = (box && (j == lo || j == hi)) ? fma(0.5, row, acc) : acc + row;
    }
    double wk = g.h * g.h * g.h;
    if (box) wk *= ((k == lo || k == hi) ? 0.5 : 1.0) * inv_vol;
    acc *= wk;
  }
  cta_partial3(acc, part, g.tiles_q);
  prof_tick3(prof);
}

inline dim3 block3() { return dim3(BX, BY, 1); }


// --------------------------------------------- fused bottom of the V-cycle

constexpr int BOTTOM3_THREADS = 512;

// Levels k0 .. K-1 of the 3D V-cycle for one sample per CTA, in shared
// memory (per level: b, e and a third array for r1, then the level's
// output): pre-smoothing from zero, residual, full weighting, the exact
// coarsest solve, trilinear prolongation and post-smoothing, with a barrier
// between steps instead of a launch. A thread forms the 27-point row of a
// node from the kappa of its 8 elements (diagonal h/3 sum of the 8 kappa,
// -h/12 times the shared kappa for the 12 edge and 8 corner neighbours, as
// the z-march does); residuals are accumulated from b (in FP64 two FMAs
// instead of a multiply, an FMA and a subtraction).
template <class T>
__global__ void __launch_bounds__(BOTTOM3_THREADS) k_bottom3(BottomLevels<T> lv, const T* __restrict__ Bv,
                                                             T* __restrict__ Out,
                                                             const int32_t* __restrict__ active,
                                                             Prof prof) {
  const int64_t smp = blockIdx.x;
  if (!active[smp]) return;
  extern __shared__ __align__(16) unsigned char bottom3_raw[];
  T* sm = reinterpret_cast<T*>(bottom3_raw);
  const int L = lv.L;
  const int tid = threadIdx.x;
  auto nodes = [&](int l) { const int N1 = lv.g[l].n + 1; return N1 * N1 * N1; };
  auto base = [&](int l) -> T* {
    int off = 0;
    for (int m = 0; m < l; ++m) off += 3 * nodes(m);
    return sm + off;
  };
  // f - (A e) at the interior node (i, j, k) of level l (e in shared memory)
  auto resid = [&](int l, const T* e, int i, int j, int k, T f) -> T {
    const Grid& g = lv.g[l];
    const int n = g.n, N1 = n + 1, P = N1 * N1, o = (k * N1 + j) * N1 + i;
    const T* K = lv.kap[l] + smp * g.es;
    T kk[2][2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const T* r = K + ((k - 1 + c) * n + (j - 1 + b)) * n + (i - 1);
        kk[c][b][0] = __ldg(r);
        kk[c][b][1] = __ldg(r + 1);
      }
    auto v = [&](int dx, int dy, int dz) { return e[o + dz * P + dy * N1 + dx]; };
    T u = T(0);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        u = fma(kk[0][q][p] + kk[1][q][p], v(2 * p - 1, 2 * q - 1, 0), u);   // edges in the xy-plane
        u = fma(kk[q][0][p] + kk[q][1][p], v(2 * p - 1, 0, 2 * q - 1), u);   // edges in the xz-plane
        u = fma(kk[q][p][0] + kk[q][p][1], v(0, 2 * p - 1, 2 * q - 1), u);   // edges in the yz-plane
      }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) u = fma(kk[c][b][a], v(2 * a - 1, 2 * b - 1, 2 * c - 1), u);
    const T S = ((kk[0][0][0] + kk[0][0][1]) + (kk[0][1][0] + kk[0][1][1])) +
                ((kk[1][0][0] + kk[1][0][1]) + (kk[1][1][0] + kk[1][1][1]));
    return fma(T(g.c12), u, fma(-T(g.c3), S * v(0, 0, 0), f));
  };
  auto interior = [](int n, int i, int j, int k) {
    return i > 0 && i < n && j > 0 && j < n && k > 0 && k < n;
  };
  {
    T* b = base(0);
    const T* src = Bv + smp * lv.g[0].ns;
    for (int x = tid; x < nodes(0); x += BOTTOM3_THREADS) b[x] = src[x];
  }
  __syncthreads();
  // down: e = W b, r1 = b - A e, b_{l+1} = R r1
  for (int l = 0; l < L - 1; ++l) {
    const int n = lv.g[l].n, N1 = n + 1, nn = nodes(l);
    T* b = base(l);
    T* e = b + nn;
    T* t = e + nn;
    const T* W = lv.w[l] + smp * lv.g[l].ns;
    for (int x = tid; x < nn; x += BOTTOM3_THREADS) e[x] = __ldg(W + x) * b[x];
    __syncthreads();
    for (int x = tid; x < nn; x += BOTTOM3_THREADS) {
      const int k = x / (N1 * N1), r = x - k * N1 * N1, j = r / N1, i = r - j * N1;
      t[x] = interior(n, i, j, k) ? resid(l, e, i, j, k, b[x]) : T(0);
    }
    __syncthreads();
    const int nc = lv.g[l + 1].n, C1 = nc + 1;
    T* bc = base(l + 1);
    for (int x = tid; x < C1 * C1 * C1; x += BOTTOM3_THREADS) {
      const int K = x / (C1 * C1), r = x - K * C1 * C1, J = r / C1, I = r - J * C1;
      T v = T(0);
      if (interior(nc, I, J, K)) {
        const int P = N1 * N1;
        const T* rr0 = t + ((2 * K) * N1 + 2 * J) * N1 + 2 * I;
        const T wt[3] = {T(0.5), T(1), T(0.5)};
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
          T pl = T(0);
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy) {
            const T* rr = rr0 + dz * P + dy * N1;
            const T row = T(0.5) * rr[-1] + rr[0] + T(0.5) * rr[1];
            pl += wt[dy + 1] * row;
          }
          v += wt[dz + 1] * pl;
        }
      }
      bc[x] = v;
    }
    __syncthreads();
  }
  // coarsest grid (n = 2, one unknown at (1, 1, 1)): e = b / D
  {
    T* b = base(L - 1);
    T* e = b + 27;
    if (tid == 0) {
      const T* k = lv.kap[L - 1] + smp * lv.g[L - 1].es;
      T s = T(0);
      for (int q = 0; q < 8; ++q) s += k[q];
      const T d = T(lv.g[L - 1].c3) * s;
      for (int q = 0; q < 27; ++q) e[q] = T(0);
      e[13] = b[13] / d;
    }
  }
  __syncthreads();
  // up: e += P e_c, out = e + W (b - A e)
  for (int l = L - 2; l >= 0; --l) {
    const int n = lv.g[l].n, N1 = n + 1, nn = nodes(l);
    T* b = base(l);
    T* e = b + nn;
    T* t = e + nn;
    const int C1 = lv.g[l + 1].n + 1, ncn = nodes(l + 1);
    const T* ec = base(l + 1) + ((l + 1 == L - 1) ? ncn : 2 * ncn);
    for (int x = tid; x < nn; x += BOTTOM3_THREADS) {
      const int k = x / (N1 * N1), r = x - k * N1 * N1, j = r / N1, i = r - j * N1;
      if (!interior(n, i, j, k)) continue;
      const int I = i >> 1, J = j >> 1, Kc = k >> 1, ox = i & 1, oy = j & 1, oz = k & 1;
      T s0 = T(0), s1 = T(0);
      for (int c = 0; c <= oz; ++c)
        for (int bq = 0; bq <= oy; ++bq) {
          const T* row = ec + ((Kc + c) * C1 + (J + bq)) * C1;
          s0 += row[I];
          if (ox) s1 += row[I + 1];
        }
      const int rows = oy + oz;
      const T inv = rows == 0 ? T(1) : (rows == 1 ? T(0.5) : T(0.25));
      e[x] = e[x] + (ox ? T(0.5) * (s0 + s1) * inv : s0 * inv);
    }
    __syncthreads();
    const T* W = lv.w[l] + smp * lv.g[l].ns;
    for (int x = tid; x < nn; x += BOTTOM3_THREADS) {
      const int k = x / (N1 * N1), r = x - k * N1 * N1, j = r / N1, i = r - j * N1;
      T ov = T(0);
      if (interior(n, i, j, k)) ov = fma(__ldg(W + x), resid(l, e, i, j, k, b[x]), e[x]);
      t[x] = ov;
    }
    __syncthreads();
  }
  {
    const T* t = base(0) + 2 * nodes(0);
    T* dst = Out + smp * lv.g[0].ns;
    for (int x = tid; x < nodes(0); x += BOTTOM3_THREADS) dst[x] = t[x];
  }
  if (prof.acc && tid == 0) atomicAdd(prof.acc, prof.per_sample);
}

}  // namespace

namespace d3 {

template <class T>
cudaError_t apply(cudaStream_t s, const Grid& g, const T* kappa, const T* x, T* y, int64_t B, Prof p) {
  launch_zm3<T>(s, g, B, kappa, LdX<T>{x, g.ns}, nullptr, EpiApply<T>{y, g.ns}, nullptr, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t winv(cudaStream_t s, const Grid& g, const T* kappa, double omega, T* w, int64_t B) {
  const int pz = node_pz(g.n);
  k_winv3<T><<<dim3(node_col3_blocks(g.n, pz), (unsigned)B, 1), block3(), 0, s>>>(g, kappa, omega, w, pz);
  return cudaGetLastError();
}
template <class T>
cudaError_t pcg_init(cudaStream_t s, const Grid& g, T* x, T* r, int64_t B, Prof p) {
  if (!r) return d2::zero_nodes<T>(s, g, x, B, p);   // flat: node layout does not matter
  k_init3<T><<<dim3((unsigned)(g.n + 1), (unsigned)B, 1), block3(), 0, s>>>(g, x, r, p);
  return cudaGetLastError();
}
template <class T>
cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const T* kappa, const T* z, const T* p_old, T* p_new,
                   T* q, const Scalars& sc, double* part, int64_t B, Prof p, const T* ks) {
  launch_zm3<T>(s, g, B, kappa, LdPupd<T>{z, p_old, sc.beta, g.ns, T(0)}, sc.active,
                EpiAq<T>{q, p_new, g.ns}, part, p, ks);
  return cudaGetLastError();
}
template <class T>
cudaError_t mg_pre(cudaStream_t s, const Grid& g, const T* kappa, const T* w, const T* b, T* e, T* r1,
                   const int32_t* active, int64_t B, Prof p, const T* ks) {
  launch_zm3<T>(s, g, B, kappa, LdWb<T>{w, b, g.ns}, active, EpiMgRes<T>{b, r1, e, g.ns}, nullptr, p, ks);
  return cudaGetLastError();
}
template <class T>
cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const T* r1, T* bc,
                      const int32_t* active, int64_t B, Prof p) {
  const int pz = node_pz(coarse.n);
  k_restrict3<T><<<dim3(node_col3_blocks(coarse.n, pz), (unsigned)B, 1), block3(), 0, s>>>(coarse, fine.ns, r1,
                                                                                          bc, active, p, pz);
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
                    double* part, int64_t B, Prof p, const T* ks) {
  k_prolong3<T><<<prolong3_grid(g, B), dim3(32, 8, 1), 0, s>>>(g, coarse.ns, e, ec, tmp, active,
                                                                 Prof{nullptr, 0.0});
  launch_zm3<T>(s, g, B, kappa, LdX<T>{tmp, g.ns}, active, EpiMgPost<T>{w, b, out, g.ns}, part, p, ks);
  return cudaGetLastError();
}
template <class T>
cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol, const T* x,
                double* part, int64_t B, Prof p) {
  k_qoi3<T><<<dim3((unsigned)(g.n + 1), (unsigned)B, 1), block3(), 0, s>>>(g, box, L, H, inv_vol, x, part, p);
  return cudaGetLastError();
}
cudaError_t prolong_guess(cudaStream_t s, const Grid& g, const Grid& coarse, const double* uc,
                          double* x, const int32_t* active, int64_t B, Prof p) {
  k_prolong3<double><<<prolong3_grid(g, B), dim3(32, 8, 1), 0, s>>>(g, coarse.ns, nullptr, uc, x, active, p);
  return cudaGetLastError();
}

cudaError_t resid64(cudaStream_t s, const Grid& g, const double* kappa, const double* u, double* r,
                    const int32_t* active, double* part, int64_t B, Prof p, const double* ks) {
  if (ks)
    k_zm3q<LdX<double>, EpiResid><<<gridz(g, B), dim3(ZTX, ZTY / ZRY, 1), 0, s>>>(
        g, kappa, ks, 4 * g.ns, LdX<double>{u, g.ns}, active, EpiResid{r, g.ns, g.h * g.h * g.h}, part, p);
  else
    launch_zm3<double>(s, g, B, kappa, LdX<double>{u, g.ns}, active, EpiResid{r, g.ns, g.h * g.h * g.h},
                       part, p);
  return cudaGetLastError();
}

cudaError_t ksum(cudaStream_t s, const Grid& g, const double* kappa, double* ks, int64_t B) {
  const int pz = node_pz(g.n);
  k_ksum3<<<dim3(node_col3_blocks(g.n, pz), (unsigned)B, 1), block3(), 0, s>>>(g, kappa, ks, 4 * g.ns, pz);
  return cudaGetLastError();
}

template <class T>
cudaError_t mg_bottom(cudaStream_t s, const BottomLevels<T>& lv, const T* b, T* out,
                      const int32_t* active, int64_t B, Prof p) {
  if (lv.L < 2 || lv.L > MAX_BOTTOM || lv.g[lv.L - 1].n != 2 || lv.g[0].n > BOTTOM_MAX_N3)
    return cudaErrorInvalidValue;
  size_t smem = 0;
  for (int l = 0; l < lv.L; ++l) {
    const size_t N1 = lv.g[l].n + 1;
    smem += 3 * N1 * N1 * N1 * sizeof(T);
  }
  // opt in (once per device) to the shared memory of the largest fused chain (16^3 .. 2^3)
  static std::atomic<uint64_t> opted{0};
  const cudaError_t attr = once_per_device(opted, [] {
    size_t most = 0;
    for (int n = BOTTOM_MAX_N3; n >= 2; n /= 2) most += 3 * (size_t)(n + 1) * (n + 1) * (n + 1) * sizeof(T);
    return cudaFuncSetAttribute(k_bottom3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
  });
  if (attr != cudaSuccess) return attr;
  k_bottom3<T><<<(unsigned)B, BOTTOM3_THREADS, smem, s>>>(lv, b, out, active, p);
  return cudaGetLastError();
}

// Waits of the bulk-copy z-march that gave up since the last call on this
// device (the counter is reset); read on `s` after the caller's own sync.
cudaError_t take_wait_timeouts(cudaStream_t s, unsigned* out) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_zt_timeouts, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h != 0) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbolAsync(g_zt_timeouts, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  *out = h;
  return e;
}

#define MLMC_INST3(T)                                                                              \
  template cudaError_t apply<T>(cudaStream_t, const Grid&, const T*, const T*, T*, int64_t, Prof); \
  template cudaError_t winv<T>(cudaStream_t, const Grid&, const T*, double, T*, int64_t);          \
  template cudaError_t pcg_init<T>(cudaStream_t, const Grid&, T*, T*, int64_t, Prof);              \
  template cudaError_t pcg_pq<T>(cudaStream_t, const Grid&, const T*, const T*, const T*, T*, T*,  \
                                 const Scalars&, double*, int64_t, Prof, const T*);                \
  template cudaError_t mg_pre<T>(cudaStream_t, const Grid&, const T*, const T*, const T*, T*, T*,  \
                                 const int32_t*, int64_t, Prof, const T*);                         \
  template cudaError_t restrict_<T>(cudaStream_t, const Grid&, const Grid&, const T*, T*,          \
                                    const int32_t*, int64_t, Prof);                                \
  template cudaError_t coarse_solve<T>(cudaStream_t, const Grid&, const T*, const T*, T*,          \
                                       const int32_t*, int64_t);                                   \
  template cudaError_t mg_post<T>(cudaStream_t, const Grid&, const Grid&, const T*, const T*,      \
                                  const T*, const T*, const T*, T*, T*, const int32_t*, double*,   \
                                  int64_t, Prof, const T*);                                        \
  template cudaError_t qoi<T>(cudaStream_t, const Grid&, int, int, int, double, const T*, double*, \
                              int64_t, Prof);                                                      \
  template cudaError_t mg_bottom<T>(cudaStream_t, const BottomLevels<T>&, const T*, T*,            \
                                    const int32_t*, int64_t, Prof);

MLMC_INST3(double)
MLMC_INST3(float)

}  // namespace d3
}  // namespace mlmc
