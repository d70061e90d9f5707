// 2D matrix-free Q1 operator, batched PCG vector kernels and geometric
// multigrid kernels, templated on the value type (double: the FP64 form and
// the FP64 residual of the mixed form; float: the FP32 inner solve).
//
// Operator (Eq. (model), Sec. 2.1, Q1 on a uniform grid, kappa constant per
// element, homogeneous Dirichlet): at an interior node c with surrounding
// elements SW, SE, NW, NE (kappa values kSW..kNE) the row of A is
//   diagonal           2/3 (kSW + kSE + kNW + kNE)
//   edge neighbours   -1/6 (sum of kappa of the two elements sharing the edge)
//   corner neighbours -1/3 kappa of the one element shared.
//
// Stencil kernels stream: each warp owns a strip of 32 node columns (30
// outputs; the two edge lanes only supply neighbours) and walks down SROWS
// rows, keeping a 3-row window of the field and a 2-row window of kappa in
// registers; x-neighbours come from warp shuffles. The field the stencil
// acts on (p = z + beta p_old, e = W b, e + P e_c, ...) is formed once per
// node as its row enters the window, and the next row is fetched before the
// current one is consumed. No shared memory, no barriers.
//
// The multigrid levels of at most 64^2 cells below the finest run as one
// kernel per V-cycle (k_bottom2): one CTA per sample, every level's arrays
// in shared memory, a barrier between the steps instead of a launch.
//
// Pointwise kernels treat each sample's node array as a flat vector
// (boundary entries are 0 and stay 0) with 16-byte vector accesses.
//
// Node arrays carry the boundary nodes (always 0). Per-sample reductions
// write one FP64 partial per warp (stencil kernels, g.tiles_s per sample)
// or per CTA (flat kernels, g.tiles_f per sample), summed in a fixed order
// by k_finalize.
#include "mlmc_internal.cuh"

namespace mlmc {
namespace {

template <class T>
struct Consts {
  static constexpr T c23 = T(2) / T(3);
  static constexpr T c16 = T(1) / T(6);
  static constexpr T c13 = T(1) / T(3);
};

__device__ __forceinline__ bool interior2(int n, int i, int j) {
  return i > 0 && i < n && j > 0 && j < n;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------ warp strips

struct Strip {
  int n;        // cells per side
  int N1;       // nodes per row
  int c;        // node column of this lane (may be -1 or > n)
  bool out;     // this lane produces outputs (lanes 1..30, column <= n)
  int y0, y1;   // output rows [y0, y1)
  int64_t part_idx;
};

__device__ __forceinline__ Strip strip_of(const Grid& g) {
  Strip s;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int strip = blockIdx.x * SWARPS + warp;
  s.n = g.n;
  s.N1 = g.n + 1;
  s.c = strip * 30 - 1 + lane;
  s.out = (lane >= 1) && (lane <= 30) && (s.c <= g.n);
  s.y0 = blockIdx.y * SROWS;
  s.y1 = min(s.y0 + SROWS, g.n + 1);
  s.part_idx = (int64_t)blockIdx.z * g.tiles_s + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * SWARPS + warp;
  return s;
}

__device__ __forceinline__ bool first_thread() {
  return blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0;
}

__device__ __forceinline__ void prof_tick(const Prof& p) {
  if (p.acc && first_thread()) atomicAdd(p.acc, p.per_sample);
}

// kappa of element (e, r) of one sample, 0 outside the grid.
template <class T>
__device__ __forceinline__ T kap_at(const T* __restrict__ k, int n, int e, int r) {
  return (e >= 0 && e < n && r >= 0 && r < n) ? __ldg(k + (int64_t)r * n + e) : T(0);
}

// Two loads of one node, combined when the node enters the window.
template <class T>
struct Pair {
  T a, b;
};

// Field rows j-1, j, j+1 at columns c-1, c, c+1 and kappa of the elements
// (c-1, j-1), (c, j-1), (c-1, j), (c, j) around node (c, j).
template <class T>
struct Win {
  T vm, v0, vp;
  T lm, l0, lp;
  T rm, r0, rp;
  T ka, kb, kal, kbl;
};

template <class T>
__device__ __forceinline__ T stencil_win(const Win<T>& w) {
  const T ksw = w.kal, kse = w.ka, knw = w.kbl, kne = w.kb;
  const T kS = ksw + kse, kN = knw + kne, kW = ksw + knw, kE = kse + kne;
  const T edge = kE * w.r0 + kW * w.l0 + kN * w.vp + kS * w.vm;
  const T corner = kne * w.rp + knw * w.lp + kse * w.rm + ksw * w.lm;
  return Consts<T>::c23 * (kS + kN) * w.v0 - Consts<T>::c16 * edge - Consts<T>::c13 * corner;
}

// Node coefficients of the 2D operator, precomputed once per solve (FP64
// form): per sample cd (diagonal), ce (coupling with the east neighbour),
// cn (coupling with the north neighbour) at every node, and q (corner
// coupling) per element, laid out [cd | ce | cn] in node strides, then q.
// With them a row of the operator costs 1 multiply and 8 FMAs instead of 17
// FP64 operations on kappa (the west and south couplings are the east and
// north ones of the neighbours).
template <class T>
struct WinC {
  T vm, v0, vp, lm, l0, lp, rm, r0, rp;   // field, as in Win
  T qa, qb, qal, qbl;                     // corner couplings of elements (c, j-1), (c, j), (c-1, j-1), (c-1, j)
  T cd, ce, ceW, cnN, cnS;                // diagonal, east, west, north, south couplings
};

template <class T>
__device__ __forceinline__ T stencil_coef(const WinC<T>& w) {
  T a = w.cd * w.v0;
  a = fma(w.ce, w.r0, a);
  a = fma(w.ceW, w.l0, a);
  a = fma(w.cnN, w.vp, a);
  a = fma(w.cnS, w.vm, a);
  a = fma(w.qb, w.rp, a);
  a = fma(w.qbl, w.lp, a);
  a = fma(w.qa, w.rm, a);
  return fma(w.qal, w.lm, a);
}

// FP64 kernels are bound by the FP64 pipe, so they take the forms with the
// fewest FP64 instructions (residuals accumulated from the right-hand side,
// the streamed prolongation of the post-smoother); FP32 kernels are bound by instruction
// issue, where the plain forms need fewer instructions in all.
template <class T>
constexpr bool kResidualForm = sizeof(T) == 8;

// rhs - (A x) at the window's centre, accumulated from rhs with negated
// couplings: 9 FMAs where rhs - stencil_coef costs a multiply, 8 FMAs and a
// subtraction.
template <class T>
__device__ __forceinline__ T stencil_coef_res(const WinC<T>& w, T rhs) {
  T a = fma(-w.cd, w.v0, rhs);
  a = fma(-w.ce, w.r0, a);
  a = fma(-w.ceW, w.l0, a);
  a = fma(-w.cnN, w.vp, a);
  a = fma(-w.cnS, w.vm, a);
  a = fma(-w.qb, w.rp, a);
  a = fma(-w.qbl, w.lp, a);
  a = fma(-w.qa, w.rm, a);
  return fma(-w.qal, w.lm, a);
}

// Row-loop unrolling of the strip kernels: by 6 in FP64 (a multiple of the
// 3-row field window and the 2-row kappa / coefficient windows, so the
// windows rotate by renaming; the FP64 post-smoother gets 6% faster), none
// in FP32 (where unrolling made the post-smoother 10% slower).
template <class T>
constexpr int kStripUnroll = sizeof(T) == 8 ? 6 : 1;

// FP32 strips on paired rows: a lane takes the output rows j and j + 1 per
// step, and their two stencils run on float2 pairs (row j in .x, row j + 1
// in .y) with the paired FP32 instructions, so the stencil arithmetic and the
// loop overhead per node halve; loads, shuffles and outputs stay per node.
// The field comes in row pairs (y0 - 1 + 2p, y0 + 2p): fetch2(j) issues the
// loads of rows j and j + 1 and form2(raw, j) turns them into the two field
// values (0 outside the interior), called once per pair in increasing j, one
// pair after its fetch (so form2 may carry state from pair to pair). The
// next pair's field rows and kappa rows are fetched before the current pair
// is consumed. out(j, x, A x) as in stream_strip_rf (kappa form).
__device__ __forceinline__ float2 pf2(float a, float b) { return make_float2(a, b); }

template <class Fetch2F, class Form2F, class OutF>
__device__ __forceinline__ void stream_strip_pair(const Strip& s, const float* __restrict__ kap,
                                                  Fetch2F&& fetch2, Form2F&& form2, OutF&& out) {
  const int n = s.n;
  constexpr unsigned FULL = 0xffffffffu;
  // carried from the previous pair: field rows j - 1 (a) and j (b), kappa row j - 1
  const float2 vab = form2(fetch2(s.y0 - 1), s.y0 - 1);
  float va = vab.x, vb = vab.y;
  float la = __shfl_up_sync(FULL, va, 1), ra = __shfl_down_sync(FULL, va, 1);
  float lb = __shfl_up_sync(FULL, vb, 1), rb = __shfl_down_sync(FULL, vb, 1);
  float ka = kap_at(kap, n, s.c, s.y0 - 1);
  float kal = __shfl_up_sync(FULL, ka, 1);
  // in flight: field rows j + 1, j + 2 and kappa rows j, j + 1
  auto rcd = fetch2(s.y0 + 1);
  float kb = kap_at(kap, n, s.c, s.y0), kc = kap_at(kap, n, s.c, s.y0 + 1);
  const float2 c23 = pf2(Consts<float>::c23, Consts<float>::c23);
  const float2 mc16 = pf2(-Consts<float>::c16, -Consts<float>::c16);
  const float2 mc13 = pf2(-Consts<float>::c13, -Consts<float>::c13);
  for (int j = s.y0; j < s.y1; j += 2) {
    const float2 vcd = form2(rcd, j + 1);
    const float vc = vcd.x, vd = vcd.y;
    const float lc = __shfl_up_sync(FULL, vc, 1), rcx = __shfl_down_sync(FULL, vc, 1);
    const float ld = __shfl_up_sync(FULL, vd, 1), rdx = __shfl_down_sync(FULL, vd, 1);
    const float kbl = __shfl_up_sync(FULL, kb, 1), kcl = __shfl_up_sync(FULL, kc, 1);
    const float kb_ = kb, kc_ = kc;
    if (j + 2 < s.y1) {   // the next pair's rows before this pair is consumed
      rcd = fetch2(j + 3);
      kb = kap_at(kap, n, s.c, j + 2);
      kc = kap_at(kap, n, s.c, j + 3);
    }
    if (s.out) {
      // elements around node (c, r), r = j (.x) and j + 1 (.y)
      const float2 ksw = pf2(kal, kbl), kse = pf2(ka, kb_), knw = pf2(kbl, kcl), kne = pf2(kb_, kc_);
      const float2 kS = __fadd2_rn(ksw, kse), kN = __fadd2_rn(knw, kne);
      const float2 kW = __fadd2_rn(ksw, knw), kE = __fadd2_rn(kse, kne);
      const float2 vm = pf2(va, vb), v0 = pf2(vb, vc), vp = pf2(vc, vd);
      const float2 lm = pf2(la, lb), l0 = pf2(lb, lc), lp = pf2(lc, ld);
      const float2 rm = pf2(ra, rb), r0 = pf2(rb, rcx), rp = pf2(rcx, rdx);
      float2 edge = __fmul2_rn(kE, r0);
      edge = __ffma2_rn(kW, l0, edge);
      edge = __ffma2_rn(kN, vp, edge);
      edge = __ffma2_rn(kS, vm, edge);
      float2 corner = __fmul2_rn(kne, rp);
      corner = __ffma2_rn(knw, lp, corner);
      corner = __ffma2_rn(kse, rm, corner);
      corner = __ffma2_rn(ksw, lm, corner);
      float2 y = __fmul2_rn(__fmul2_rn(c23, __fadd2_rn(kS, kN)), v0);
      y = __ffma2_rn(mc16, edge, y);
      y = __ffma2_rn(mc13, corner, y);
      out(j, vb, interior2(n, s.c, j) ? y.x : 0.f);
      if (j + 1 < s.y1) out(j + 1, vc, interior2(n, s.c, j + 1) ? y.y : 0.f);
    }
    va = vc;
    la = lc;
    ra = rcx;
    vb = vd;
    lb = ld;
    rb = rdx;
    ka = kc_;
    kal = kcl;
  }
}

// Per-row fields (field issues a node's loads, form combines them) on paired rows.
template <class FieldF, class FormF, class OutF>
__device__ __forceinline__ void stream_strip_pair_rows(const Strip& s, const float* __restrict__ kap,
                                                       FieldF&& field, FormF&& form, OutF&& out) {
  const int n = s.n;
  using Raw = decltype(field(0, 0));
  struct Raw2 {
    Raw a, b;
  };
  auto fetch = [&](int j) -> Raw {
    Raw r{};
    if (interior2(n, s.c, j)) r = field(s.c, j);
    return r;
  };
  auto fld = [&](int j, const Raw& r) -> float { return interior2(n, s.c, j) ? float(form(r, s.c, j)) : 0.f; };
  stream_strip_pair(
      s, kap, [&](int j) { return Raw2{fetch(j), fetch(j + 1)}; },
      [&](const Raw2& r, int j) { return pf2(fld(j, r.a), fld(j + 1, r.b)); }, out);
}

// Streams one warp strip. The stencilled field at an interior node (c, j)
// is form(field(c, j), c, j): field issues the node's loads (called for
// consecutive rows j, two rows ahead of use) and form combines them when
// the row enters the window, one stencil row later, so the loads have that
// row's arithmetic to land (form = identity when field returns the value).
// out(j, x, y, f) runs for each output row j of an output lane with the
// field x at (c, j) and y = (A x)(c, j) (R false) or y = f - (A x)(c, j)
// with f = rhs(j) (R true); y is 0 at boundary nodes. rhs(j) is called for
// output lanes only, one row ahead of its use. C selects the operator
// source: kappa per element (src = kappa of the sample), or the precomputed
// coefficients (src = coefficient block of the sample, ns its node stride).
// Every lane executes the loads and shuffles.
template <class T, bool C, bool R, class FieldF, class FormF, class RhsF, class OutF>
__device__ __forceinline__ void stream_strip_rf(const Strip& s, const T* __restrict__ src, int64_t ns,
                                                FieldF&& field, FormF&& form, RhsF&& rhs, OutF&& out) {
  if constexpr (sizeof(T) == 4 && !C && !R) {
    stream_strip_pair_rows(s, src, field, form, [&](int j, float x, float ax) { out(j, x, ax, 0.f); });
    return;
  }
  const int n = s.n;
  using Raw = decltype(field(0, 0));
  auto fetch = [&](int j) -> Raw {
    Raw r{};
    if (interior2(n, s.c, j)) r = field(s.c, j);
    return r;
  };
  auto fld = [&](int j, const Raw& r) -> T { return interior2(n, s.c, j) ? T(form(r, s.c, j)) : T(0); };
  T fn = T(0);
  if constexpr (R) {
    if (s.out && s.y0 < s.y1) fn = rhs(s.y0);
  }
  if constexpr (!C) {
    const T* __restrict__ kap = src;
    Win<T> w;
    w.v0 = fld(s.y0 - 1, fetch(s.y0 - 1));
    w.vp = fld(s.y0, fetch(s.y0));
    w.l0 = __shfl_up_sync(0xffffffffu, w.v0, 1);
    w.r0 = __shfl_down_sync(0xffffffffu, w.v0, 1);
    w.lp = __shfl_up_sync(0xffffffffu, w.vp, 1);
    w.rp = __shfl_down_sync(0xffffffffu, w.vp, 1);
    w.kb = kap_at(kap, n, s.c, s.y0 - 1);
    w.kbl = __shfl_up_sync(0xffffffffu, w.kb, 1);
    Raw rn = fetch(s.y0 + 1);
    T kn = kap_at(kap, n, s.c, s.y0);
#pragma unroll kStripUnroll<T>
    for (int j = s.y0; j < s.y1; ++j) {
      w.vm = w.v0; w.lm = w.l0; w.rm = w.r0;
      w.v0 = w.vp; w.l0 = w.lp; w.r0 = w.rp;
      w.vp = fld(j + 1, rn);
      w.lp = __shfl_up_sync(0xffffffffu, w.vp, 1);
      w.rp = __shfl_down_sync(0xffffffffu, w.vp, 1);
      w.ka = w.kb; w.kal = w.kbl;
      w.kb = kn;
      w.kbl = __shfl_up_sync(0xffffffffu, kn, 1);
      const T f = fn;
      if (j + 1 < s.y1) {          // fetch the next rows before consuming this one
        rn = fetch(j + 2);
        kn = kap_at(kap, n, s.c, j + 1);
        if constexpr (R) {
          if (s.out) fn = rhs(j + 1);
        }
      }
      if (s.out) {
        T y = T(0);
        if (interior2(n, s.c, j)) y = R ? f - stencil_win(w) : stencil_win(w);
        out(j, w.v0, y, f);
      }
    }
  } else {
    const T* __restrict__ cd = src;
    const T* __restrict__ ce = src + ns;
    const T* __restrict__ cn = src + 2 * ns;
    const T* __restrict__ q = src + 3 * ns;
    const int N1 = n + 1;
    auto node = [&](const T* __restrict__ a, int j) -> T {
      return (s.c <= n && j >= 0 && j <= n) ? __ldg(a + (int64_t)j * N1 + s.c) : T(0);
    };
    WinC<T> w;
    w.v0 = fld(s.y0 - 1, fetch(s.y0 - 1));
    w.vp = fld(s.y0, fetch(s.y0));
    w.l0 = __shfl_up_sync(0xffffffffu, w.v0, 1);
    w.r0 = __shfl_down_sync(0xffffffffu, w.v0, 1);
    w.lp = __shfl_up_sync(0xffffffffu, w.vp, 1);
    w.rp = __shfl_down_sync(0xffffffffu, w.vp, 1);
    w.qb = kap_at(q, n, s.c, s.y0 - 1);
    w.qbl = __shfl_up_sync(0xffffffffu, w.qb, 1);
    Raw rn = fetch(s.y0 + 1);
    T qn = kap_at(q, n, s.c, s.y0);
    T cn_prev = node(cn, s.y0 - 1);
    T cdn = node(cd, s.y0), cen = node(ce, s.y0), cnn = node(cn, s.y0);
#pragma unroll kStripUnroll<T>
    for (int j = s.y0; j < s.y1; ++j) {
      w.vm = w.v0; w.lm = w.l0; w.rm = w.r0;
      w.v0 = w.vp; w.l0 = w.lp; w.r0 = w.rp;
      w.vp = fld(j + 1, rn);
      w.lp = __shfl_up_sync(0xffffffffu, w.vp, 1);
      w.rp = __shfl_down_sync(0xffffffffu, w.vp, 1);
      w.qa = w.qb; w.qal = w.qbl;
      w.qb = qn;
      w.qbl = __shfl_up_sync(0xffffffffu, qn, 1);
      w.cd = cdn;
      w.ce = cen;
      w.ceW = __shfl_up_sync(0xffffffffu, cen, 1);
      w.cnN = cnn;
      w.cnS = cn_prev;
      cn_prev = cnn;
      const T f = fn;
      if (j + 1 < s.y1) {          // fetch the next rows before consuming this one
        rn = fetch(j + 2);
        qn = kap_at(q, n, s.c, j + 1);
        cdn = node(cd, j + 1);
        cen = node(ce, j + 1);
        cnn = node(cn, j + 1);
        if constexpr (R) {
          if (s.out) fn = rhs(j + 1);
        }
      }
      if (s.out) {
        T y = T(0);
        if (interior2(n, s.c, j)) y = R ? stencil_coef_res(w, f) : stencil_coef(w);
        out(j, w.v0, y, f);
      }
    }
  }
}

// Fields that are formed when fetched (form = identity).
template <class T, bool C, bool R, class FieldF, class RhsF, class OutF>
__device__ __forceinline__ void stream_strip_r(const Strip& s, const T* __restrict__ src, int64_t ns,
                                               FieldF&& field, RhsF&& rhs, OutF&& out) {
  stream_strip_rf<T, C, R>(s, src, ns, field, [](T v, int, int) { return v; }, rhs, out);
}

// The operator-apply form: out(j, x, A x).
template <class T, bool C, class FieldF, class OutF>
__device__ __forceinline__ void stream_strip(const Strip& s, const T* __restrict__ src, int64_t ns,
                                             FieldF&& field, OutF&& out) {
  stream_strip_r<T, C, false>(s, src, ns, field, [](int) { return T(0); },
                              [&](int j, T x, T ax, T) { out(j, x, ax); });
}

// The operator-apply form with a deferred field (see stream_strip_rf).
template <class T, bool C, class FieldF, class FormF, class OutF>
__device__ __forceinline__ void stream_strip_f(const Strip& s, const T* __restrict__ src, int64_t ns,
                                               FieldF&& field, FormF&& form, OutF&& out) {
  stream_strip_rf<T, C, false>(s, src, ns, field, form, [](int) { return T(0); },
                               [&](int j, T x, T ax, T) { out(j, x, ax); });
}

// This warp's partial: per-lane sums (in T) are added across the warp in FP64.
template <class T>
__device__ __forceinline__ void warp_partial(T v, double* __restrict__ part, int64_t idx) {
  const double d = warp_sum((double)v);
  if ((threadIdx.x & 31) == 0) part[idx] = d;
}

inline dim3 sgrid(const Grid& g, int64_t B) { return dim3((unsigned)g.sx, (unsigned)g.sy, (unsigned)B); }
constexpr int SBLOCK = SWARPS * 32;

template <class T>
__global__ void __launch_bounds__(SBLOCK) k_apply2(Grid g, const T* __restrict__ K,
                                                   const T* __restrict__ X, T* __restrict__ Y,
                                                   Prof prof) {
  const Strip s = strip_of(g);
  const int64_t b = blockIdx.z;
  const T* x = X + b * g.ns;
  T* y = Y + b * g.ns;
  stream_strip<T, false>(s, K + b * g.es, g.ns,
                         [&](int c, int j) { return __ldg(x + (int64_t)j * s.N1 + c); },
                         [&](int j, T, T ax) { y[(int64_t)j * s.N1 + s.c] = ax; });
  prof_tick(prof);
}

// p_new = z + beta p_old (beta == 0: p_new = z), q = A p_new, partials of p.q
// (K: kappa, or with C the coefficient blocks, cs doubles per sample)
template <class T, bool C>
__global__ void __launch_bounds__(SBLOCK) k_pq2(Grid g, const T* __restrict__ K, int64_t cs,
                                                const T* __restrict__ Z, const T* __restrict__ Pold,
                                                T* __restrict__ Pnew, T* __restrict__ Q,
                                                const double* __restrict__ beta,
                                                const int32_t* __restrict__ active,
                                                double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  const Strip s = strip_of(g);
  const T bb = (T)beta[b];
  const T* z = Z + b * g.ns;
  const T* po = Pold + b * g.ns;
  T* pn = Pnew + b * g.ns;
  T* q = Q + b * g.ns;
  T dot = T(0);
  auto out = [&](int j, T pv, T ax) {
    const int64_t o = (int64_t)j * s.N1 + s.c;
    dot = fma(pv, ax, dot);
    pn[o] = pv;
    q[o] = ax;
  };
  const T* src = K + b * cs;
  if (bb == T(0)) {
    stream_strip<T, C>(s, src, g.ns, [&](int c, int j) { return __ldg(z + (int64_t)j * s.N1 + c); }, out);
  } else if constexpr (sizeof(T) == 4) {
    stream_strip_f<T, C>(s, src, g.ns,
                         [&](int c, int j) {
                           const int64_t o = (int64_t)j * s.N1 + c;
                           return Pair<T>{__ldg(z + o), __ldg(po + o)};
                         },
                         [&](const Pair<T>& r, int, int) { return fma(bb, r.b, r.a); }, out);
  } else {
    stream_strip<T, C>(s, src, g.ns, [&](int c, int j) {
      const int64_t o = (int64_t)j * s.N1 + c;
      return fma(bb, __ldg(po + o), __ldg(z + o));
    }, out);
  }
  warp_partial(dot, part, s.part_idx);
  prof_tick(prof);
}

// Pre-smoothing from zero and residual: e = W b, r1 = b - A e.
template <class T, bool C>
__global__ void __launch_bounds__(SBLOCK) k_mgpre2(Grid g, const T* __restrict__ K, int64_t cs,
                                                   const T* __restrict__ W,
                                                   const T* __restrict__ Bv, T* __restrict__ E,
                                                   T* __restrict__ R1,
                                                   const int32_t* __restrict__ active, Prof prof) {
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  const Strip s = strip_of(g);
  const T* w_ = W + b * g.ns;
  const T* bv = Bv + b * g.ns;
  T* e = E + b * g.ns;
  T* r1 = R1 + b * g.ns;
  auto field = [&](int c, int j) {
    const int64_t o = (int64_t)j * s.N1 + c;
    return __ldg(w_ + o) * __ldg(bv + o);
  };
  if constexpr (kResidualForm<T>) {
    stream_strip_r<T, C, true>(s, K + b * cs, g.ns, field,
                               [&](int j) { return __ldg(bv + (int64_t)j * s.N1 + s.c); },
                               [&](int j, T ev, T rv, T) {
                                 const int64_t o = (int64_t)j * s.N1 + s.c;
                                 e[o] = ev;
                                 r1[o] = rv;
                               });
  } else {
    stream_strip_f<T, C>(s, K + b * cs, g.ns,
                         [&](int c, int j) {
                           const int64_t o = (int64_t)j * s.N1 + c;
                           return Pair<T>{__ldg(w_ + o), __ldg(bv + o)};
                         },
                         [&](const Pair<T>& r, int, int) { return r.a * r.b; },
                         [&](int j, T ev, T ax) {
                           const int64_t o = (int64_t)j * s.N1 + s.c;
                           e[o] = ev;
                           r1[o] = interior2(s.n, s.c, j) ? __ldg(bv + o) - ax : T(0);
                         });
  }
  prof_tick(prof);
}

// Bilinear prolongation of the coarse correction at fine node (i, j).
template <class T>
__device__ __forceinline__ T prolong2(const T* __restrict__ Ec, int nc, int i, int j) {
  const int N1c = nc + 1;
  const T* e = Ec + (int64_t)(j >> 1) * N1c + (i >> 1);
  const bool ox = i & 1, oy = j & 1;
  T v0 = __ldg(e);
  if (ox) v0 = T(0.5) * (v0 + __ldg(e + 1));
  if (!oy) return v0;
  T v1 = __ldg(e + N1c);
  if (ox) v1 = T(0.5) * (v1 + __ldg(e + N1c + 1));
  return T(0.5) * (v0 + v1);
}

// The same value split into its loads (the node's e and the coarse values
// it interpolates, 0 where the parity needs none) and their combination, for
// fields formed one row after they are fetched.
template <class T>
struct RawP2 {
  T e, a, b, c, d;
};
template <class T>
__device__ __forceinline__ RawP2<T> prolong2_fetch(const T* __restrict__ e_node, const T* __restrict__ Ec,
                                                   int nc, int i, int j) {
  const int N1c = nc + 1;
  const T* p = Ec + (int64_t)(j >> 1) * N1c + (i >> 1);
  const bool ox = i & 1, oy = j & 1;
  RawP2<T> r;
  r.e = __ldg(e_node);
  r.a = __ldg(p);
  r.b = ox ? __ldg(p + 1) : T(0);
  r.c = oy ? __ldg(p + N1c) : T(0);
  r.d = (ox && oy) ? __ldg(p + N1c + 1) : T(0);
  return r;
}
template <class T>
__device__ __forceinline__ T prolong2_form(const RawP2<T>& r, int i, int j) {
  const bool ox = i & 1, oy = j & 1;
  T v0 = r.a;
  if (ox) v0 = T(0.5) * (v0 + r.b);
  if (!oy) return r.e + v0;
  T v1 = r.c;
  if (ox) v1 = T(0.5) * (v1 + r.d);
  return r.e + T(0.5) * (v0 + v1);
}

// Bilinear prolongation of the coarse correction, streamed down one fine
// node column i: at fine row j with coarse row J = j / 2, let H(J) be the sum
// of the two coarse values at columns i / 2 and (i + 1) / 2 of row J (twice
// the value when i is even). Then (P ec)(i, j) = H(J) / 2 on even rows and
// (H(J) + H(J + 1)) / 4 on odd rows; x + P ec is one FMA (even rows) or an
// add and an FMA (odd rows), and each coarse row sum is formed once per
// column. Rows must be visited in increasing order; the values equal the
// textbook form 0.5 (0.5 (a + b) + 0.5 (c + d)) bit for bit (the scalings
// are exact).
template <class T>
struct Prolong2 {
  const T* __restrict__ ec;   // coarse correction of the sample
  int N1c;                    // coarse nodes per row
  int jc = -2;                // coarse row held in hc
  bool have_next = false;     // hn holds H(jc + 1)
  T hc = T(0), hn = T(0);
  __device__ __forceinline__ T row_sum(int J, int i) const {
    const T* r = ec + (int64_t)J * N1c + (i >> 1);
    return __ldg(r) + __ldg(r + (i & 1));
  }
  // x + (P ec)(i, j)
  __device__ __forceinline__ T add(T x, int i, int j) {
    const int J = j >> 1;
    if (J != jc) {
      hc = (have_next && J == jc + 1) ? hn : row_sum(J, i);
      jc = J;
      have_next = false;
    }
    if (!(j & 1)) return fma(T(0.5), hc, x);
    if (!have_next) {
      hn = row_sum(J + 1, i);
      have_next = true;
    }
    return fma(T(0.25), hc + hn, x);
  }
};

// out = e' + W (b - A e'), e' = e + P ec; partials of b.out when part != nullptr.
template <class T, bool C>
__global__ void __launch_bounds__(SBLOCK) k_mgpost2(Grid g, int64_t nsc, const T* __restrict__ K, int64_t cs,
                                                    const T* __restrict__ W,
                                                    const T* __restrict__ Bv,
                                                    const T* __restrict__ E,
                                                    const T* __restrict__ Ec, T* __restrict__ Out,
                                                    const int32_t* __restrict__ active,
                                                    double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  const Strip s = strip_of(g);
  const int nc = g.n / 2;
  const T* ec = Ec + b * nsc;
  const T* e = E + b * g.ns;
  const T* w_ = W + b * g.ns;
  const T* bv = Bv + b * g.ns;
  T* out = Out + b * g.ns;
  T dot = T(0);
  if constexpr (kResidualForm<T>) {
    Prolong2<T> pr{ec, nc + 1};
    stream_strip_r<T, C, true>(s, K + b * cs, g.ns,
                               [&](int c, int j) { return pr.add(__ldg(e + (int64_t)j * s.N1 + c), c, j); },
                               [&](int j) { return __ldg(bv + (int64_t)j * s.N1 + s.c); },
                               [&](int j, T ev, T rv, T bval) {
                                 const int64_t o = (int64_t)j * s.N1 + s.c;
                                 T ov = T(0);
                                 if (interior2(s.n, s.c, j)) {
                                   ov = fma(__ldg(w_ + o), rv, ev);
                                   dot = fma(bval, ov, dot);
                                 }
                                 out[o] = ov;
                               });
  } else {
    stream_strip_f<T, C>(s, K + b * cs, g.ns,
                       [&](int c, int j) { return prolong2_fetch(e + (int64_t)j * s.N1 + c, ec, nc, c, j); },
                       [&](const RawP2<T>& r, int c, int j) { return prolong2_form(r, c, j); },
                       [&](int j, T ev, T ax) {
                         const int64_t o = (int64_t)j * s.N1 + s.c;
                         T ov = T(0);
                         if (interior2(s.n, s.c, j)) {
                           const T bval = __ldg(bv + o);
                           ov = fma(__ldg(w_ + o), bval - ax, ev);
                           dot = fma(bval, ov, dot);
                         }
                         out[o] = ov;
                       });
  }
  if (part) warp_partial(dot, part, s.part_idx);
  prof_tick(prof);
}

// k_mgpost2 for the FP32 inner solve (kappa form), on paired rows with the
// prolongation streamed as in Prolong2; its own kernel so that it can be
// held to 56 registers (9 CTAs per SM) without touching the FP64 kernels.
__global__ void __launch_bounds__(SBLOCK, 9) k_mgpost2f(Grid g, int64_t nsc, const float* __restrict__ K,
                                                        const float* __restrict__ W,
                                                        const float* __restrict__ Bv,
                                                        const float* __restrict__ E,
                                                        const float* __restrict__ Ec, float* __restrict__ Out,
                                                        const int32_t* __restrict__ active,
                                                        double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  const Strip s = strip_of(g);
  const int nc = g.n / 2;
  const float* ec = Ec + b * nsc;
  const float* e = E + b * g.ns;
  const float* w_ = W + b * g.ns;
  const float* bv = Bv + b * g.ns;
  float* out = Out + b * g.ns;
  float dot = 0.f;
  // FP32 on paired rows with the prolongation streamed as in Prolong2.
  // Strips start on even rows, so a pair is (j, j + 1) = (2J + 1, 2J + 2):
  // x(2J + 1) = e + H(J)/4 + H(J + 1)/4 and x(2J + 2) = e + H(J + 1)/2, with
  // H(J) the sum of the coarse values at columns c / 2 and (c + 1) / 2 of
  // coarse row J. The fetch of a pair loads coarse row J + 1; H(J) is the
  // previous pair's (hprev). Bitwise equal to prolong2_form (the scalings
  // are exact).
  static_assert(SROWS % 2 == 0, "strips start on even rows");
  const int n = s.n, c = s.c, N1c = nc + 1;
  const bool cin = c >= 1 && c < n;
  const float* __restrict__ ecol = ec + (cin ? (c >> 1) : 0);
  const int dc = c & 1;
  auto hrow = [&](int J, float& a, float& bb) {
    a = bb = 0.f;
    if (cin && J >= 0 && J <= nc) {
      const float* p = ecol + J * N1c;
      a = __ldg(p);
      bb = __ldg(p + dc);
    }
  };
  float hprev;
  {
    float a, bb;
    hrow(s.y0 / 2 - 1, a, bb);
    hprev = a + bb;
  }
  // The pair of field rows (j, j + 1) is formed in the step that outputs rows
  // j - 1 and j, so its fetch also loads b and W of those two rows (bw):
  // they get the same step of latency as the field.
  struct RawPE {
    float e0, e1, a, b, b0, b1, w0, w1;
  };
  float bw[4] = {0.f, 0.f, 0.f, 0.f};   // b, W of the even and the odd output row of the step
  stream_strip_pair(
      s, K + b * g.es,
      [&](int j) {
        RawPE r;
        const float* ej = e + (j * s.N1 + c);
        r.e0 = interior2(n, c, j) ? __ldg(ej) : 0.f;
        r.e1 = interior2(n, c, j + 1) ? __ldg(ej + s.N1) : 0.f;
        hrow((j + 1) >> 1, r.a, r.b);
        const bool o0 = s.out && interior2(n, c, j - 1), o1 = s.out && interior2(n, c, j);
        r.b0 = o0 ? __ldg(bv + (j - 1) * s.N1 + c) : 0.f;
        r.w0 = o0 ? __ldg(w_ + (j - 1) * s.N1 + c) : 0.f;
        r.b1 = o1 ? __ldg(bv + j * s.N1 + c) : 0.f;
        r.w1 = o1 ? __ldg(w_ + j * s.N1 + c) : 0.f;
        return r;
      },
      [&](const RawPE& r, int j) {
        const float h = r.a + r.b;
        const float x0 = interior2(n, c, j) ? fmaf(0.25f, hprev + h, r.e0) : 0.f;
        const float x1 = interior2(n, c, j + 1) ? fmaf(0.5f, h, r.e1) : 0.f;
        hprev = h;
        bw[0] = r.b0;
        bw[1] = r.w0;
        bw[2] = r.b1;
        bw[3] = r.w1;
        return make_float2(x0, x1);
      },
      [&](int j, float ev, float ax) {
        // the step's even output row takes bw[0..1], its odd one bw[2..3]
        const int o = j * s.N1 + c;
        const float bval = (j & 1) ? bw[2] : bw[0];
        const float wval = (j & 1) ? bw[3] : bw[1];
        float ov = 0.f;
        if (interior2(n, c, j)) {
          ov = fmaf(wval, bval - ax, ev);
          dot = fmaf(bval, ov, dot);
        }
        out[o] = ov;
      });
  if (part) warp_partial(dot, part, s.part_idx);
  prof_tick(prof);
}

// Mixed form, outer FP64 residual: r = b - A(kappa) u (b_i = h^2), partials of r.r.
template <bool C>
__global__ void __launch_bounds__(SBLOCK) k_resid2(Grid g, const double* __restrict__ K, int64_t cs,
                                                   const double* __restrict__ U,
                                                   double* __restrict__ R,
                                                   const int32_t* __restrict__ active,
                                                   double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  const Strip s = strip_of(g);
  const double h2 = g.h * g.h;
  const double* u = U + b * g.ns;
  double* r = R + b * g.ns;
  double dot = 0.0;
  stream_strip_r<double, C, true>(s, K + b * cs, g.ns,
                                  [&](int c, int j) { return __ldg(u + (int64_t)j * s.N1 + c); },
                                  [&](int) { return h2; },
                                  [&](int j, double, double rv, double) {
                                    dot = fma(rv, rv, dot);
                                    r[(int64_t)j * s.N1 + s.c] = rv;
                                  });
  warp_partial(dot, part, s.part_idx);
  prof_tick(prof);
}

// Coefficient blocks of the FP64 2D operator (see WinC): per sample
// cd, ce, cn at every node (kappa outside the mesh counts as 0), then
// q = -kappa/3 per element; with W, also the smoother weights W = omega / D
// (the same values k_winv2 computes, without a second pass over kappa).
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_coef2(Grid g, const T* __restrict__ K,
                                                        T* __restrict__ Cb, int64_t cs, double omega,
                                                        T* __restrict__ W) {
  const int64_t b = blockIdx.y;
  const int n = g.n, N1 = n + 1;
  const int64_t nn = (int64_t)N1 * N1, ne = (int64_t)n * n;
  const T* k = K + b * g.es;
  T* cd = Cb + b * cs;
  T* ce = cd + g.ns;
  T* cn = cd + 2 * g.ns;
  T* q = cd + 3 * g.ns;
  const int64_t e0 = (int64_t)blockIdx.x * FLAT_ELEMS;
  const int64_t e1 = min(e0 + (int64_t)FLAT_ELEMS, g.ns);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += FLAT_THREADS) {
    T d = T(0), xe = T(0), xn = T(0);
    if (e < nn) {
      const int ei = (int)e, j = ei / N1, i = ei - j * N1;
      const T ksw = kap_at(k, n, i - 1, j - 1), kse = kap_at(k, n, i, j - 1);
      const T knw = kap_at(k, n, i - 1, j), kne = kap_at(k, n, i, j);
      if (interior2(n, i, j)) d = Consts<T>::c23 * ((ksw + kse) + (knw + kne));
      xe = -Consts<T>::c16 * (kse + kne);
      xn = -Consts<T>::c16 * (knw + kne);
    }
    cd[e] = d;
    ce[e] = xe;
    cn[e] = xn;
    if (W) W[b * g.ns + e] = d != T(0) ? T(omega) / d : T(0);   // d = 0 exactly off the interior
    if (e < g.es) q[e] = e < ne ? -Consts<T>::c13 * __ldg(k + e) : T(0);
  }
}

// ------------------------------------------------------------ flat kernels

template <class T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int L = 4;
};
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int L = 2;
};

// 16-byte vector viewed as an array of lanes (kept in registers).
template <class T>
union Pack {
  typename Vec<T>::V v;
  T a[Vec<T>::L];
};

// CTA-wide sum of per-thread partials into part[b * tiles_f + blockIdx.x].
__device__ __forceinline__ void cta_partial(double v, double* __restrict__ part, int64_t tiles_f) {
  __shared__ double s_w[FLAT_THREADS / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
#pragma unroll
    for (int w = 0; w < FLAT_THREADS / 32; ++w) r += s_w[w];
    part[(int64_t)blockIdx.y * tiles_f + blockIdx.x] = r;
  }
}

inline dim3 fgrid(const Grid& g, int64_t B) { return dim3((unsigned)g.fx, (unsigned)B, 1); }

// Nodes of one sample: (n+1)^d. Entries between that and the sample stride
// are padding that no kernel reads or writes.
__device__ __forceinline__ int64_t nodes_of(const Grid& g) {
  const int64_t N1 = g.n + 1;
  return g.dim == 2 ? N1 * N1 : N1 * N1 * N1;
}

// Range of whole 16-byte vectors of this CTA within one sample's nodes, and
// the scalar tail [tail0, nn) that the last CTA handles element by element.
template <class T>
__device__ __forceinline__ void flat_range(const Grid& g, int64_t& v0, int64_t& v1, int64_t& tail0,
                                           int64_t& nn) {
  nn = nodes_of(g);
  const int64_t nv = nn / Vec<T>::L;
  const int64_t per = FLAT_ELEMS / Vec<T>::L;
  v0 = (int64_t)blockIdx.x * per;
  v1 = min(v0 + per, nv);
  tail0 = (blockIdx.x == gridDim.x - 1) ? nv * Vec<T>::L : nn;
}

// x = 0 at every node of every sample (16-byte stores; the initial iterate
// of a solve whose residual is set elsewhere)
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_zero_flat(Grid g, T* __restrict__ X, Prof prof) {
  using V = typename Vec<T>::V;
  const int64_t b = blockIdx.y;
  int64_t v0, v1, t0, nn;
  flat_range<T>(g, v0, v1, t0, nn);
  V* x = reinterpret_cast<V*>(X + b * g.ns);
  V zero;
  memset(&zero, 0, sizeof(zero));
  for (int64_t v = v0 + threadIdx.x; v < v1; v += FLAT_THREADS) x[v] = zero;
  for (int64_t e = t0 + threadIdx.x; e < nn; e += FLAT_THREADS) X[b * g.ns + e] = T(0);
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// x += alpha p, r -= alpha q, partials of r.r
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_xr_flat(Grid g, T* __restrict__ X,
                                                          const T* __restrict__ P, T* __restrict__ R,
                                                          const T* __restrict__ Q,
                                                          const double* __restrict__ alpha,
                                                          const int32_t* __restrict__ active,
                                                          double* __restrict__ part, Prof prof) {
  using V = typename Vec<T>::V;
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const T a = (T)alpha[b];
  int64_t v0, v1, t0, nn;
  flat_range<T>(g, v0, v1, t0, nn);
  V* x = reinterpret_cast<V*>(X + b * g.ns);
  const V* p = reinterpret_cast<const V*>(P + b * g.ns);
  V* r = reinterpret_cast<V*>(R + b * g.ns);
  const V* q = reinterpret_cast<const V*>(Q + b * g.ns);
  T dot = T(0);
  for (int64_t v = v0 + threadIdx.x; v < v1; v += FLAT_THREADS) {
    Pack<T> xv, pv, rv, qv;
    xv.v = x[v];
    pv.v = p[v];
    rv.v = r[v];
    qv.v = q[v];
#pragma unroll
    for (int i = 0; i < Vec<T>::L; ++i) {
      xv.a[i] = fma(a, pv.a[i], xv.a[i]);
      rv.a[i] = fma(-a, qv.a[i], rv.a[i]);
      dot = fma(rv.a[i], rv.a[i], dot);
    }
    x[v] = xv.v;
    r[v] = rv.v;
  }
  for (int64_t e = t0 + threadIdx.x; e < nn; e += FLAT_THREADS) {
    T* xs = X + b * g.ns;
    T* rs = R + b * g.ns;
    xs[e] = fma(a, P[b * g.ns + e], xs[e]);
    rs[e] = fma(-a, Q[b * g.ns + e], rs[e]);
    dot = fma(rs[e], rs[e], dot);
  }
  cta_partial((double)dot, part, g.tiles_f);
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// z = Winv r, partials of r.z
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_jz_flat(Grid g, const T* __restrict__ Wv,
                                                          const T* __restrict__ R, T* __restrict__ Z,
                                                          const int32_t* __restrict__ active,
                                                          double* __restrict__ part, Prof prof) {
  using V = typename Vec<T>::V;
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  int64_t v0, v1, t0, nn;
  flat_range<T>(g, v0, v1, t0, nn);
  const V* w = reinterpret_cast<const V*>(Wv + b * g.ns);
  const V* r = reinterpret_cast<const V*>(R + b * g.ns);
  V* z = reinterpret_cast<V*>(Z + b * g.ns);
  T dot = T(0);
  for (int64_t v = v0 + threadIdx.x; v < v1; v += FLAT_THREADS) {
    Pack<T> wv, rv, zv;
    wv.v = w[v];
    rv.v = r[v];
#pragma unroll
    for (int i = 0; i < Vec<T>::L; ++i) {
      zv.a[i] = wv.a[i] * rv.a[i];
      dot = fma(rv.a[i], zv.a[i], dot);
    }
    z[v] = zv.v;
  }
  for (int64_t e = t0 + threadIdx.x; e < nn; e += FLAT_THREADS) {
    const T rv = R[b * g.ns + e];
    const T zv = Wv[b * g.ns + e] * rv;
    Z[b * g.ns + e] = zv;
    dot = fma(rv, zv, dot);
  }
  cta_partial((double)dot, part, g.tiles_f);
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// x = 0 and, if R != nullptr, r = h^2 at interior nodes (b_i = int phi_i for f = 1).
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_init_flat(Grid g, T* __restrict__ X,
                                                            T* __restrict__ R, Prof prof) {
  const int64_t b = blockIdx.y;
  const int64_t e0 = (int64_t)blockIdx.x * FLAT_ELEMS;
  const int64_t e1 = min(e0 + (int64_t)FLAT_ELEMS, g.ns);
  const int N1 = g.n + 1;
  const int64_t nn = (int64_t)N1 * N1;
  const T h2 = T(g.h * g.h);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += FLAT_THREADS) {
    X[b * g.ns + e] = T(0);
    if (R) {
      T v = T(0);
      if (e < nn) {
        const int ei = (int)e, j = ei / N1, i = ei - j * N1;   // e < (n + 1)^2 < 2^31
        if (interior2(g.n, i, j)) v = h2;
      }
      R[b * g.ns + e] = v;
    }
  }
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// Partials of w_i x_i for the QoI weights (exact Q1 integral mean):
// domain: w = h^2 at interior nodes; box [L, H]^2 in node indices:
// w = h^2 chi_x chi_y / |box|, chi = 1 strictly inside, 1/2 on a face.
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_qoi_flat(Grid g, int box, int L, int H,
                                                           double inv_vol,
                                                           const T* __restrict__ X,
                                                           double* __restrict__ part, Prof prof) {
  const int64_t b = blockIdx.y;
  const int64_t e0 = (int64_t)blockIdx.x * FLAT_ELEMS;
  const int64_t e1 = min(e0 + (int64_t)FLAT_ELEMS, g.ns);
  const int N1 = g.n + 1;
  const int64_t nn = (int64_t)N1 * N1;
  const double h2 = g.h * g.h;
  double v = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1 && e < nn; e += FLAT_THREADS) {
    const int ei = (int)e, j = ei / N1, i = ei - j * N1;   // e < (n + 1)^2 < 2^31
    if (!interior2(g.n, i, j)) continue;
    double w = h2;
    if (box) {
      const double cx = (i > L && i < H) ? 1.0 : ((i == L || i == H) ? 0.5 : 0.0);
      const double cy = (j > L && j < H) ? 1.0 : ((j == L || j == H) ? 0.5 : 0.0);
      w = h2 * cx * cy * inv_vol;
    }
    v += w * (double)X[b * g.ns + e];
  }
  cta_partial(v, part, g.tiles_f);
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// Mixed form, pointwise refinement steps per active sample:
//   mode 0: rhs32 = r / scale   (unit-norm right-hand side of the inner solve)
//   mode 1: u += scale * d32    (apply the inner correction)
__global__ void __launch_bounds__(FLAT_THREADS) k_refine_flat(Grid g, int mode,
                                                              double* __restrict__ Dbl,
                                                              float* __restrict__ Flt,
                                                              const double* __restrict__ scale,
                                                              const int32_t* __restrict__ active,
                                                              Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const double sc = scale[b];
  __shared__ double s_inv;   // one division per CTA, not per thread
  if (threadIdx.x == 0) s_inv = 1.0 / sc;
  __syncthreads();
  const double inv = s_inv;
  int64_t v0, v1, t0, nn;
  flat_range<float>(g, v0, v1, t0, nn);
  double2* d = reinterpret_cast<double2*>(Dbl + b * g.ns);
  float4* f = reinterpret_cast<float4*>(Flt + b * g.ns);
  for (int64_t v = v0 + threadIdx.x; v < v1; v += FLAT_THREADS) {
    double2 a = d[2 * v], c = d[2 * v + 1];
    if (mode == 0) {
      f[v] = make_float4((float)(a.x * inv), (float)(a.y * inv), (float)(c.x * inv),
                         (float)(c.y * inv));
    } else {
      const float4 fv = f[v];
      a.x = fma(sc, (double)fv.x, a.x);
      a.y = fma(sc, (double)fv.y, a.y);
      c.x = fma(sc, (double)fv.z, c.x);
      c.y = fma(sc, (double)fv.w, c.y);
      d[2 * v] = a;
      d[2 * v + 1] = c;
    }
  }
  for (int64_t e = t0 + threadIdx.x; e < nn; e += FLAT_THREADS) {
    if (mode == 0) {
      Flt[b * g.ns + e] = (float)(Dbl[b * g.ns + e] * inv);
    } else {
      Dbl[b * g.ns + e] = fma(sc, (double)Flt[b * g.ns + e], Dbl[b * g.ns + e]);
    }
  }
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// --------------------------------------------------------- per-node kernels

// W = omega / D at every node (0 on the boundary).
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_winv2(Grid g, const T* __restrict__ K,
                                                        double omega, T* __restrict__ W) {
  const int64_t b = blockIdx.y;
  const int N1 = g.n + 1;
  const int64_t nn = (int64_t)N1 * N1;
  const T* k = K + b * g.es;
  const int64_t e0 = (int64_t)blockIdx.x * FLAT_ELEMS;
  const int64_t e1 = min(e0 + (int64_t)FLAT_ELEMS, g.ns);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += FLAT_THREADS) {
    T w = T(0);
    if (e < nn) {
      const int ei = (int)e, j = ei / N1, i = ei - j * N1;   // e < (n + 1)^2 < 2^31
      if (interior2(g.n, i, j)) {
        const T* r0 = k + (int64_t)(j - 1) * g.n + (i - 1);
        const T d = Consts<T>::c23 * ((r0[0] + r0[1]) + (r0[g.n] + r0[g.n + 1]));
        w = T(omega) / d;
      }
    }
    W[b * g.ns + e] = w;
  }
}

// Full weighting (transpose of bilinear prolongation), one thread per coarse node:
// bc(I, J) = sum_{di,dj in -1..1} w(di) w(dj) r1(2I + di, 2J + dj), w(0) = 1, w(+-1) = 1/2.
template <class T>
__global__ void __launch_bounds__(FLAT_THREADS) k_restrict2(Grid gc, int64_t nsf,
                                                            const T* __restrict__ R1,
                                                            T* __restrict__ Bc,
                                                            const int32_t* __restrict__ active,
                                                            Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const int nc = gc.n;
  const int N1c = nc + 1;
  const int N1 = 2 * nc + 1;
  const int64_t nn = (int64_t)N1c * N1c;
  const int64_t e0 = (int64_t)blockIdx.x * FLAT_ELEMS;
  const int64_t e1 = min(e0 + (int64_t)FLAT_ELEMS, gc.ns);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += FLAT_THREADS) {
    T v = T(0);
    if (e < nn) {
      const int ei = (int)e, J = ei / N1c, I = ei - J * N1c;
      if (interior2(nc, I, J)) {
        const T* r = R1 + b * nsf + (int64_t)(2 * J) * N1 + 2 * I;
        const T h = T(0.5);
        const T row0 = h * __ldg(r - N1 - 1) + __ldg(r - N1) + h * __ldg(r - N1 + 1);
        const T row1 = h * __ldg(r - 1) + __ldg(r) + h * __ldg(r + 1);
        const T row2 = h * __ldg(r + N1 - 1) + __ldg(r + N1) + h * __ldg(r + N1 + 1);
        v = h * (row0 + row2) + row1;
      }
    }
    Bc[b * gc.ns + e] = v;
  }
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// The same full weighting on warp strips (the FP64 form): a warp owns 32
// coarse columns I (one per lane) and walks RSTRIP_ROWS coarse rows J. On
// each fine row a lane loads one aligned pair of fine values, (2I, 2I + 1) on
// even rows and (2I - 1, 2I) on odd rows (fine rows have an odd length, so on
// odd rows the pair starting at 2I - 1 is the aligned one), and takes the
// third value of its row sum h a + b + h c from the neighbouring lane (lanes
// 0 and 31 load theirs); the sum over the odd fine row 2J + 1 is carried to
// coarse row J + 1, so each fine value is read once (twice on the first row
// of a chunk). Every node of the coarse rows is written (0 off the interior).
constexpr int RSTRIP_ROWS = 16;
template <class T>
struct Vec2;
template <>
struct Vec2<float> {
  using V = float2;
};
template <>
struct Vec2<double> {
  using V = double2;
};

template <class T>
__global__ void __launch_bounds__(SBLOCK) k_restrict2s(Grid gc, int64_t nsf, const T* __restrict__ R1,
                                                       T* __restrict__ Bc, const int32_t* __restrict__ active,
                                                       Prof prof) {
  using V2 = typename Vec2<T>::V;
  constexpr unsigned FULL = 0xffffffffu;
  const int64_t b = blockIdx.z;
  if (!active[b]) return;
  if (prof.acc && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
  const int nc = gc.n, N1c = nc + 1, N1 = 2 * nc + 1;
  const int lane = threadIdx.x & 31;
  const int I0 = (blockIdx.x * SWARPS + (threadIdx.x >> 5)) * 32;
  if (I0 > nc) return;   // the whole strip lies beyond the row
  const int I = I0 + lane;
  const int J0 = blockIdx.y * RSTRIP_ROWS, J1 = min(J0 + RSTRIP_ROWS, N1c);
  const T* __restrict__ r = R1 + b * nsf;
  T* __restrict__ bc = Bc + b * gc.ns;
  const T h = T(0.5);
  const bool ev_ld = I < nc;              // (2I, 2I + 1) lies in the fine row
  const bool od_ld = I >= 1 && I <= nc;   // (2I - 1, 2I) lies in the fine row
  // h f(2I - 1) + f(2I) + h f(2I + 1) on the even fine row fr (fr * N1 even)
  auto even_sum = [&](int fr) -> T {
    const T* row = r + (int64_t)fr * N1;
    V2 p{T(0), T(0)};
    if (ev_ld) p = __ldg(reinterpret_cast<const V2*>(row + 2 * I));
    T left = __shfl_up_sync(FULL, p.y, 1);
    if (lane == 0) left = I >= 1 ? __ldg(row + 2 * I - 1) : T(0);
    return h * left + p.x + h * p.y;
  };
  // the same on the odd fine row fr (fr * N1 odd)
  auto odd_sum = [&](int fr) -> T {
    const T* row = r + (int64_t)fr * N1;
    V2 p{T(0), T(0)};
    if (od_ld) p = __ldg(reinterpret_cast<const V2*>(row + 2 * I - 1));
    T right = __shfl_down_sync(FULL, p.x, 1);
    if (lane == 31) right = I < nc ? __ldg(row + 2 * I + 1) : T(0);
    return h * p.x + p.y + h * right;
  };
  T oprev = J0 >= 1 ? odd_sum(2 * J0 - 1) : T(0);
#pragma unroll 4
  for (int J = J0; J < J1; ++J) {
    const bool jin = J >= 1 && J < nc;   // uniform across the warp
    T o = T(0), ev = T(0);
    if (J < nc) o = odd_sum(2 * J + 1);
    if (jin) ev = even_sum(2 * J);
    T v = T(0);
    if (jin && I >= 1 && I < nc) v = h * (oprev + o) + ev;
    if (I <= nc) bc[(int64_t)J * N1c + I] = v;
    oprev = o;
  }
}

// Nested initial guess: x = P uc, the coarse-mesh solution interpolated
// bilinearly to the fine mesh (0 on the boundary), one thread per node.
__global__ void __launch_bounds__(FLAT_THREADS) k_prolong_guess2(Grid g, int64_t nsc,
                                                                 const double* __restrict__ Uc,
                                                                 double* __restrict__ X,
                                                                 const int32_t* __restrict__ active,
                                                                 Prof prof) {
  const int64_t b = blockIdx.y;
  if (!active[b]) return;
  const int n = g.n, N1 = n + 1;
  const int64_t nn = (int64_t)N1 * N1;
  const double* uc = Uc + b * nsc;
  const int64_t e0 = (int64_t)blockIdx.x * FLAT_ELEMS;
  const int64_t e1 = min(e0 + (int64_t)FLAT_ELEMS, g.ns);
  for (int64_t e = e0 + threadIdx.x; e < e1; e += FLAT_THREADS) {
    double v = 0.0;
    if (e < nn) {
      const int ei = (int)e, j = ei / N1, i = ei - j * N1;
      if (interior2(n, i, j)) v = prolong2(uc, n / 2, i, j);
    }
    X[b * g.ns + e] = v;
  }
  if (prof.acc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof.acc, prof.per_sample);
}

// Coarsest grid (n = 2, one unknown): e = b / D exactly.
template <class T>
__global__ void k_coarse2(int64_t ns, int64_t es, const T* __restrict__ K, const T* __restrict__ Bv,
                          T* __restrict__ E, const int32_t* __restrict__ active, int64_t B) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  const int64_t off = b * ns;
  const T* k = K + b * es;
  const T d = Consts<T>::c23 * ((k[0] + k[1]) + (k[2] + k[3]));
  for (int q = 0; q < 9; ++q) E[off + q] = T(0);
  E[off + 4] = Bv[off + 4] / d;
}


// --------------------------------------------- fused bottom of the V-cycle

constexpr int BOTTOM_THREADS = 512;

// Bilinear prolongation from a coarse array in shared memory.
template <class T>
__device__ __forceinline__ T prolong2_s(const T* ec, int nc, int i, int j) {
  const int N1c = nc + 1;
  const T* e = ec + (j >> 1) * N1c + (i >> 1);
  const bool ox = i & 1, oy = j & 1;
  T v0 = e[0];
  if (ox) v0 = T(0.5) * (v0 + e[1]);
  if (!oy) return v0;
  T v1 = e[N1c];
  if (ox) v1 = T(0.5) * (v1 + e[N1c + 1]);
  return T(0.5) * (v0 + v1);
}

// Levels k0 .. K-1 of the V-cycle for one sample per CTA, in shared memory
// (per level: b, e and a third array for r1, then the level's output): the
// same steps and arithmetic as k_mgpre2, k_restrict2, k_coarse2 and
// k_mgpost2 (C: FP64 coefficient form with residuals accumulated from b;
// else kappa form), with a barrier between steps instead of a launch.
// Operator data, W and kappa are read from global memory (cached).
template <class T, bool C>
__global__ void __launch_bounds__(BOTTOM_THREADS) k_bottom2(BottomLevels<T> lv, const T* __restrict__ Bv,
                                                            T* __restrict__ Out,
                                                            const int32_t* __restrict__ active,
                                                            Prof prof) {
  const int64_t smp = blockIdx.x;
  if (!active[smp]) return;
  extern __shared__ __align__(16) unsigned char bottom_raw[];
  T* sm = reinterpret_cast<T*>(bottom_raw);
  const int L = lv.L;
  const int tid = threadIdx.x;
  // level l's arrays start at 3 x (nodes of the levels before it)
  auto base = [&](int l) -> T* {
    int off = 0;
    for (int m = 0; m < l; ++m) off += 3 * (lv.g[m].n + 1) * (lv.g[m].n + 1);
    return sm + off;
  };
  // f - (A e)(c, j) at an interior node of level l (e in shared memory)
  auto resid = [&](int l, const T* e, int c, int j, T f) -> T {
    const Grid& g = lv.g[l];
    const int n = g.n, N1 = n + 1, o = j * N1 + c, eo = j * n + c;
    if constexpr (C) {
      const T* cb = lv.coef[l] + smp * (3 * g.ns + g.es);
      const T* cd = cb;
      const T* ce = cb + g.ns;
      const T* cn = cb + 2 * g.ns;
      const T* q = cb + 3 * g.ns;
      WinC<T> w;
      w.v0 = e[o]; w.l0 = e[o - 1]; w.r0 = e[o + 1];
      w.vp = e[o + N1]; w.lp = e[o + N1 - 1]; w.rp = e[o + N1 + 1];
      w.vm = e[o - N1]; w.lm = e[o - N1 - 1]; w.rm = e[o - N1 + 1];
      w.qb = __ldg(q + eo); w.qbl = __ldg(q + eo - 1);
      w.qa = __ldg(q + eo - n); w.qal = __ldg(q + eo - n - 1);
      w.cd = __ldg(cd + o); w.ce = __ldg(ce + o); w.ceW = __ldg(ce + o - 1);
      w.cnN = __ldg(cn + o); w.cnS = __ldg(cn + o - N1);
      return stencil_coef_res(w, f);
    } else {
      const T* k = lv.kap[l] + smp * g.es;
      Win<T> w;
      w.v0 = e[o]; w.l0 = e[o - 1]; w.r0 = e[o + 1];
      w.vp = e[o + N1]; w.lp = e[o + N1 - 1]; w.rp = e[o + N1 + 1];
      w.vm = e[o - N1]; w.lm = e[o - N1 - 1]; w.rm = e[o - N1 + 1];
      w.kb = __ldg(k + eo); w.kbl = __ldg(k + eo - 1);
      w.ka = __ldg(k + eo - n); w.kal = __ldg(k + eo - n - 1);
      return f - stencil_win(w);
    }
  };
  {
    const int N1 = lv.g[0].n + 1;
    T* b = base(0);
    const T* src = Bv + smp * lv.g[0].ns;
    for (int i = tid; i < N1 * N1; i += BOTTOM_THREADS) b[i] = src[i];
  }
  __syncthreads();
  // down: e = W b, r1 = b - A e, b_{l+1} = R r1
  for (int l = 0; l < L - 1; ++l) {
    const int n = lv.g[l].n, N1 = n + 1, nn = N1 * N1;
    T* b = base(l);
    T* e = b + nn;
    T* t = e + nn;
    const T* W = lv.w[l] + smp * lv.g[l].ns;
    for (int i = tid; i < nn; i += BOTTOM_THREADS) e[i] = __ldg(W + i) * b[i];
    __syncthreads();
    for (int i = tid; i < nn; i += BOTTOM_THREADS) {
      const int j = i / N1, c = i - j * N1;
      t[i] = interior2(n, c, j) ? resid(l, e, c, j, b[i]) : T(0);
    }
    __syncthreads();
    const int nc = lv.g[l + 1].n, N1c = nc + 1;
    T* bc = base(l + 1);
    for (int i = tid; i < N1c * N1c; i += BOTTOM_THREADS) {
      const int J = i / N1c, I = i - J * N1c;
      T v = T(0);
      if (interior2(nc, I, J)) {
        const T* r = t + (2 * J) * N1 + 2 * I;
        const T h = T(0.5);
        const T row0 = h * r[-N1 - 1] + r[-N1] + h * r[-N1 + 1];
        const T row1 = h * r[-1] + r[0] + h * r[1];
        const T row2 = h * r[N1 - 1] + r[N1] + h * r[N1 + 1];
        v = h * (row0 + row2) + row1;
      }
      bc[i] = v;
    }
    __syncthreads();
  }
  // coarsest grid (n = 2, one unknown): e = b / D
  {
    T* b = base(L - 1);
    T* e = b + 9;
    if (tid == 0) {
      const T* k = lv.kap[L - 1] + smp * lv.g[L - 1].es;
      const T d = Consts<T>::c23 * ((k[0] + k[1]) + (k[2] + k[3]));
      for (int q = 0; q < 9; ++q) e[q] = T(0);
      e[4] = b[4] / d;
    }
  }
  __syncthreads();
  // up: e += P e_c, out = e + W (b - A e)
  for (int l = L - 2; l >= 0; --l) {
    const int n = lv.g[l].n, N1 = n + 1, nn = N1 * N1;
    T* b = base(l);
    T* e = b + nn;
    T* t = e + nn;
    const int ncn = (lv.g[l + 1].n + 1) * (lv.g[l + 1].n + 1);
    const T* ec = base(l + 1) + ((l + 1 == L - 1) ? ncn : 2 * ncn);
    for (int i = tid; i < nn; i += BOTTOM_THREADS) {
      const int j = i / N1, c = i - j * N1;
      if (interior2(n, c, j)) e[i] = e[i] + prolong2_s(ec, n / 2, c, j);
    }
    __syncthreads();
    const T* W = lv.w[l] + smp * lv.g[l].ns;
    for (int i = tid; i < nn; i += BOTTOM_THREADS) {
      const int j = i / N1, c = i - j * N1;
      T ov = T(0);
      if (interior2(n, c, j)) ov = fma(__ldg(W + i), resid(l, e, c, j, b[i]), e[i]);
      t[i] = ov;
    }
    __syncthreads();
  }
  {
    const int N1 = lv.g[0].n + 1;
    const T* t = base(0) + 2 * N1 * N1;
    T* dst = Out + smp * lv.g[0].ns;
    for (int i = tid; i < N1 * N1; i += BOTTOM_THREADS) dst[i] = t[i];
  }
  if (prof.acc && tid == 0) atomicAdd(prof.acc, prof.per_sample);
}

}  // namespace

// ------------------------------------------------------------- launchers

namespace d2 {

cudaError_t prolong_guess(cudaStream_t s, const Grid& g, const Grid& coarse, const double* uc,
                          double* x, const int32_t* active, int64_t B, Prof p) {
  k_prolong_guess2<<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, coarse.ns, uc, x, active, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t apply(cudaStream_t s, const Grid& g, const T* kappa, const T* x, T* y, int64_t B, Prof p) {
  k_apply2<T><<<sgrid(g, B), SBLOCK, 0, s>>>(g, kappa, x, y, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t winv(cudaStream_t s, const Grid& g, const T* kappa, double omega, T* w, int64_t B) {
  k_winv2<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, kappa, omega, w);
  return cudaGetLastError();
}

template <class T>
cudaError_t pcg_init(cudaStream_t s, const Grid& g, T* x, T* r, int64_t B, Prof p) {
  if (r)
    k_init_flat<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, x, r, p);
  else
    k_zero_flat<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, x, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t zero_nodes(cudaStream_t s, const Grid& g, T* x, int64_t B, Prof p) {
  k_zero_flat<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, x, p);
  return cudaGetLastError();
}

// The coefficient-block stride per sample (node arrays cd, ce, cn, then q).
inline int64_t coef_stride(const Grid& g) { return 3 * g.ns + g.es; }

template <class T>
cudaError_t coef(cudaStream_t s, const Grid& g, const T* kappa, T* coef, int64_t B, double omega, T* w) {
  k_coef2<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, kappa, coef, coef_stride(g), omega, w);
  return cudaGetLastError();
}

template <class T>
cudaError_t pcg_pq(cudaStream_t s, const Grid& g, const T* kappa, const T* z, const T* p_old,
                   T* p_new, T* q, const Scalars& sc, double* part, int64_t B, Prof p, const T* coef) {
  if (coef)
    k_pq2<T, true><<<sgrid(g, B), SBLOCK, 0, s>>>(g, coef, coef_stride(g), z, p_old, p_new, q, sc.beta,
                                                  sc.active, part, p);
  else
    k_pq2<T, false><<<sgrid(g, B), SBLOCK, 0, s>>>(g, kappa, g.es, z, p_old, p_new, q, sc.beta, sc.active,
                                                   part, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t pcg_xr(cudaStream_t s, const Grid& g, T* x, const T* pv, T* r, const T* q,
                   const Scalars& sc, double* part, int64_t B, Prof p) {
  k_xr_flat<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, x, pv, r, q, sc.alpha, sc.active, part, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t jacobi_z(cudaStream_t s, const Grid& g, const T* winv, const T* r, T* z,
                     const Scalars& sc, double* part, int64_t B, Prof p) {
  k_jz_flat<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, winv, r, z, sc.active, part, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t mg_pre(cudaStream_t s, const Grid& g, const T* kappa, const T* w, const T* b, T* e,
                   T* r1, const int32_t* active, int64_t B, Prof p, const T* coef) {
  if (coef)
    k_mgpre2<T, true><<<sgrid(g, B), SBLOCK, 0, s>>>(g, coef, coef_stride(g), w, b, e, r1, active, p);
  else
    k_mgpre2<T, false><<<sgrid(g, B), SBLOCK, 0, s>>>(g, kappa, g.es, w, b, e, r1, active, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t restrict_(cudaStream_t s, const Grid& fine, const Grid& coarse, const T* r1, T* bc,
                      const int32_t* active, int64_t B, Prof p) {
  // FP64: warp strips (each fine value read once; 12% less restriction time
  // than one thread per node in the 2d-scale FP64 step). FP32: one thread per
  // node, whose independent loads hide the latency of the mostly L2-resident
  // FP32 arrays better (the strips took 31% longer there).
  if constexpr (sizeof(T) == 8) {
    const int N1c = coarse.n + 1;
    const dim3 grid((unsigned)((N1c + 32 * SWARPS - 1) / (32 * SWARPS)),
                    (unsigned)((N1c + RSTRIP_ROWS - 1) / RSTRIP_ROWS), (unsigned)B);
    k_restrict2s<T><<<grid, SBLOCK, 0, s>>>(coarse, fine.ns, r1, bc, active, p);
  } else {
    k_restrict2<T><<<fgrid(coarse, B), FLAT_THREADS, 0, s>>>(coarse, fine.ns, r1, bc, active, p);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t coarse_solve(cudaStream_t s, const Grid& g, const T* kappa, const T* b, T* e,
                         const int32_t* active, int64_t B) {
  k_coarse2<T><<<(unsigned)((B + 127) / 128), 128, 0, s>>>(g.ns, g.es, kappa, b, e, active, B);
  return cudaGetLastError();
}

template <class T>
cudaError_t mg_post(cudaStream_t s, const Grid& g, const Grid& coarse, const T* kappa, const T* w,
                    const T* b, const T* e, const T* ec, T* out, const int32_t* active,
                    double* part, int64_t B, Prof p, const T* coef) {
  if (coef)
    k_mgpost2<T, true><<<sgrid(g, B), SBLOCK, 0, s>>>(g, coarse.ns, coef, coef_stride(g), w, b, e, ec, out,
                                                      active, part, p);
  else if constexpr (sizeof(T) == 4)
    k_mgpost2f<<<sgrid(g, B), SBLOCK, 0, s>>>(g, coarse.ns, kappa, w, b, e, ec, out, active, part, p);
  else
    k_mgpost2<T, false><<<sgrid(g, B), SBLOCK, 0, s>>>(g, coarse.ns, kappa, g.es, w, b, e, ec, out,
                                                       active, part, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t qoi(cudaStream_t s, const Grid& g, int box, int L, int H, double inv_vol, const T* x,
                double* part, int64_t B, Prof p) {
  k_qoi_flat<T><<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, box, L, H, inv_vol, x, part, p);
  return cudaGetLastError();
}

cudaError_t resid64(cudaStream_t s, const Grid& g, const double* kappa, const double* u,
                    double* r, const int32_t* active, double* part, int64_t B, Prof p,
                    const double* coef) {
  if (coef)
    k_resid2<true><<<sgrid(g, B), SBLOCK, 0, s>>>(g, coef, coef_stride(g), u, r, active, part, p);
  else
    k_resid2<false><<<sgrid(g, B), SBLOCK, 0, s>>>(g, kappa, g.es, u, r, active, part, p);
  return cudaGetLastError();
}

cudaError_t to_rhs32(cudaStream_t s, const Grid& g, const double* r, const double* scale,
                     float* r32, const int32_t* active, int64_t B, Prof p) {
  k_refine_flat<<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, 0, const_cast<double*>(r), r32, scale,
                                                     active, p);
  return cudaGetLastError();
}

cudaError_t add_correction(cudaStream_t s, const Grid& g, double* u, const float* d32,
                           const double* scale, const int32_t* active, int64_t B, Prof p) {
  k_refine_flat<<<fgrid(g, B), FLAT_THREADS, 0, s>>>(g, 1, u, const_cast<float*>(d32), scale,
                                                     active, p);
  return cudaGetLastError();
}

template <class T>
cudaError_t mg_bottom(cudaStream_t s, const BottomLevels<T>& lv, const T* b, T* out,
                      const int32_t* active, int64_t B, Prof p) {
  if (lv.L < 2 || lv.L > MAX_BOTTOM || lv.g[lv.L - 1].n != 2 || lv.g[0].n > BOTTOM_MAX_N2)
    return cudaErrorInvalidValue;
  size_t smem = 0;
  for (int l = 0; l < lv.L; ++l) smem += 3 * (size_t)(lv.g[l].n + 1) * (lv.g[l].n + 1) * sizeof(T);
  // opt in (once per device) to the shared memory of the largest fused chain (64^2 .. 2^2)
  static std::atomic<uint64_t> opted{0};
  const cudaError_t attr = once_per_device(opted, [] {
    size_t most = 0;
    for (int n = BOTTOM_MAX_N2; n >= 2; n /= 2) most += 3 * (size_t)(n + 1) * (n + 1) * sizeof(T);
    cudaError_t e1 = cudaFuncSetAttribute(k_bottom2<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    cudaError_t e2 = cudaFuncSetAttribute(k_bottom2<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    return e1 != cudaSuccess ? e1 : e2;
  });
  if (attr != cudaSuccess) return attr;
  if (lv.coef[0])
    k_bottom2<T, true><<<(unsigned)B, BOTTOM_THREADS, smem, s>>>(lv, b, out, active, p);
  else
    k_bottom2<T, false><<<(unsigned)B, BOTTOM_THREADS, smem, s>>>(lv, b, out, active, p);
  return cudaGetLastError();
}

#define MLMC_INST2(T)                                                                              \
  template cudaError_t apply<T>(cudaStream_t, const Grid&, const T*, const T*, T*, int64_t, Prof); \
  template cudaError_t winv<T>(cudaStream_t, const Grid&, const T*, double, T*, int64_t);          \
  template cudaError_t pcg_init<T>(cudaStream_t, const Grid&, T*, T*, int64_t, Prof);              \
  template cudaError_t zero_nodes<T>(cudaStream_t, const Grid&, T*, int64_t, Prof);                \
  template cudaError_t pcg_pq<T>(cudaStream_t, const Grid&, const T*, const T*, const T*, T*, T*,  \
                                 const Scalars&, double*, int64_t, Prof, const T*);                \
  template cudaError_t coef<T>(cudaStream_t, const Grid&, const T*, T*, int64_t, double, T*);      \
  template cudaError_t pcg_xr<T>(cudaStream_t, const Grid&, T*, const T*, T*, const T*,            \
                                 const Scalars&, double*, int64_t, Prof);                          \
  template cudaError_t jacobi_z<T>(cudaStream_t, const Grid&, const T*, const T*, T*,              \
                                   const Scalars&, double*, int64_t, Prof);                        \
  template cudaError_t mg_pre<T>(cudaStream_t, const Grid&, const T*, const T*, const T*, T*, T*,  \
                                 const int32_t*, int64_t, Prof, const T*);                         \
  template cudaError_t restrict_<T>(cudaStream_t, const Grid&, const Grid&, const T*, T*,          \
                                    const int32_t*, int64_t, Prof);                                \
  template cudaError_t coarse_solve<T>(cudaStream_t, const Grid&, const T*, const T*, T*,          \
                                       const int32_t*, int64_t);                                   \
  template cudaError_t mg_post<T>(cudaStream_t, const Grid&, const Grid&, const T*, const T*,      \
                                  const T*, const T*, const T*, T*, const int32_t*, double*,       \
                                  int64_t, Prof, const T*);                                        \
  template cudaError_t qoi<T>(cudaStream_t, const Grid&, int, int, int, double, const T*, double*, \
                              int64_t, Prof);                                                      \
  template cudaError_t mg_bottom<T>(cudaStream_t, const BottomLevels<T>&, const T*, T*,            \
                                    const int32_t*, int64_t, Prof);

MLMC_INST2(double)
MLMC_INST2(float)

}  // namespace d2
}  // namespace mlmc
