// C ABI of libmlmc: plan, workspace, batched coupled solves, estimator.
//
// Host orchestration only: every numerical step runs in the kernels of
// xi.cu, field.cu, stencil2d.cu and reduce.cu. The plan owns the KLE
// eigenpairs (solved on the host once, a scalar root-finding), the per-mesh
// eigenfunction tables, the level states and one workspace buffer that is
// carved per batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <vector>

#include "mlmc_internal.cuh"

namespace mlmc {

Grid make_grid(int dim, int n, int z_chunk, int stencil_tile) {
  Grid g{};
  g.dim = dim;
  g.zt = stencil_tile;
  g.n = n;
  g.ns = round_up(ipow(n + 1, dim), 32);
  g.es = round_up(ipow(n, dim), 32);
  g.h = 1.0 / n;
  g.c3 = g.h / 3.0;
  g.c12 = g.h / 12.0;
  if (dim == 2) {
    const int strips = (n + 1 + 29) / 30;
    g.sx = (strips + SWARPS - 1) / SWARPS;
    g.sy = (n + 1 + SROWS - 1) / SROWS;
    g.tiles_s = (int64_t)g.sx * g.sy * SWARPS;
  } else {
    // stencil kernels: one CTA per 32 x 16 column tile and chunk of zc planes
    // (sx: the 32 x 8 node tiles of all planes, kept for the tile counts)
    g.sx = ((n + 1 + 31) / 32) * ((n + 1 + 7) / 8) * (n + 1);
    g.sy = 1;
    g.zc = (n + 1 <= 24) ? n + 1 : 16;
    if (z_chunk > 0) g.zc = std::min(z_chunk, n + 1);
    g.zx = ((n + 31) / 32) * ((n + 15) / 16) * ((n + 1 + g.zc - 1) / g.zc);
    g.tiles_s = g.zx;
  }
  g.fx = (int)((g.ns + FLAT_ELEMS - 1) / FLAT_ELEMS);
  g.tiles_f = g.fx;
  // the 2D QoI kernel is flat, the 3D one runs one CTA per z-plane
  g.tiles_q = dim == 2 ? g.tiles_f : (int64_t)(n + 1);
  return g;
}

namespace {

const char* kKernelNames[NUM_KERNELS] = {
    "draw_xi", "kle_table", "kappa", "coarsen_kappa", "apply", "pcg_init", "pcg_pq", "pcg_xr",
    "jacobi_z", "mg_pre", "restrict", "coarse_solve", "mg_post", "qoi", "finalize", "welford",
    "estimate", "count_active", "setup", "refine", "resid64", "mg_bottom"};

// Bump allocator over the workspace (base == nullptr: size only).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base((char*)b) {}
  template <class T>
  T* take(int64_t count) {
    off = (size_t)round_up((int64_t)off, 256);
    T* p = base ? (T*)(base + off) : nullptr;
    off += sizeof(T) * (size_t)std::max<int64_t>(count, 0);
    return p;
  }
};

constexpr int MAX_MG = 16;

struct MeshInfo {
  int n;
  int K;                 // multigrid levels (1 = no multigrid)
  Grid g[MAX_MG];
  double* table;         // n x m KLE table on the device
};

// Views of the workspace for one batched PCG solve on one mesh, value type T.
template <class T>
struct SolveWs {
  T *x, *r, *p0, *p1, *q, *z;
  T* kap[MAX_MG];
  T* coef[MAX_MG];   // FP64 2D: precomputed operator coefficients per level (else null)
  T* w[MAX_MG];
  T *e[MAX_MG], *r1[MAX_MG], *bk[MAX_MG], *eo[MAX_MG];
  double* part;
  Scalars sc;
  int32_t* count;
  int32_t* it;       // device iteration counter (graph-driven loop)
  int32_t* execs;    // device count of loop-body executions (graph-driven loop)
};

template <class T>
void carve_solve(Carve& c, const MeshInfo& mi, int64_t B, bool own_kappa0, SolveWs<T>& w) {
  // the FP64 stencils run on precomputed operator data where a stencil
  // kernel runs: 2D coefficients (3 node + 1 element arrays per level), 3D
  // kappa sums (4 node arrays per level)
  const bool coef = sizeof(T) == 8;
  const bool d2c = mi.g[0].dim == 2;
  const Grid& g0 = mi.g[0];
  w.x = c.take<T>(B * g0.ns);
  w.r = c.take<T>(B * g0.ns);
  w.p0 = c.take<T>(B * g0.ns);
  w.p1 = c.take<T>(B * g0.ns);
  w.q = c.take<T>(B * g0.ns);
  w.z = c.take<T>(B * g0.ns);
  for (int k = 0; k < mi.K; ++k) {
    const Grid& g = mi.g[k];
    w.kap[k] = (k == 0 && !own_kappa0) ? nullptr : c.take<T>(B * g.es);
    w.coef[k] = (coef && (k == 0 || k < mi.K - 1)) ? c.take<T>(B * (d2c ? 3 * g.ns + g.es : 4 * g.ns)) : nullptr;
    w.w[k] = c.take<T>(B * g.ns);
    if (mi.K > 1) {
      w.e[k] = c.take<T>(B * g.ns);
      w.r1[k] = (k < mi.K - 1) ? c.take<T>(B * g.ns) : nullptr;
      w.bk[k] = (k == 0) ? w.r : c.take<T>(B * g.ns);
      w.eo[k] = (k == 0) ? w.z : ((k < mi.K - 1) ? c.take<T>(B * g.ns) : w.e[k]);
    }
  }
  w.part = c.take<double>(B * g0.tiles());
  w.sc.gamma = c.take<double>(B);
  w.sc.delta = c.take<double>(B);
  w.sc.alpha = c.take<double>(B);
  w.sc.beta = c.take<double>(B);
  w.sc.rho = c.take<double>(B);
  w.sc.tol = c.take<double>(B);
  w.sc.active = c.take<int32_t>(B);
  w.sc.iters = c.take<int32_t>(B);
  w.sc.scale = nullptr;
  w.sc.total = nullptr;
  w.count = c.take<int32_t>(1);
  w.it = c.take<int32_t>(1);
  w.execs = c.take<int32_t>(1);
}

// Mixed form: FP64 solution / residual / kappa plus the FP32 inner solve.
struct MixedWs {
  double* u;
  double* r;
  double* kap64;
  double* coef64;   // operator data of the outer FP64 residual: 2D coefficients, 3D kappa sums
  const double* xi_tc;  // KLE coefficients: the FP32 kappa from the tensor cores (else the cast)
  Scalars outer;
  int32_t* outer_count;
  int32_t* outer_it;
  int32_t* outer_execs;
  SolveWs<float> in;
};

void carve_mixed(Carve& c, const MeshInfo& mi, int64_t B, MixedWs& w) {
  const Grid& g0 = mi.g[0];
  w.u = c.take<double>(B * g0.ns);
  w.r = c.take<double>(B * g0.ns);
  w.kap64 = c.take<double>(B * g0.es);
  w.coef64 = g0.dim == 2 ? c.take<double>(B * (3 * g0.ns + g0.es)) : c.take<double>(B * 4 * g0.ns);
  w.xi_tc = nullptr;
  w.outer.gamma = w.outer.delta = w.outer.alpha = w.outer.beta = nullptr;
  w.outer.rho = c.take<double>(B);
  w.outer.tol = c.take<double>(B);
  w.outer.scale = c.take<double>(B);
  w.outer.active = c.take<int32_t>(B);
  w.outer.iters = c.take<int32_t>(B);
  w.outer.total = c.take<int32_t>(B);
  // the outer scalars' gamma..beta are written by the scalar-init kernel: give them storage
  w.outer.gamma = c.take<double>(B);
  w.outer.delta = c.take<double>(B);
  w.outer.alpha = c.take<double>(B);
  w.outer.beta = c.take<double>(B);
  w.outer_count = c.take<int32_t>(1);
  w.outer_it = c.take<int32_t>(1);
  w.outer_execs = c.take<int32_t>(1);
  carve_solve(c, mi, B, true, w.in);
}

// Workspace of one coupled batch: xi, outputs, the coarse solution that
// seeds the fine solve (nested initial guess; guess_ns doubles per sample,
// 0 when unused) and the solve views of the finer mesh (the coarse solve
// reuses them).
struct CoupledWs {
  double* xi;
  double* qf;
  double* qc;
  int32_t* itf;
  int32_t* itc;
  double* uc;           // coarse-mesh solution (nested guess) or null
  double* kap;          // FP64 kappa of the mesh being solved
  SolveWs<double> s;    // FP64 form
  MixedWs mx;           // mixed form
};

// side: 0 for the solve on mesh `level`, 1 for mesh `level - 1`. The two
// solves share the region after the prefix; their loop-execution counters,
// which are read after both have run, live in the prefix.
void carve_coupled(Carve& c, const MeshInfo& mi, int M, int64_t B, bool mixed, int64_t guess_ns,
                   int side, CoupledWs& w) {
  w.xi = c.take<double>(B * M);
  w.qf = c.take<double>(B);
  w.qc = c.take<double>(B);
  w.itf = c.take<int32_t>(B);
  w.itc = c.take<int32_t>(B);
  int32_t* execs = c.take<int32_t>(4);
  w.uc = guess_ns > 0 ? c.take<double>(B * guess_ns) : nullptr;
  if (mixed) {
    carve_mixed(c, mi, B, w.mx);
    w.kap = w.mx.kap64;
    w.mx.xi_tc = w.xi;   // used when the plan takes its FP32 kappa from the tensor cores
    w.mx.outer_execs = execs ? execs + 2 * side : nullptr;
    w.mx.in.execs = execs ? execs + 2 * side + 1 : nullptr;
  } else {
    carve_solve(c, mi, B, true, w.s);
    w.kap = w.s.kap[0];
    w.s.execs = execs ? execs + 2 * side : nullptr;
  }
}

// Nested initial guess of a fine-mesh solve: the coarse-mesh solution of
// the same sample (uc, on grid gc), or none (uc == nullptr: x0 = 0).
struct Guess {
  const double* uc = nullptr;
  Grid gc{};
};

struct PendingEvent {
  int kid;
  cudaEvent_t a, b;
};

}  // namespace
}  // namespace mlmc

// An instantiated solve graph and the kernel counts of its parts (for the
// launch counter: setup + body * executions + epilogue).
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  int64_t n_static = 0;   // kernels outside every loop
  // per loop: device count of loop-control calls and kernels per call
  std::vector<std::pair<int32_t*, int64_t>> loops;
};

// A loop body to be captured after the graph that contains its while-node.
struct Deferred {
  cudaGraph_t body;
  std::function<mlmc_status()> fill;
  int32_t* execs;   // incremented by the loop control kernel(s) of the body
  int halves;       // loop-control calls per body execution
};

namespace mlmc {
namespace {

}  // namespace
}  // namespace mlmc

using namespace mlmc;

struct mlmc_plan_s {
  mlmc_config cfg;
  cudaStream_t stream = nullptr;
  int M = 0;                      // KLE coefficients per sample
  int32_t* d_slot = nullptr;      // total-order truncation: full-basis index of each coefficient
  double sqrt_sigma2 = 1.0;
  std::vector<MeshInfo> meshes;
  double* d_omega = nullptr;
  double* d_theta = nullptr;
  int32_t* d_even = nullptr;
  mlmc_level_state* d_states = nullptr;
  double* d_cost = nullptr;
  double* d_small = nullptr;      // scratch for estimate / allocate (64 doubles)
  int64_t* d_N = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  size_t ws_budget = 0;
  bool ws_borrowed = false;       // ws belongs to the caller (mlmc_plan_set_workspace)
  double* d_fold = nullptr;       // staging of mlmc_level_fold
  int64_t fold_cap = 0;
  void* h_pin = nullptr;
  size_t h_pin_bytes = 0;
  // tracing
  bool prof_on = false;
  uint32_t prof_mask = 0;
  double* d_prof = nullptr;       // NUM_KERNELS byte accumulators
  std::vector<PendingEvent> pending;
  std::vector<cudaEvent_t> pool;
  double ms[NUM_KERNELS] = {0};
  int64_t kl[NUM_KERNELS] = {0};
  int64_t launches = 0;
  bool tc_used = false;           // the tensor-core KLE kernel has run on this plan
  bool zw_used = false;   // mlmc_apply32 ran the 3D FP32 z-march (bounded waits to check)
  // graph-captured solves, keyed by (form, mesh, batch, workspace) and the
  // arrays they bake in (kappa, solution, QoI, iteration counts, guess)
  std::map<std::tuple<int, int, int64_t, const void*, const void*, const void*, const void*,
                      const void*, const void*>,
           struct GraphRec> graphs;
  // whole allocation rounds (one branch per level), keyed by form, batch
  // counts and first sample indices
  std::map<std::vector<int64_t>, struct GraphRec> round_graphs;
  std::vector<struct Deferred>* todo = nullptr;      // set while a graph is built
  std::vector<cudaStream_t> branch;                  // capture streams of round branches
  std::vector<cudaEvent_t> branch_ev;
  cudaEvent_t round_done = nullptr;                  // recorded after a launched round
  std::vector<int64_t> round_count;                  // samples per level (non-empty: a round in flight)
  struct Chunk {
    int level;
    size_t off;          // workspace region
    int64_t first, count;
  };
  std::vector<Chunk> round_chunks;                   // batched solves of the round in flight
  std::vector<size_t> done_off;                      // the last finished round, while its
  std::vector<int64_t> done_count;                   // per-sample values are still in place
  // a round over several plans driven by this one (cross-request batching):
  // its workspace, the coefficients carved per sample and, per member plan
  // and level, the samples it holds
  char* round_ws = nullptr;
  int round_M = 0;
  std::vector<mlmc_plan> group;
  std::vector<int64_t> group_count;                  // members x levels
  GraphRec group_graph;
  cudaStream_t cap_stream = nullptr;   // private stream the solve graphs are captured on
  // executed graphs whose kernel counts are settled at the next sync point
  std::vector<const GraphRec*> pending_graphs;
};

namespace {

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return MLMC_ERR_CUDA;  \
  } while (0)

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Number of KLE coefficients: m^dim, or the modes with k_x + k_y (+ k_z) <= K.
int64_t coef_count(const mlmc_config* c) {
  const int m = c->modes_per_dim;
  if (c->total_order < 0) return ipow(m, c->dim);
  int64_t M = 0;
  for (int kz = 0; kz < (c->dim == 3 ? m : 1); ++kz)
    for (int ky = 0; ky < m; ++ky)
      for (int kx = 0; kx < m; ++kx)
        if (kx + ky + kz <= c->total_order) ++M;
  return M;
}

// Full-basis flat index (k_z m + k_y) m + k_x of each kept coefficient.
std::vector<int32_t> coef_slots(const mlmc_config* c) {
  std::vector<int32_t> slot;
  const int m = c->modes_per_dim;
  for (int kz = 0; kz < (c->dim == 3 ? m : 1); ++kz)
    for (int ky = 0; ky < m; ++ky)
      for (int kx = 0; kx < m; ++kx)
        if (c->total_order < 0 || kx + ky + kz <= c->total_order)
          slot.push_back((int32_t)((kz * m + ky) * m + kx));
  return slot;
}

mlmc_status validate(const mlmc_config* c) {
  if (c && (c->total_order < -1 || c->z_chunk < 0 || (c->nested_guess != 0 && c->nested_guess != 1) ||
            (c->kle_tensor != 0 && c->kle_tensor != 1) || (c->stencil_tile < 0 || c->stencil_tile > 2) ||
            c->batch_split < 0 || c->batch_split > 64))
    return MLMC_ERR_INVALID;
  if (!c) return MLMC_ERR_INVALID;
  if (c->dim != 2 && c->dim != 3) return MLMC_ERR_INVALID;
  if (c->n_levels < 1 || c->n_levels > 16) return MLMC_ERR_INVALID;
  if (c->coarse_cells < 2) return MLMC_ERR_INVALID;
  if (c->modes_per_dim < 1 || c->modes_per_dim > (c->dim == 2 ? 32 : 16)) return MLMC_ERR_INVALID;
  if (!(c->sigma2 > 0.0) || !(c->corr_len > 0.0)) return MLMC_ERR_INVALID;
  if (!(c->rtol > 0.0) || c->max_iter < 1) return MLMC_ERR_INVALID;
  if (c->qoi != MLMC_QOI_DOMAIN_MEAN && c->qoi != MLMC_QOI_BOX_MEAN) return MLMC_ERR_INVALID;
  if (c->solver != MLMC_JACOBI_PCG && c->solver != MLMC_GMG_PCG) return MLMC_ERR_INVALID;
  const int64_t nf = (int64_t)c->coarse_cells << (c->n_levels - 1);
  if (nf > (c->dim == 2 ? 16384 : 1024)) return MLMC_ERR_INVALID;
  if (c->solver == MLMC_GMG_PCG) {
    if (!is_pow2(c->coarse_cells)) return MLMC_ERR_INVALID;
    if (!(c->mg_omega > 0.0 && c->mg_omega < 2.0) || c->mg_smooth != 1) return MLMC_ERR_INVALID;
    if (c->mg_coarsest != 2) return MLMC_ERR_INVALID;
  }
  if (c->qoi == MLMC_QOI_BOX_MEAN) {
    const double lo = c->box_lo * c->coarse_cells, hi = c->box_hi * c->coarse_cells;
    if (!(c->box_lo >= 0.0 && c->box_hi <= 1.0 && c->box_lo < c->box_hi)) return MLMC_ERR_INVALID;
    if (std::fabs(lo - std::round(lo)) > 1e-9 || std::fabs(hi - std::round(hi)) > 1e-9)
      return MLMC_ERR_INVALID;
  }
  if (c->precision != MLMC_FP64 && c->precision != MLMC_MIXED) return MLMC_ERR_INVALID;
  if (c->precision == MLMC_MIXED &&
      (!(c->inner_rtol > 0.0 && c->inner_rtol < 1.0) || c->inner_max_iter < 1 || c->outer_max_iter < 1))
    return MLMC_ERR_INVALID;
  return MLMC_OK;
}

// Roots of the 1D exponential-covariance KLE (Ghanem & Spanos closed form):
// with c = 1/corr_len on [0, 1] (half-width 1/2), mode k has its root in
// (k pi, (k+1) pi): even k solves c cos(w/2) - w sin(w/2) = 0, odd k solves
// w cos(w/2) + c sin(w/2) = 0; theta_k = 2c / (w^2 + c^2).
void kle_roots(double corr_len, int m, std::vector<double>& omega, std::vector<double>& theta,
               std::vector<int32_t>& even) {
  const double c = 1.0 / corr_len;
  const double pi = 3.14159265358979323846;
  omega.resize(m);
  theta.resize(m);
  even.resize(m);
  for (int k = 0; k < m; ++k) {
    const bool ev = (k % 2 == 0);
    auto f = [&](double w) {
      return ev ? c * std::cos(0.5 * w) - w * std::sin(0.5 * w)
                : w * std::cos(0.5 * w) + c * std::sin(0.5 * w);
    };
    double lo = k * pi, hi = (k + 1) * pi;
    double flo = f(lo);
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      const double fm = f(mid);
      if ((fm < 0) == (flo < 0)) {
        lo = mid;
        flo = fm;
      } else {
        hi = mid;
      }
    }
    omega[k] = 0.5 * (lo + hi);
    theta[k] = 2.0 * c / (omega[k] * omega[k] + c * c);
    even[k] = ev ? 1 : 0;
  }
}

int64_t interior_dofs(int dim, int64_t n) { return ipow(n - 1, dim); }

double level_cost_cfg(const mlmc_config* c, int level) {
  const int64_t n = (int64_t)c->coarse_cells << level;
  double cost = (double)interior_dofs(c->dim, n);
  if (level > 0) cost += (double)interior_dofs(c->dim, n / 2);
  return cost;
}

// --- tracing helpers --------------------------------------------------

void harvest(mlmc_plan p) {
  if (p->pending.empty()) return;
  cudaStreamSynchronize(p->stream);
  for (auto& e : p->pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) p->ms[e.kid] += t;
    p->kl[e.kid] += 1;
    p->pool.push_back(e.a);
    p->pool.push_back(e.b);
  }
  p->pending.clear();
}

cudaEvent_t get_event(mlmc_plan p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

Prof prof_for(mlmc_plan p, int kid, double per_sample) {
  Prof pr;
  pr.acc = (p->prof_on && (p->prof_mask >> kid & 1u)) ? p->d_prof + kid : nullptr;
  pr.per_sample = per_sample;
  return pr;
}

// Launch `f` as kernel `kid`, bracketed by events when tracing is on.
template <class F>
cudaError_t run(mlmc_plan p, int kid, F&& f) {
  p->launches += 1;
  if (!p->prof_on || !(p->prof_mask >> kid & 1u)) return f();
  PendingEvent pe;
  pe.kid = kid;
  pe.a = get_event(p);
  pe.b = get_event(p);
  cudaEventRecord(pe.a, p->stream);
  cudaError_t e = f();
  cudaEventRecord(pe.b, p->stream);
  p->pending.push_back(pe);
  if (p->pending.size() > 8192) harvest(p);
  return e;
}

double nodes_of(const Grid& g) { return (double)ipow(g.n + 1, g.dim); }
double elems_of(const Grid& g) { return (double)ipow(g.n, g.dim); }

// --- workspace --------------------------------------------------------

// Workspaces of destroyed plans (and the smaller block a growing plan gives
// up) are kept for the next plan on the same device instead of going back
// to the driver: freeing a multi-GB block unmaps its pages (milliseconds per
// plan) and the next plan would map them again. At most kWsCacheBlocks
// blocks are kept (the oldest is freed first); an allocation that fails
// frees this device's cached blocks and tries once more;
// mlmc_release_cached_memory() frees them all.
struct WsBlock {
  int dev;
  void* ptr;
  size_t bytes;
};
constexpr size_t kWsCacheBlocks = 4;
std::mutex g_ws_mu;
std::vector<WsBlock> g_ws_cache;   // oldest first

// A block of at least `bytes` on the current device: the smallest cached one
// that fits, else a new allocation. Sets *got to its size.
cudaError_t ws_acquire(size_t bytes, void** out, size_t* got) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    int best = -1;
    for (int k = 0; k < (int)g_ws_cache.size(); ++k) {
      const WsBlock& w = g_ws_cache[k];
      if (w.dev == dev && w.bytes >= bytes && (best < 0 || w.bytes < g_ws_cache[best].bytes)) best = k;
    }
    if (best >= 0) {
      *out = g_ws_cache[best].ptr;
      *got = g_ws_cache[best].bytes;
      g_ws_cache.erase(g_ws_cache.begin() + best);
      return cudaSuccess;
    }
  }
  e = cudaMalloc(out, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    std::vector<void*> mine;
    {
      std::lock_guard<std::mutex> lk(g_ws_mu);
      for (auto it = g_ws_cache.begin(); it != g_ws_cache.end();) {
        if (it->dev == dev) {
          mine.push_back(it->ptr);
          it = g_ws_cache.erase(it);
        } else {
          ++it;
        }
      }
    }
    if (mine.empty()) return e;
    for (void* q : mine) cudaFree(q);
    e = cudaMalloc(out, bytes);
  }
  if (e == cudaSuccess) *got = bytes;
  return e;
}

// Hands a block back to the cache (the caller has synchronised its uses).
void ws_release(void* ptr, size_t bytes) {
  if (!ptr) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaFree(ptr);
    return;
  }
  void* evict = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    g_ws_cache.push_back({dev, ptr, bytes});
    if (g_ws_cache.size() > kWsCacheBlocks) {
      evict = g_ws_cache.front().ptr;
      g_ws_cache.erase(g_ws_cache.begin());
    }
  }
  if (evict) cudaFree(evict);
}

void clear_graphs(mlmc_plan p);
mlmc_status settle_graph_launches(mlmc_plan p);

mlmc_status ensure_ws(mlmc_plan p, size_t bytes) {
  p->done_count.clear();   // the workspace is about to be reused
  if (bytes <= p->ws_bytes) return MLMC_OK;
  if (p->ws_borrowed) return MLMC_ERR_OOM;   // a borrowed workspace never grows
  if (p->ws) {
    cudaStreamSynchronize(p->stream);
    if (settle_graph_launches(p) != MLMC_OK) return MLMC_ERR_CUDA;
    clear_graphs(p);
    ws_release(p->ws, p->ws_bytes);
    p->ws = nullptr;
    p->ws_bytes = 0;
  }
  size_t got = 0;
  if (ws_acquire(bytes, &p->ws, &got) != cudaSuccess) {
    cudaGetLastError();
    p->ws = nullptr;
    return MLMC_ERR_OOM;
  }
  p->ws_bytes = got;
  return MLMC_OK;
}

mlmc_status ensure_pin(mlmc_plan p, size_t bytes) {
  if (bytes <= p->h_pin_bytes) return MLMC_OK;
  if (p->h_pin) {
    cudaStreamSynchronize(p->stream);
    cudaFreeHost(p->h_pin);
    p->h_pin = nullptr;
  }
  const size_t b = std::max<size_t>(bytes, 1 << 16);
  if (cudaMallocHost(&p->h_pin, b) != cudaSuccess) {
    cudaGetLastError();
    p->h_pin_bytes = 0;
    return MLMC_ERR_OOM;
  }
  p->h_pin_bytes = b;
  return MLMC_OK;
}

bool is_mixed(mlmc_plan p) { return p->cfg.precision == MLMC_MIXED; }

// Grids of mesh `l` of a configuration (no tables): enough to size workspaces.
void mesh_info_shape(const mlmc_config& c, int l, MeshInfo& mi) {
  mi.n = c.coarse_cells << l;
  mi.K = 1;
  mi.table = nullptr;
  mi.g[0] = make_grid(c.dim, mi.n, c.z_chunk, c.stencil_tile);
  if (c.solver == MLMC_GMG_PCG && mi.n > 2) {
    int n = mi.n;
    while (n > 2 && mi.K < MAX_MG) {
      n /= 2;
      mi.g[mi.K++] = make_grid(c.dim, n, c.z_chunk, c.stencil_tile);
    }
  }
}

size_t coupled_bytes(const MeshInfo& mi, int M, int64_t B, bool mixed, int64_t guess_ns) {
  Carve c(nullptr);
  CoupledWs w;
  carve_coupled(c, mi, M, B, mixed, guess_ns, 0, w);
  return c.off + 256;
}

// Node stride of mesh level - 1 when its solution seeds the solve on mesh
// `level` (nested initial guess), else 0.
int64_t guess_ns_of(const mlmc_config& c, int level) {
  if (!c.nested_guess || level <= 0) return 0;
  return make_grid(c.dim, c.coarse_cells << (level - 1), c.z_chunk).ns;
}

size_t solve_bytes(const MeshInfo& mi, int64_t B, bool mixed) {
  Carve c(nullptr);
  if (mixed) {
    MixedWs w;
    carve_mixed(c, mi, B, w);
  } else {
    SolveWs<double> w;
    carve_solve(c, mi, B, false, w);
  }
  return c.off + 256;
}

template <class SizeFn>
int64_t max_batch(mlmc_plan p, SizeFn size_of, int64_t want) {
  int64_t B = std::min<int64_t>(want, 65535);
  if (B <= 0) return 0;
  const size_t one = size_of(1);
  const size_t per = std::max<size_t>(size_of(2) - one, 1);
  if (size_of(B) > p->ws_budget) {
    B = (int64_t)((p->ws_budget > one ? p->ws_budget - one : 0) / per) + 1;
    while (B > 1 && size_of(B) > p->ws_budget) --B;
  }
  return std::max<int64_t>(B, 1);
}

// --- the batched PCG --------------------------------------------------

// z = M r (GMG V-cycle or Jacobi), with per-tile partials of r.z in w.part.
template <class T>
mlmc_status precondition(mlmc_plan p, const MeshInfo& mi, SolveWs<T>& w, int64_t B,
                         int64_t* tiles) {
  cudaStream_t s = p->stream;
  const Grid& g0 = mi.g[0];
  const double vb = (double)sizeof(T);
  const double nn0 = nodes_of(g0);
  if (mi.K == 1) {
    CK(run(p, KID_JACOBI_Z, [&] {
      return op::jacobi_z<T>(s, g0, w.w[0], w.r, w.z, w.sc, w.part, B,
                             prof_for(p, KID_JACOBI_Z, 3 * nn0 * vb));
    }));
    *tiles = g0.tiles_f;
    return MLMC_OK;
  }
  const int K = mi.K;
  // the levels below the finest whose grids have at most BOTTOM_MAX_N2 (2D)
  // or BOTTOM_MAX_N3 (3D) cells per side run as one fused kernel
  // (k0 .. K-1), one CTA per sample
  const int nmax = g0.dim == 2 ? BOTTOM_MAX_N2 : BOTTOM_MAX_N3;
  int k0 = K - 1;
  while (k0 - 1 >= 1 && mi.g[k0 - 1].n <= nmax) --k0;
  const bool fuse = k0 < K - 1 && K - k0 <= MAX_BOTTOM;
  const int kd = fuse ? k0 : K - 1;   // levels above the bottom
  for (int k = 0; k < kd; ++k) {
    const Grid& g = mi.g[k];
    const double nn = nodes_of(g), ne = elems_of(g);
    CK(run(p, KID_MG_PRE, [&] {
      return op::mg_pre<T>(s, g, w.kap[k], w.w[k], w.bk[k], w.e[k], w.r1[k], w.sc.active, B,
                           prof_for(p, KID_MG_PRE, (4 * nn + ne) * vb), w.coef[k]);
    }));
    CK(run(p, KID_RESTRICT, [&] {
      return op::restrict_<T>(s, g, mi.g[k + 1], w.r1[k], w.bk[k + 1], w.sc.active, B,
                              prof_for(p, KID_RESTRICT, (nn + nodes_of(mi.g[k + 1])) * vb));
    }));
  }
  if (fuse) {
    BottomLevels<T> lv{};
    lv.L = K - k0;
    double bytes = 2 * nodes_of(mi.g[k0]);
    for (int l = 0; l < lv.L; ++l) {
      lv.g[l] = mi.g[k0 + l];
      lv.kap[l] = w.kap[k0 + l];
      lv.coef[l] = w.coef[k0 + l];
      lv.w[l] = w.w[k0 + l];
      bytes += nodes_of(mi.g[k0 + l]) + elems_of(mi.g[k0 + l]);
    }
    CK(run(p, KID_MG_BOTTOM, [&] {
      return op::mg_bottom<T>(s, lv, w.bk[k0], w.eo[k0], w.sc.active, B,
                              prof_for(p, KID_MG_BOTTOM, bytes * vb));
    }));
  } else {
    CK(run(p, KID_COARSE, [&] {
      return op::coarse_solve<T>(s, mi.g[K - 1], w.kap[K - 1], w.bk[K - 1], w.e[K - 1], w.sc.active, B);
    }));
  }
  for (int k = kd - 1; k >= 0; --k) {
    const Grid& g = mi.g[k];
    const double nn = nodes_of(g), ne = elems_of(g), nc = nodes_of(mi.g[k + 1]);
    CK(run(p, KID_MG_POST, [&] {
      // r1[k] is dead once restricted: it serves as the 3D scratch for e + P e_c
      return op::mg_post<T>(s, g, mi.g[k + 1], w.kap[k], w.w[k], w.bk[k], w.e[k], w.eo[k + 1],
                            w.eo[k], w.r1[k], w.sc.active, k == 0 ? w.part : nullptr, B,
                            prof_for(p, KID_MG_POST, (4 * nn + ne + nc) * vb), w.coef[k]);
    }));
  }
  *tiles = g0.tiles_s;
  return MLMC_OK;
}

// Multigrid kappa hierarchy and W = omega / D per level (w.kap[0] given).
template <class T>
mlmc_status setup_levels(mlmc_plan p, const MeshInfo& mi, SolveWs<T>& w, int64_t B) {
  cudaStream_t s = p->stream;
  const int K = mi.K;
  const double vb = (double)sizeof(T);
  for (int k = 1; k < K; ++k) {
    CK(run(p, KID_COARSEN, [&] {
      return launch_coarsen<T>(s, mi.g[k - 1], mi.g[k], w.kap[k - 1], w.kap[k], B,
                               prof_for(p, KID_COARSEN, (elems_of(mi.g[k - 1]) + elems_of(mi.g[k])) * vb));
    }));
  }
  const double omega = (K > 1) ? p->cfg.mg_omega : 1.0;
  const int kw = std::max(1, K - 1);   // levels that smooth (W = omega / D)
  // 2D levels with operator coefficients get W from the same kernel; 3D
  // levels get their kappa sums (FP64) and W separately
  const bool d2c = mi.g[0].dim == 2;
  for (int k = 0; k < K; ++k)
    if (w.coef[k])
      CK(run(p, KID_SETUP, [&] {
        if (d2c) return d2::coef<T>(s, mi.g[k], w.kap[k], w.coef[k], B, omega, k < kw ? w.w[k] : nullptr);
        if constexpr (std::is_same<T, double>::value) return d3::ksum(s, mi.g[k], w.kap[k], w.coef[k], B);
        return cudaErrorInvalidValue;
      }));
  for (int k = 0; k < kw; ++k)
    if (!d2c || !w.coef[k])
      CK(run(p, KID_SETUP, [&] { return op::winv<T>(s, mi.g[k], w.kap[k], omega, w.w[k], B); }));
  return MLMC_OK;
}

// First preconditioning and gamma = r.z; sets the device iteration counter to 1.
template <class T>
mlmc_status pcg_prologue(mlmc_plan p, const MeshInfo& mi, SolveWs<T>& w, int64_t B, int max_iter) {
  int64_t Tp = 0;
  mlmc_status st = precondition<T>(p, mi, w, B, &Tp);
  if (st != MLMC_OK) return st;
  CK(run(p, KID_FINALIZE, [&] { return launch_finalize(p->stream, FIN_GAMMA0, w.part, Tp, w.sc, nullptr, 0, max_iter, B); }));
  CK(run(p, KID_SETUP, [&] { return launch_set_int(p->stream, w.it, 1); }));
  return MLMC_OK;
}

// One PCG iteration with p_old -> p_new; with a graph handle, the loop
// control kernel advances the device counter and sets the while-condition.
template <class T>
mlmc_status pcg_iteration(mlmc_plan p, const MeshInfo& mi, SolveWs<T>& w, int64_t B, int max_iter,
                          int it, T* pold, T* pnew, const cudaGraphConditionalHandle* h,
                          bool* done) {
  cudaStream_t s = p->stream;
  const Grid& g0 = mi.g[0];
  const double vb = (double)sizeof(T);
  const double nn0 = nodes_of(g0), ne0 = elems_of(g0);
  const int32_t* itd = h ? w.it : nullptr;
  CK(run(p, KID_PCG_PQ, [&] {
    return op::pcg_pq<T>(s, g0, w.kap[0], w.z, pold, pnew, w.q, w.sc, w.part, B,
                         prof_for(p, KID_PCG_PQ, (4 * nn0 + ne0) * vb), w.coef[0]);
  }));
  CK(run(p, KID_FINALIZE, [&] { return launch_finalize(s, FIN_ALPHA, w.part, g0.tiles_s, w.sc, nullptr, it, max_iter, B, itd); }));
  CK(run(p, KID_PCG_XR, [&] {
    return op::pcg_xr<T>(s, g0, w.x, pnew, w.r, w.q, w.sc, w.part, B,
                         prof_for(p, KID_PCG_XR, 6 * nn0 * vb));
  }));
  CK(run(p, KID_FINALIZE, [&] { return launch_finalize(s, FIN_CONV, w.part, g0.tiles_f, w.sc, nullptr, it, max_iter, B, itd); }));
  if (h) {
    CK(run(p, KID_COUNT, [&] { return launch_loop_ctl(s, w.sc.active, B, w.it, max_iter, w.count, w.execs, *h); }));
  } else {
    int check = p->cfg.check_every;
    if (check <= 0) check = (B * nn0 > 4e6) ? 1 : 4;
    if (it % check == 0 || it == max_iter) {
      int32_t* h_count = (int32_t*)p->h_pin;
      CK(run(p, KID_COUNT, [&] { return launch_count_active(s, w.sc.active, B, w.count); }));
      CK(cudaMemcpyAsync(h_count, w.count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*h_count == 0) {
        *done = true;
        return MLMC_OK;
      }
    }
  }
  int64_t Tp = 0;
  mlmc_status st = precondition<T>(p, mi, w, B, &Tp);
  if (st != MLMC_OK) return st;
  CK(run(p, KID_FINALIZE, [&] { return launch_finalize(s, FIN_BETA, w.part, Tp, w.sc, nullptr, it, max_iter, B, itd); }));
  return MLMC_OK;
}

// Host-driven PCG iterations (scalars, x and r initialised; prologue done).
template <class T>
mlmc_status pcg_loop(mlmc_plan p, const MeshInfo& mi, SolveWs<T>& w, int64_t B, int max_iter) {
  if (ensure_pin(p, 64) != MLMC_OK) return MLMC_ERR_OOM;
  T* pold = w.p0;
  T* pnew = w.p1;
  for (int it = 1; it <= max_iter; ++it) {
    bool done = false;
    mlmc_status st = pcg_iteration<T>(p, mi, w, B, max_iter, it, pold, pnew, nullptr, &done);
    if (st != MLMC_OK) return st;
    if (done) break;
    std::swap(pold, pnew);
  }
  return MLMC_OK;
}

// Body of the graph-driven loop: two iterations (p0 -> p1, p1 -> p0), each
// followed by the loop control; iterations after convergence are no-ops
// because every kernel skips inactive samples.
template <class T>
mlmc_status pcg_graph_body(mlmc_plan p, const MeshInfo& mi, SolveWs<T>& w, int64_t B, int max_iter,
                           cudaGraphConditionalHandle h) {
  bool done = false;
  mlmc_status st = pcg_iteration<T>(p, mi, w, B, max_iter, 0, w.p0, w.p1, &h, &done);
  if (st != MLMC_OK) return st;
  return pcg_iteration<T>(p, mi, w, B, max_iter, 0, w.p1, w.p0, &h, &done);
}

// --- CUDA-graph capture -----------------------------------------------
//
// A solve is captured on the plan's private stream into one graph. Loops are
// while-nodes inserted into the graph being captured; every kernel that sets
// a loop condition is a direct node of the body of that loop, or an upstream
// node of the same graph (to re-arm a nested loop).

// Launches issued while capturing go to the plan's private capture stream.
struct CaptureStream {
  mlmc_plan p;
  cudaStream_t saved;
  explicit CaptureStream(mlmc_plan pp) : p(pp), saved(pp->stream) { p->stream = p->cap_stream; }
  ~CaptureStream() { p->stream = saved; }
};

// Runs f while capturing into `graph` (new graph if *graph == nullptr).
template <class F>
mlmc_status capture(mlmc_plan p, cudaGraph_t* graph, F&& f, int64_t* nk = nullptr) {
  CaptureStream cs(p);
  const int64_t l0 = p->launches;
  cudaError_t e = (*graph == nullptr)
                      ? cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal)
                      : cudaStreamBeginCaptureToGraph(p->stream, *graph, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return MLMC_ERR_CUDA;
  mlmc_status st = f();
  cudaGraph_t g = *graph;
  e = cudaStreamEndCapture(p->stream, &g);
  if (nk) *nk = p->launches - l0;
  p->launches = l0;   // captured launches are counted when the graph executes
  if (st != MLMC_OK || e != cudaSuccess) {
    if (g && *graph == nullptr) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != MLMC_OK ? st : MLMC_ERR_CUDA;
  }
  *graph = g;
  return MLMC_OK;
}

// Graph being captured on p->stream.
mlmc_status capture_graph(mlmc_plan p, cudaGraph_t* g) {
  cudaStreamCaptureStatus cs;
  if (cudaStreamGetCaptureInfo(p->stream, &cs, nullptr, g, nullptr, nullptr, nullptr) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return MLMC_ERR_CUDA;
  return MLMC_OK;
}

// Inserts a while-node after everything captured so far on p->stream; later
// launches depend on it. Creates its handle (default 1 at graph launch)
// unless have_handle. *body receives the (empty) body graph.
mlmc_status insert_while(mlmc_plan p, cudaGraphConditionalHandle* h, cudaGraph_t* body,
                         bool have_handle) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(p->stream, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return MLMC_ERR_CUDA;
  if (!have_handle && cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return MLMC_ERR_CUDA;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, ed, nd, &np) != cudaSuccess) return MLMC_ERR_CUDA;
  if (cudaStreamUpdateCaptureDependencies(p->stream, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies) != cudaSuccess)
    return MLMC_ERR_CUDA;
  *body = np.conditional.phGraph_out[0];
  return MLMC_OK;
}

void clear_graphs(mlmc_plan p) {
  for (auto& kv : p->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  for (auto& kv : p->round_graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  p->graphs.clear();
  p->round_graphs.clear();
  p->pending_graphs.clear();
}

// Inserts a while-node (see insert_while) whose body is captured later by
// build_graph through body_fn(handle). With `given`, that handle is used.
template <class F>
mlmc_status issue_loop(mlmc_plan p, int32_t* execs, int halves, F body_fn,
                       const cudaGraphConditionalHandle* given = nullptr) {
  cudaGraphConditionalHandle h;
  if (given) h = *given;
  cudaGraph_t body = nullptr;
  mlmc_status st = insert_while(p, &h, &body, given != nullptr);
  if (st != MLMC_OK) return st;
  if (!p->todo) return MLMC_ERR_CUDA;
  p->todo->push_back(Deferred{body, [h, body_fn]() mutable { return body_fn(h); }, execs, halves});
  return MLMC_OK;
}

// Captures issue() into a new graph, then every loop body it (recursively)
// deferred, and instantiates it.
mlmc_status build_graph(mlmc_plan p, const std::function<mlmc_status()>& issue, GraphRec* out) {
  std::vector<Deferred> todo;
  p->todo = &todo;
  GraphRec rec;
  cudaGraph_t P = nullptr;
  mlmc_status st = capture(p, &P, issue, &rec.n_static);
  for (size_t i = 0; st == MLMC_OK && i < todo.size(); ++i) {
    Deferred d = todo[i];
    int64_t nk = 0;
    st = capture(p, &d.body, d.fill, &nk);
    rec.loops.emplace_back(d.execs, nk / d.halves);
  }
  p->todo = nullptr;
  if (st != MLMC_OK) {
    if (P) cudaGraphDestroy(P);
    return st;
  }
  if (cudaGraphInstantiate(&rec.exec, P, 0) != cudaSuccess) {
    cudaGraphDestroy(P);
    cudaGetLastError();
    return MLMC_ERR_CUDA;
  }
  cudaGraphDestroy(P);
  *out = rec;
  return MLMC_OK;
}

// Adds the kernels executed by graphs launched since the last sync point;
// for 3D mixed-form plans also checks that no bounded wait of the FP32
// z-march gave up (MLMC_ERR_TIMEOUT).
mlmc_status settle_graph_launches(mlmc_plan p) {
  if (p->cfg.dim == 3 && (p->cfg.precision == MLMC_MIXED || p->zw_used)) {
    unsigned timeouts = 0;
    CK(d3::take_wait_timeouts(p->stream, &timeouts));
    if (timeouts) return MLMC_ERR_TIMEOUT;
  }
  if (p->tc_used) {
    unsigned timeouts = 0;
    CK(take_tc_timeouts(p->stream, &timeouts));
    if (timeouts) return MLMC_ERR_TIMEOUT;
  }
  for (const GraphRec* r : p->pending_graphs) {
    p->launches += r->n_static;
    for (const auto& lp : r->loops) {
      int32_t ex = 0;
      CK(cudaMemcpy(&ex, lp.first, sizeof(int32_t), cudaMemcpyDeviceToHost));
      p->launches += (int64_t)ex * lp.second;
    }
  }
  p->pending_graphs.clear();
  return MLMC_OK;
}

bool graphs_on(mlmc_plan p) { return p->cfg.use_graphs != 0 && !p->prof_on && p->cap_stream; }

double b_norm(const mlmc_config& c, const Grid& g0) {
  return std::pow(g0.h, c.dim) * std::sqrt((double)interior_dofs(c.dim, g0.n));
}

// QoI of the FP64 solution u into q_dev (Sec. 2.1; exact Q1 integral mean).
mlmc_status qoi_of(mlmc_plan p, const Grid& g0, const double* u, double* part, const Scalars& sc,
                   double* q_dev, int64_t B) {
  const mlmc_config& c = p->cfg;
  const int64_t nf = g0.n;
  const int L = (int)std::lround(c.box_lo * nf), H = (int)std::lround(c.box_hi * nf);
  const double vol = std::pow(c.box_hi - c.box_lo, c.dim);
  const int box = (c.qoi == MLMC_QOI_BOX_MEAN) ? 1 : 0;
  CK(run(p, KID_QOI, [&] {
    return op::qoi<double>(p->stream, g0, box, L, H, box ? 1.0 / vol : 1.0, u, part, B,
                           prof_for(p, KID_QOI, nodes_of(g0) * 8));
  }));
  const int64_t tq = g0.tiles_q;
  CK(run(p, KID_FINALIZE, [&] { return launch_finalize(p->stream, FIN_QOI, part, tq, sc, q_dev, 0, c.max_iter, B); }));
  return MLMC_OK;
}

// u = P uc (the coarse solution interpolated to the fine mesh) and its FP64
// residual r = b - A u, with per-tile partials of r.r in part.
mlmc_status init_from_guess(mlmc_plan p, const Grid& g0, const Guess& gs, const double* kappa,
                            const double* coef, double* u, double* r, const int32_t* active,
                            double* part, int64_t B) {
  const double nn0 = nodes_of(g0), ne0 = elems_of(g0);
  CK(run(p, KID_PCG_INIT, [&] {
    return op::prolong_guess(p->stream, g0, gs.gc, gs.uc, u, active, B,
                             prof_for(p, KID_PCG_INIT, (nn0 + nodes_of(gs.gc)) * 8));
  }));
  CK(run(p, KID_RESID64, [&] {
    return op::resid64(p->stream, g0, kappa, u, r, active, part, B,
                       prof_for(p, KID_RESID64, (2 * nn0 + ne0) * 8), coef);
  }));
  return MLMC_OK;
}

// FP64 form, launch sequences.
mlmc_status fp64_setup(mlmc_plan p, const MeshInfo& mi, SolveWs<double>& w, int64_t B, const Guess& gs) {
  cudaStream_t s = p->stream;
  const mlmc_config& c = p->cfg;
  const Grid& g0 = mi.g[0];
  mlmc_status st = setup_levels<double>(p, mi, w, B);
  if (st != MLMC_OK) return st;
  CK(run(p, KID_SETUP, [&] { return launch_scalars_init(s, w.sc, c.rtol * b_norm(c, g0), 0.0, B); }));
  CK(run(p, KID_SETUP, [&] { return launch_set_int(s, w.execs, 0); }));
  if (gs.uc) {
    st = init_from_guess(p, g0, gs, w.kap[0], w.coef[0], w.x, w.r, w.sc.active, w.part, B);
    if (st != MLMC_OK) return st;
  } else {
    CK(run(p, KID_PCG_INIT, [&] {
      return op::pcg_init<double>(s, g0, w.x, w.r, B, prof_for(p, KID_PCG_INIT, 2 * nodes_of(g0) * 8));
    }));
  }
  return pcg_prologue<double>(p, mi, w, B, c.max_iter);
}

mlmc_status fp64_epilogue(mlmc_plan p, const MeshInfo& mi, SolveWs<double>& w, int64_t B,
                          double* q_dev, int32_t* iters_dev) {
  mlmc_status st = qoi_of(p, mi.g[0], w.x, w.part, w.sc, q_dev, B);
  if (st != MLMC_OK) return st;
  if (iters_dev) CK(cudaMemcpyAsync(iters_dev, w.sc.iters, sizeof(int32_t) * B, cudaMemcpyDeviceToDevice, p->stream));
  return MLMC_OK;
}

// FP64 solve issued into the graph being captured: setup -> while(two PCG
// iterations + loop control) -> QoI epilogue.
mlmc_status issue_fp64(mlmc_plan p, const MeshInfo& mi, SolveWs<double>& w, int64_t B,
                       double* q_dev, int32_t* iters_dev, const Guess& gs) {
  mlmc_status st = fp64_setup(p, mi, w, B, gs);
  if (st != MLMC_OK) return st;
  const MeshInfo* mip = &mi;
  SolveWs<double> wc = w;   // copied into the deferred body (mutable lambda)
  const int maxit = p->cfg.max_iter;
  st = issue_loop(p, w.execs, 2, [p, mip, wc, B, maxit](cudaGraphConditionalHandle h) mutable {
    return pcg_graph_body<double>(p, *mip, wc, B, maxit, h);
  });
  if (st != MLMC_OK) return st;
  return fp64_epilogue(p, mi, w, B, q_dev, iters_dev);
}

// FP64 form: solve A(kappa) u = b for B samples; w.kap[0] holds kappa.
// Leaves u in w.x, writes q (device) and iters (device). With graphs on,
// the whole solve is one graph: setup -> while(two PCG iterations) -> QoI.
mlmc_status solve_fp64(mlmc_plan p, int mesh, const MeshInfo& mi, SolveWs<double>& w, int64_t B,
                       double* q_dev, int32_t* iters_dev, const Guess& gs) {
  const mlmc_config& c = p->cfg;
  if (!graphs_on(p)) {
    mlmc_status st = fp64_setup(p, mi, w, B, gs);
    if (st != MLMC_OK) return st;
    st = pcg_loop<double>(p, mi, w, B, c.max_iter);
    if (st != MLMC_OK) return st;
    return fp64_epilogue(p, mi, w, B, q_dev, iters_dev);
  }
  const auto key = std::make_tuple(0, mesh, B, (const void*)p->ws, (const void*)w.kap[0],
                                   (const void*)w.x, (const void*)q_dev, (const void*)iters_dev,
                                   (const void*)gs.uc);
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    GraphRec rec;
    mlmc_status st = build_graph(p, [&] { return issue_fp64(p, mi, w, B, q_dev, iters_dev, gs); }, &rec);
    if (st != MLMC_OK) return st;
    it = p->graphs.emplace(key, rec).first;
  }
  CK(cudaGraphLaunch(it->second.exec, p->stream));
  p->pending_graphs.push_back(&it->second);
  return MLMC_OK;
}

// Mixed form, launch sequences.
mlmc_status mixed_setup(mlmc_plan p, const MeshInfo& mi, MixedWs& w, int64_t B, const Guess& gs) {
  cudaStream_t s = p->stream;
  const mlmc_config& c = p->cfg;
  const Grid& g0 = mi.g[0];
  if (w.xi_tc && c.kle_tensor) {
    CK(run(p, KID_KAPPA, [&] {
      return launch_kappa32_tc(s, g0, c.modes_per_dim, p->sqrt_sigma2, mi.table, w.xi_tc, p->M, p->d_slot, B,
                               w.in.kap[0]);
    }));
  } else {
    CK(run(p, KID_SETUP, [&] { return launch_cast_kappa(s, g0, w.kap64, w.in.kap[0], B); }));
  }
  if (w.coef64)
    CK(run(p, KID_SETUP, [&] {
      return g0.dim == 2 ? d2::coef<double>(s, g0, w.kap64, w.coef64, B) : d3::ksum(s, g0, w.kap64, w.coef64, B);
    }));
  mlmc_status st = setup_levels<float>(p, mi, w.in, B);
  if (st != MLMC_OK) return st;
  const double bn = b_norm(c, g0);
  CK(run(p, KID_SETUP, [&] { return launch_scalars_init(s, w.outer, c.rtol * bn, bn, B); }));
  CK(run(p, KID_SETUP, [&] { return launch_set_int(s, w.outer_it, 1); }));
  CK(run(p, KID_SETUP, [&] { return launch_set_int(s, w.outer_execs, 0); }));
  CK(run(p, KID_SETUP, [&] { return launch_set_int(s, w.in.execs, 0); }));
  if (gs.uc) {
    st = init_from_guess(p, g0, gs, w.kap64, w.coef64, w.u, w.r, w.outer.active, w.in.part, B);
    if (st != MLMC_OK) return st;
    // ||r0|| becomes the scale of the first inner right-hand side
    CK(run(p, KID_FINALIZE, [&] {
      return launch_outer_step(s, w.in.part, g0.tiles_s, w.outer, nullptr, c.inner_max_iter, 0,
                               c.outer_max_iter, B, nullptr);
    }));
  } else {
    CK(run(p, KID_PCG_INIT, [&] {
      return op::pcg_init<double>(s, g0, w.u, w.r, B, prof_for(p, KID_PCG_INIT, 2 * nodes_of(g0) * 8));
    }));
  }
  return MLMC_OK;
}

// Before each inner solve: unit-norm FP32 right-hand side, inner scalars, d = 0, prologue.
mlmc_status mixed_pre_inner(mlmc_plan p, const MeshInfo& mi, MixedWs& w, int64_t B) {
  cudaStream_t s = p->stream;
  const mlmc_config& c = p->cfg;
  const Grid& g0 = mi.g[0];
  const double nn0 = nodes_of(g0);
  CK(run(p, KID_REFINE, [&] {
    return op::to_rhs32(s, g0, w.r, w.outer.scale, w.in.r, w.outer.active, B,
                        prof_for(p, KID_REFINE, nn0 * (8 + 4)));
  }));
  CK(run(p, KID_SETUP, [&] { return launch_inner_init(s, w.in.sc, w.outer, c.inner_rtol, B); }));
  CK(run(p, KID_PCG_INIT, [&] {
    return op::pcg_init<float>(s, g0, w.in.x, nullptr, B, prof_for(p, KID_PCG_INIT, nn0 * 4));
  }));
  return pcg_prologue<float>(p, mi, w.in, B, c.inner_max_iter);
}

// After each inner solve: u += s d, FP64 residual, outer convergence test.
mlmc_status mixed_post_inner(mlmc_plan p, const MeshInfo& mi, MixedWs& w, int64_t B, int outer,
                             const int32_t* outer_it_dev) {
  cudaStream_t s = p->stream;
  const mlmc_config& c = p->cfg;
  const Grid& g0 = mi.g[0];
  const double nn0 = nodes_of(g0), ne0 = elems_of(g0);
  CK(run(p, KID_REFINE, [&] {
    return op::add_correction(s, g0, w.u, w.in.x, w.outer.scale, w.outer.active, B,
                              prof_for(p, KID_REFINE, nn0 * (8 + 4 + 8)));
  }));
  CK(run(p, KID_RESID64, [&] {
    return op::resid64(s, g0, w.kap64, w.u, w.r, w.outer.active, w.in.part, B,
                       prof_for(p, KID_RESID64, (2 * nn0 + ne0) * 8), w.coef64);
  }));
  CK(run(p, KID_FINALIZE, [&] {
    return launch_outer_step(s, w.in.part, g0.tiles_s, w.outer, w.in.sc.iters, c.inner_max_iter,
                             outer, c.outer_max_iter, B, outer_it_dev);
  }));
  return MLMC_OK;
}

mlmc_status mixed_epilogue(mlmc_plan p, const MeshInfo& mi, MixedWs& w, int64_t B, double* q_dev,
                           int32_t* iters_dev) {
  mlmc_status st = qoi_of(p, mi.g[0], w.u, w.in.part, w.outer, q_dev, B);
  if (st != MLMC_OK) return st;
  if (iters_dev) CK(cudaMemcpyAsync(iters_dev, w.outer.iters, sizeof(int32_t) * B, cudaMemcpyDeviceToDevice, p->stream));
  return MLMC_OK;
}

// Mixed solve issued into the graph being captured: setup ->
// while_outer(pre, re-arm inner, while_inner(PCG), post, outer control) -> QoI.
mlmc_status issue_mixed(mlmc_plan p, const MeshInfo& mi, MixedWs& w, int64_t B, double* q_dev,
                        int32_t* iters_dev, const Guess& gs) {
  mlmc_status st = mixed_setup(p, mi, w, B, gs);
  if (st != MLMC_OK) return st;
  const MeshInfo* mip = &mi;
  MixedWs wc = w;           // copied into the deferred bodies (mutable lambdas)
  const int imax = p->cfg.inner_max_iter, omax = p->cfg.outer_max_iter;
  st = issue_loop(p, w.outer_execs, 1, [p, mip, wc, B, imax, omax](cudaGraphConditionalHandle ho) mutable {
    mlmc_status s2 = mixed_pre_inner(p, *mip, wc, B);
    if (s2 != MLMC_OK) return s2;
    // the inner loop's condition is re-armed before every inner while-node
    cudaGraph_t g = nullptr;
    if ((s2 = capture_graph(p, &g)) != MLMC_OK) return s2;
    cudaGraphConditionalHandle hi;
    if (cudaGraphConditionalHandleCreate(&hi, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
      return MLMC_ERR_CUDA;
    CK(run(p, KID_SETUP, [&] { return launch_set_cond(p->stream, hi, 1u); }));
    s2 = issue_loop(p, wc.in.execs, 2, [p, mip, wc, B, imax](cudaGraphConditionalHandle h) mutable {
      return pcg_graph_body<float>(p, *mip, wc.in, B, imax, h);
    }, &hi);
    if (s2 != MLMC_OK) return s2;
    if ((s2 = mixed_post_inner(p, *mip, wc, B, 0, wc.outer_it)) != MLMC_OK) return s2;
    CK(run(p, KID_COUNT, [&] {
      return launch_loop_ctl(p->stream, wc.outer.active, B, wc.outer_it, omax, wc.outer_count,
                             wc.outer_execs, ho);
    }));
    return MLMC_OK;
  });
  if (st != MLMC_OK) return st;
  return mixed_epilogue(p, mi, w, B, q_dev, iters_dev);
}

// Mixed form: FP64 iterative refinement around FP32 GMG/Jacobi-PCG
// (kappa32 = rounded kappa64). w.kap64 holds kappa. Leaves u in w.u. With
// graphs on the whole solve is one graph (issue_mixed).
mlmc_status solve_mixed(mlmc_plan p, int mesh, const MeshInfo& mi, MixedWs& w, int64_t B,
                        double* q_dev, int32_t* iters_dev, const Guess& gs) {
  cudaStream_t s = p->stream;
  const mlmc_config& c = p->cfg;
  if (!graphs_on(p)) {
    mlmc_status st = mixed_setup(p, mi, w, B, gs);
    if (st != MLMC_OK) return st;
    if (ensure_pin(p, 64) != MLMC_OK) return MLMC_ERR_OOM;
    int32_t* h_count = (int32_t*)p->h_pin;
    for (int outer = 1; outer <= c.outer_max_iter; ++outer) {
      if ((st = mixed_pre_inner(p, mi, w, B)) != MLMC_OK) return st;
      if ((st = pcg_loop<float>(p, mi, w.in, B, c.inner_max_iter)) != MLMC_OK) return st;
      if ((st = mixed_post_inner(p, mi, w, B, outer, nullptr)) != MLMC_OK) return st;
      CK(run(p, KID_COUNT, [&] { return launch_count_active(s, w.outer.active, B, w.outer_count); }));
      CK(cudaMemcpyAsync(h_count, w.outer_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*h_count == 0) break;
    }
    return mixed_epilogue(p, mi, w, B, q_dev, iters_dev);
  }
  const auto key = std::make_tuple(1, mesh, B, (const void*)p->ws, (const void*)w.kap64,
                                   (const void*)w.u, (const void*)q_dev, (const void*)iters_dev,
                                   (const void*)gs.uc);
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    GraphRec rec;
    mlmc_status st = build_graph(p, [&] { return issue_mixed(p, mi, w, B, q_dev, iters_dev, gs); }, &rec);
    if (st != MLMC_OK) return st;
    it = p->graphs.emplace(key, rec).first;
  }
  CK(cudaGraphLaunch(it->second.exec, p->stream));
  p->pending_graphs.push_back(&it->second);
  return MLMC_OK;
}

mlmc_status make_kappa(mlmc_plan p, int mesh, const double* xi, int64_t B, double* kappa) {
  const MeshInfo& mi = p->meshes[mesh];
  CK(run(p, KID_KAPPA, [&] {
    return launch_kappa(p->stream, mi.g[0], p->cfg.modes_per_dim, p->sqrt_sigma2, mi.table, xi, p->M,
                        p->d_slot, B, kappa, prof_for(p, KID_KAPPA, elems_of(mi.g[0]) * 8));
  }));
  return MLMC_OK;
}

// --- one allocation round as one graph ----------------------------------

// Nested guess wiring of one side of a coupled batch: the coarse solve
// (side 1) writes its solution into w.uc, the fine solve (side 0) starts
// from it. No-op when the batch has no guess buffer.
Guess guess_views(mlmc_plan p, int level, int side, bool mixed, CoupledWs& w) {
  Guess gs;
  if (!w.uc) return gs;
  if (side == 1) {
    if (mixed) w.mx.u = w.uc;
    else w.s.x = w.uc;
  } else {
    gs.uc = w.uc;
    gs.gc = p->meshes[level - 1].g[0];
  }
  return gs;
}

// Coupled batch of `level` issued into the graph being captured on p->stream,
// in the workspace region at `region`: xi, kappa and solve on mesh `level`,
// kappa and solve on mesh `level - 1`, Welford fold in sample order.
mlmc_status fold_batch(mlmc_plan p, int level, int64_t B, void* region);

mlmc_status issue_level(mlmc_plan p, int level, int64_t first, int64_t B, void* region, bool fold = true) {
  const bool mixed = is_mixed(p);
  const int M = p->M;
  const int64_t gns = guess_ns_of(p->cfg, level);
  const int sides = level > 0 ? 2 : 1;
  mlmc_status st;
  for (int k = 0; k < sides; ++k) {
    // side 0: mesh `level`, side 1: mesh `level - 1`; with the nested guess
    // the coarse mesh goes first and its solution seeds the fine solve
    const int side = gns > 0 ? sides - 1 - k : k;
    const int mesh = level - side;
    const MeshInfo& mi = p->meshes[mesh];
    Carve c(region);
    CoupledWs w;
    carve_coupled(c, mi, M, B, mixed, gns, side, w);
    if (k == 0 && (st = mlmc_draw_xi(p, level, first, B, w.xi)) != MLMC_OK) return st;
    if ((st = make_kappa(p, mesh, w.xi, B, w.kap)) != MLMC_OK) return st;
    double* qd = side == 0 ? w.qf : w.qc;
    int32_t* itd = side == 0 ? w.itf : w.itc;
    const Guess gs = guess_views(p, level, side, mixed, w);
    st = mixed ? issue_mixed(p, mi, w.mx, B, qd, itd, gs) : issue_fp64(p, mi, w.s, B, qd, itd, gs);
    if (st != MLMC_OK) return st;
  }
  return fold ? fold_batch(p, level, B, region) : MLMC_OK;
}

// Y = Q_f - Q_c of the coupled batch in `region` folded into the level state in sample order.
mlmc_status fold_batch(mlmc_plan p, int level, int64_t B, void* region) {
  Carve c(region);
  CoupledWs w;
  carve_coupled(c, p->meshes[level], p->M, B, is_mixed(p), guess_ns_of(p->cfg, level), 0, w);
  const double cost = level_cost_cfg(&p->cfg, level);
  CK(run(p, KID_WELFORD, [&] {
    return launch_welford(p->stream, w.qf, level > 0 ? w.qc : nullptr, B, p->d_states + level, cost);
  }));
  return MLMC_OK;
}

// Capture streams and events for `branches` parallel branches of a round.
mlmc_status ensure_branches(mlmc_plan p, size_t branches, size_t events) {
  while (p->branch.size() < branches) {
    cudaStream_t bs;
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return MLMC_ERR_CUDA;
    p->branch.push_back(bs);
  }
  while (p->branch_ev.size() < events) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return MLMC_ERR_CUDA;
    p->branch_ev.push_back(ev);
  }
  return MLMC_OK;
}

// Batched solves of a round: per level, the samples in batch_split
// near-equal chunks (one chunk when it is 0 or 1), each with its own
// workspace region.
size_t round_chunks_of(const mlmc_config& c, const MeshInfo* meshes, int M, const std::vector<int64_t>& first,
                       const std::vector<int64_t>& count, std::vector<mlmc_plan_s::Chunk>* out) {
  const bool mixed = c.precision == MLMC_MIXED;
  size_t total = 0;
  for (int l = 0; l < c.n_levels; ++l) {
    if (count[l] <= 0) continue;
    const int64_t k = std::max<int64_t>(1, std::min<int64_t>(c.batch_split, count[l]));
    const int64_t w = (count[l] + k - 1) / k;
    for (int64_t s0 = 0; s0 < count[l]; s0 += w) {
      const int64_t cnt = std::min<int64_t>(w, count[l] - s0);
      if (out) out->push_back({l, total, first[l] + s0, cnt});
      total += (size_t)round_up((int64_t)coupled_bytes(meshes[l], M, cnt, mixed, guess_ns_of(c, l)), 256);
    }
  }
  return total;
}

// Samples first[l] .. first[l] + count[l] - 1 of every level in one graph
// with one branch per level (finest first), so the latency-bound coarse
// levels run beside the fine ones. Returns MLMC_ERR_UNIMPLEMENTED when the
// batches do not fit the workspace together (the caller then samples level
// by level). *bad is set when a solve hit its iteration cap.
mlmc_status round_launch(mlmc_plan p, const std::vector<int64_t>& first,
                         const std::vector<int64_t>& count) {
  const int L1 = p->cfg.n_levels;
  const bool mixed = is_mixed(p);
  for (int l = 0; l < L1; ++l)
    if (count[l] > 65535) return MLMC_ERR_UNIMPLEMENTED;
  std::vector<mlmc_plan_s::Chunk> chunks;
  const size_t total = round_chunks_of(p->cfg, p->meshes.data(), p->M, first, count, &chunks);
  p->round_count = count;
  p->round_chunks = chunks;
  p->round_M = p->M;
  if (total == 0) return MLMC_OK;
  if (total > p->ws_budget) return MLMC_ERR_UNIMPLEMENTED;
  // branches: one per chunk; events: the fork, one per chunk, one per level
  mlmc_status st = ensure_branches(p, chunks.size(), 1 + chunks.size() + L1);
  if (st != MLMC_OK) return st;
  st = ensure_ws(p, total);
  if (st != MLMC_OK) return st;
  p->round_ws = (char*)p->ws;
  std::vector<int64_t> key = {mixed ? 1 : 0, (int64_t)(uintptr_t)p->ws, p->cfg.batch_split};
  key.insert(key.end(), first.begin(), first.end());
  key.insert(key.end(), count.begin(), count.end());
  auto it = p->round_graphs.find(key);
  if (it == p->round_graphs.end()) {
    GraphRec rec;
    st = build_graph(p, [&]() -> mlmc_status {
      cudaStream_t origin = p->stream;
      const size_t nc = chunks.size();
      cudaEvent_t fork = p->branch_ev[0];
      CK(cudaEventRecord(fork, origin));
      // chunks finest level first, each on its own branch
      std::vector<size_t> order(nc);
      for (size_t i = 0; i < nc; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(),
                       [&](size_t a, size_t b) { return chunks[a].level > chunks[b].level; });
      mlmc_status s2 = MLMC_OK;
      for (size_t i = 0; i < nc && s2 == MLMC_OK; ++i) {
        const auto& ch = chunks[order[i]];
        cudaStream_t S = p->branch[order[i]];
        CK(cudaStreamWaitEvent(S, fork, 0));
        p->stream = S;
        s2 = issue_level(p, ch.level, ch.first, ch.count, (char*)p->ws + ch.off, false);
        p->stream = origin;
        if (s2 == MLMC_OK) CK(cudaEventRecord(p->branch_ev[1 + order[i]], S));
      }
      // each level's chunks are folded in sample order on the branch of its first chunk
      for (int l = 0; l < L1 && s2 == MLMC_OK; ++l) {
        int head = -1;
        for (size_t i = 0; i < nc && s2 == MLMC_OK; ++i) {
          if (chunks[i].level != l) continue;
          if (head < 0) head = (int)i;
          cudaStream_t S = p->branch[head];
          if ((int)i != head) CK(cudaStreamWaitEvent(S, p->branch_ev[1 + i], 0));
          p->stream = S;
          s2 = fold_batch(p, l, chunks[i].count, (char*)p->ws + chunks[i].off);
          p->stream = origin;
        }
        if (head >= 0 && s2 == MLMC_OK) {
          CK(cudaEventRecord(p->branch_ev[1 + nc + l], p->branch[head]));
          CK(cudaStreamWaitEvent(origin, p->branch_ev[1 + nc + l], 0));
        }
      }
      return s2;
    }, &rec);
    if (st != MLMC_OK) return st;
    it = p->round_graphs.emplace(key, rec).first;
  }
  CK(cudaGraphLaunch(it->second.exec, p->stream));
  CK(cudaEventRecord(p->round_done, p->stream));
  p->pending_graphs.push_back(&it->second);
  return MLMC_OK;
}

// ---- rounds over several plans (cross-request batching) -----------------

// Plans whose coupled batches can share one solve: the same meshes, solver,
// precision, tolerances, multigrid and QoI settings (their fields, KLE modes,
// seeds and stream ids may differ).
bool same_solve(const mlmc_config& a, const mlmc_config& b) {
  return a.dim == b.dim && a.n_levels == b.n_levels && a.coarse_cells == b.coarse_cells &&
         a.solver == b.solver && a.precision == b.precision && a.rtol == b.rtol &&
         a.max_iter == b.max_iter && a.mg_smooth == b.mg_smooth && a.mg_omega == b.mg_omega &&
         a.mg_coarsest == b.mg_coarsest && a.check_every == b.check_every &&
         a.inner_rtol == b.inner_rtol && a.inner_max_iter == b.inner_max_iter &&
         a.outer_max_iter == b.outer_max_iter && a.z_chunk == b.z_chunk &&
         a.nested_guess == b.nested_guess && a.qoi == b.qoi && a.box_lo == b.box_lo &&
         a.box_hi == b.box_hi && a.stencil_tile == b.stencil_tile && a.kle_tensor == 0 && b.kle_tensor == 0;
}

// The coupled batch of `level` over the members of p's group, issued into the
// graph being captured on p->stream: every member draws its xi (its own
// stream of sample indices first[k] ..) and forms kappa with its own KLE
// tables into its range of the batch; the solves on both meshes run once for
// the whole batch (p's solver settings, which the members share); each
// member's Y are folded into its own level state in sample order.
mlmc_status issue_level_group(mlmc_plan p, int level, const std::vector<int64_t>& first, int64_t B,
                              char* region) {
  const bool mixed = is_mixed(p);
  const int64_t gns = guess_ns_of(p->cfg, level);
  const int sides = level > 0 ? 2 : 1;
  const int L1 = p->cfg.n_levels;
  const int nm = (int)p->group.size();
  cudaStream_t S = p->stream;
  mlmc_status st;
  for (int k = 0; k < sides; ++k) {
    const int side = gns > 0 ? sides - 1 - k : k;
    const int mesh = level - side;
    const MeshInfo& mi = p->meshes[mesh];
    Carve c(region);
    CoupledWs w;
    carve_coupled(c, mi, p->round_M, B, mixed, gns, side, w);
    int64_t o = 0, xo = 0;
    for (int j = 0; j < nm; ++j) {
      mlmc_plan q = p->group[j];
      const int64_t cnt = p->group_count[(size_t)j * L1 + level];
      if (cnt <= 0) continue;
      cudaStream_t saved = q->stream;
      const int64_t l0 = q->launches;
      q->stream = S;   // the member's kernels join the graph being captured
      if (k == 0) st = mlmc_draw_xi(q, level, first[(size_t)j * L1 + level], cnt, w.xi + xo);
      else st = MLMC_OK;
      if (st == MLMC_OK) st = make_kappa(q, mesh, w.xi + xo, cnt, w.kap + o * mi.g[0].es);
      q->stream = saved;
      if (q != p) {   // counted with the driving plan's graph
        p->launches += q->launches - l0;
        q->launches = l0;
      }
      if (st != MLMC_OK) return st;
      o += cnt;
      xo += cnt * q->M;
    }
    if (mixed) w.mx.xi_tc = nullptr;   // members' coefficients differ in number: kappa32 by the cast
    double* qd = side == 0 ? w.qf : w.qc;
    int32_t* itd = side == 0 ? w.itf : w.itc;
    const Guess gs = guess_views(p, level, side, mixed, w);
    st = mixed ? issue_mixed(p, mi, w.mx, B, qd, itd, gs) : issue_fp64(p, mi, w.s, B, qd, itd, gs);
    if (st != MLMC_OK) return st;
  }
  Carve c(region);
  CoupledWs w;
  carve_coupled(c, p->meshes[level], p->round_M, B, mixed, gns, 0, w);
  const double cost = level_cost_cfg(&p->cfg, level);
  int64_t o = 0;
  for (int j = 0; j < nm; ++j) {
    mlmc_plan q = p->group[j];
    const int64_t cnt = p->group_count[(size_t)j * L1 + level];
    if (cnt <= 0) continue;
    CK(run(p, KID_WELFORD, [&] {
      return launch_welford(S, w.qf + o, level > 0 ? w.qc + o : nullptr, cnt, q->d_states + level, cost);
    }));
    o += cnt;
  }
  return MLMC_OK;
}

// One round over the plans of p's group in the caller's workspace `ws`: a
// graph with a branch per level (finest first), launched on p's stream.
mlmc_status group_launch(mlmc_plan p, const std::vector<int64_t>& first, char* ws, uint64_t ws_bytes) {
  const int L1 = p->cfg.n_levels;
  const bool mixed = is_mixed(p);
  const int nm = (int)p->group.size();
  std::vector<int64_t> B(L1, 0);
  std::vector<size_t> off(L1, 0);
  int Mmax = 1;
  for (int j = 0; j < nm; ++j) Mmax = std::max(Mmax, p->group[j]->M);
  size_t total = 0;
  for (int l = 0; l < L1; ++l) {
    for (int j = 0; j < nm; ++j) B[l] += p->group_count[(size_t)j * L1 + l];
    if (B[l] <= 0) continue;
    if (B[l] > 65535) return MLMC_ERR_UNIMPLEMENTED;
    off[l] = total;
    total += (size_t)round_up((int64_t)coupled_bytes(p->meshes[l], Mmax, B[l], mixed, guess_ns_of(p->cfg, l)),
                              256);
  }
  if (total > ws_bytes) return MLMC_ERR_OOM;
  p->round_count = B;
  p->round_chunks.clear();
  for (int l = 0; l < L1; ++l)
    if (B[l] > 0) p->round_chunks.push_back({l, off[l], 0, B[l]});
  p->round_ws = ws;
  p->round_M = Mmax;
  if (total == 0) return MLMC_OK;
  GraphRec rec;
  mlmc_status st = build_graph(p, [&]() -> mlmc_status {
    cudaStream_t origin = p->stream;
    CK(cudaEventRecord(p->branch_ev[0], origin));
    int nb = 0;
    mlmc_status s2 = MLMC_OK;
    for (int l = L1 - 1; l >= 0 && s2 == MLMC_OK; --l) {
      if (B[l] <= 0) continue;
      cudaStream_t S = p->branch[nb];
      CK(cudaStreamWaitEvent(S, p->branch_ev[0], 0));
      p->stream = S;
      s2 = issue_level_group(p, l, first, B[l], ws + off[l]);
      p->stream = origin;
      if (s2 == MLMC_OK) CK(cudaEventRecord(p->branch_ev[1 + nb], S));
      ++nb;
    }
    for (int i = 0; i < nb && s2 == MLMC_OK; ++i) CK(cudaStreamWaitEvent(origin, p->branch_ev[1 + i], 0));
    return s2;
  }, &rec);
  if (st != MLMC_OK) return st;
  p->group_graph = rec;
  CK(cudaGraphLaunch(rec.exec, p->stream));
  CK(cudaEventRecord(p->round_done, p->stream));
  p->pending_graphs.push_back(&p->group_graph);
  return MLMC_OK;
}

// Waits for the launched round, settles the launch count and checks the
// per-sample iteration counts of both meshes of every level. For a round over
// several plans, member_bad[k] (may be null) tells whether a solve of member
// k hit its iteration cap.
mlmc_status round_finish(mlmc_plan p, bool* bad, int32_t* member_bad = nullptr) {
  CK(cudaStreamSynchronize(p->stream));
  mlmc_status st = settle_graph_launches(p);
  if (st != MLMC_OK) return st;
  const int L1 = p->cfg.n_levels;
  const bool mixed = is_mixed(p);
  const int nm = (int)p->group.size();
  if (member_bad)
    for (int k = 0; k < nm; ++k) member_bad[k] = 0;
  std::vector<int32_t> h;
  bool one_per_level = true;
  std::vector<int> seen(L1, 0);
  for (const auto& ch : p->round_chunks) {
    const int l = ch.level;
    const int64_t n = ch.count;
    if (n <= 0) continue;
    if (seen[l]++) one_per_level = false;
    Carve c(p->round_ws + ch.off);
    CoupledWs w;
    carve_coupled(c, p->meshes[l], p->round_M, n, mixed, guess_ns_of(p->cfg, l), 0, w);
    h.resize(2 * n);
    // on the plan's stream: other plans' rounds keep running meanwhile
    CK(cudaMemcpyAsync(h.data(), w.itf, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(h.data() + n, w.itc, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    int k = 0;
    int64_t end = nm ? p->group_count[l] : n;   // samples of member k end at `end`
    for (int64_t b = 0; b < n; ++b) {
      while (nm && b >= end && k + 1 < nm) end += p->group_count[(size_t)(++k) * L1 + l];
      if (h[b] < 0 || (l > 0 && h[n + b] < 0)) {
        *bad = true;
        if (member_bad && nm) member_bad[k] = 1;
      }
    }
  }
  if (nm) {
    // the regions held every member's samples: no per-plan values to read back
    if (p->group_graph.exec) cudaGraphExecDestroy(p->group_graph.exec);
    p->group_graph = GraphRec{};
    p->group.clear();
    p->group_count.clear();
    p->done_count.clear();
  } else if (one_per_level) {
    p->done_off.assign(L1, 0);
    p->done_count.assign(L1, 0);
    for (const auto& ch : p->round_chunks) {
      p->done_off[ch.level] = ch.off;
      p->done_count[ch.level] = ch.count;
    }
  } else {
    p->done_count.clear();   // a level in several chunks: its values are not in one place
  }
  p->round_ws = (char*)p->ws;
  p->round_M = p->M;
  p->round_count.clear();
  p->round_chunks.clear();
  return MLMC_OK;
}

// Samples first[l] .. first[l] + count[l] - 1 of every level in one graph
// with one branch per level (finest first), so the latency-bound coarse
// levels run beside the fine ones. Returns MLMC_ERR_UNIMPLEMENTED when the
// batches do not fit the workspace together (the caller then samples level
// by level). *bad is set when a solve hit its iteration cap.
mlmc_status run_round(mlmc_plan p, const std::vector<int64_t>& first,
                      const std::vector<int64_t>& count, bool* bad) {
  mlmc_status st = round_launch(p, first, count);
  if (st != MLMC_OK) return st;
  return round_finish(p, bad);
}

// Draws the samples have[l] .. target[l] - 1 of every level and sets have
// to target: one graph per round with a branch per level when the batches
// fit the workspace together, otherwise level by level, finest first (the
// priority of the paper's incremental greedy schedule).
mlmc_status sample_phase(mlmc_plan p, std::vector<int64_t>& have, const std::vector<int64_t>& target,
                         bool* bad) {
  const int L1 = p->cfg.n_levels;
  std::vector<int64_t> count(L1);
  for (int l = 0; l < L1; ++l) count[l] = std::max<int64_t>(0, target[l] - have[l]);
  mlmc_status st = graphs_on(p) ? run_round(p, have, count, bad) : MLMC_ERR_UNIMPLEMENTED;
  if (st == MLMC_ERR_UNIMPLEMENTED) {
    for (int l = L1 - 1; l >= 0; --l) {
      if (count[l] > 0) {
        st = mlmc_sample_level(p, l, have[l], count[l], nullptr, nullptr, nullptr);
        if (st == MLMC_ERR_NOT_CONVERGED) *bad = true;
        else if (st != MLMC_OK) return st;
      }
    }
  } else if (st != MLMC_OK) {
    return st;
  }
  for (int l = 0; l < L1; ++l) have[l] = std::max(have[l], target[l]);
  return MLMC_OK;
}

}  // namespace

// ===================================================================
// C ABI
// ===================================================================

extern "C" {

void mlmc_config_default(mlmc_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->dim = 2;
  c->n_levels = 3;
  c->coarse_cells = 16;
  c->modes_per_dim = 4;
  c->sigma2 = 1.0;
  c->corr_len = 0.3;
  c->qoi = MLMC_QOI_DOMAIN_MEAN;
  c->solver = MLMC_JACOBI_PCG;
  c->box_lo = 0.25;
  c->box_hi = 0.75;
  c->rtol = 1e-10;
  c->max_iter = 20000;
  c->precision = MLMC_FP64;
  c->seed = 0;
  c->stream_id = 0;
  c->mg_smooth = 1;
  c->mg_omega = 0.9;
  c->mg_coarsest = 2;
  c->check_every = 0;
  c->workspace_bytes = 0;
  c->inner_rtol = 3e-3;
  c->inner_max_iter = 200;
  c->outer_max_iter = 40;
  c->use_graphs = 1;
  c->total_order = -1;
  c->z_chunk = 0;
  c->nested_guess = 1;
  c->kle_tensor = 0;
  c->stencil_tile = 0;
  c->batch_split = 0;
}

int64_t mlmc_node_stride(int dim, int n) {
  if ((dim != 2 && dim != 3) || n < 1) return -1;
  return make_grid(dim, n).ns;
}

int64_t mlmc_elem_stride(int dim, int n) {
  if ((dim != 2 && dim != 3) || n < 1) return -1;
  return make_grid(dim, n).es;
}

int64_t mlmc_mesh_cells(const mlmc_config* cfg, int mesh) {
  if (!cfg || mesh < 0 || mesh >= cfg->n_levels) return -1;
  return (int64_t)cfg->coarse_cells << mesh;
}

int64_t mlmc_coef_count(const mlmc_config* cfg) {
  if (validate(cfg) != MLMC_OK) return -1;
  return coef_count(cfg);
}

double mlmc_level_cost(const mlmc_config* cfg, int level) {
  if (!cfg || level < 0 || level >= cfg->n_levels) return -1.0;
  return level_cost_cfg(cfg, level);
}

const char* mlmc_status_str(mlmc_status s) {
  switch (s) {
    case MLMC_OK: return "ok";
    case MLMC_ERR_INVALID: return "invalid argument";
    case MLMC_ERR_OOM: return "out of device memory";
    case MLMC_ERR_NOT_CONVERGED: return "a solve hit max_iter";
    case MLMC_ERR_CUDA: return "CUDA error";
    case MLMC_ERR_TIMEOUT: return "device wait timed out";
    case MLMC_ERR_UNIMPLEMENTED: return "not implemented";
  }
  return "unknown status";
}

int mlmc_kernel_count(void) { return NUM_KERNELS; }

const char* mlmc_kernel_name(int kid) {
  if (kid < 0 || kid >= NUM_KERNELS) return nullptr;
  return kKernelNames[kid];
}

mlmc_status mlmc_plan_create(const mlmc_config* cfg, void* stream, mlmc_plan* out) {
  if (!out) return MLMC_ERR_INVALID;
  *out = nullptr;
  mlmc_status st = validate(cfg);
  if (st != MLMC_OK) return st;
  mlmc_plan p = new mlmc_plan_s();
  p->cfg = *cfg;
  p->stream = (cudaStream_t)stream;
  p->tc_used = cfg->kle_tensor && cfg->precision == MLMC_MIXED;
  const int m = cfg->modes_per_dim;
  p->M = (int)coef_count(cfg);
  p->sqrt_sigma2 = std::sqrt(cfg->sigma2);
  std::vector<double> omega, theta;
  std::vector<int32_t> even;
  kle_roots(cfg->corr_len, m, omega, theta, even);
  auto fail = [&](mlmc_status s) {
    mlmc_plan_destroy(p);
    return s;
  };
  if (cudaMalloc(&p->d_omega, sizeof(double) * m) != cudaSuccess ||
      cudaMalloc(&p->d_theta, sizeof(double) * m) != cudaSuccess ||
      cudaMalloc(&p->d_even, sizeof(int32_t) * m) != cudaSuccess ||
      cudaMalloc(&p->d_states, sizeof(mlmc_level_state) * cfg->n_levels) != cudaSuccess ||
      cudaMalloc(&p->d_cost, sizeof(double) * cfg->n_levels) != cudaSuccess ||
      cudaMalloc(&p->d_small, sizeof(double) * 64) != cudaSuccess ||
      cudaMalloc(&p->d_N, sizeof(int64_t) * 16) != cudaSuccess ||
      cudaMalloc(&p->d_prof, sizeof(double) * NUM_KERNELS) != cudaSuccess) {
    cudaGetLastError();
    return fail(MLMC_ERR_OOM);
  }
  if (cfg->total_order >= 0) {
    const std::vector<int32_t> slot = coef_slots(cfg);
    if (cudaMalloc(&p->d_slot, sizeof(int32_t) * slot.size()) != cudaSuccess) {
      p->d_slot = nullptr;
      cudaGetLastError();
      return fail(MLMC_ERR_OOM);
    }
    if (cudaMemcpy(p->d_slot, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(MLMC_ERR_CUDA);
  }
  std::vector<double> cost(cfg->n_levels);
  for (int l = 0; l < cfg->n_levels; ++l) cost[l] = level_cost_cfg(cfg, l);
  if (cudaMemcpyAsync(p->d_omega, omega.data(), sizeof(double) * m, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaMemcpyAsync(p->d_theta, theta.data(), sizeof(double) * m, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaMemcpyAsync(p->d_even, even.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaMemcpyAsync(p->d_cost, cost.data(), sizeof(double) * cfg->n_levels, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_states, 0, sizeof(mlmc_level_state) * cfg->n_levels, p->stream) != cudaSuccess ||
      cudaMemsetAsync(p->d_prof, 0, sizeof(double) * NUM_KERNELS, p->stream) != cudaSuccess)
    return fail(MLMC_ERR_CUDA);
  if (init_kle_exp() != cudaSuccess) return fail(MLMC_ERR_CUDA);
  p->meshes.resize(cfg->n_levels);
  for (int l = 0; l < cfg->n_levels; ++l) {
    MeshInfo& mi = p->meshes[l];
    mi.n = cfg->coarse_cells << l;
    mi.K = 1;
    mi.g[0] = make_grid(cfg->dim, mi.n, cfg->z_chunk, cfg->stencil_tile);
    if (cfg->solver == MLMC_GMG_PCG && mi.n > 2) {
      int n = mi.n;
      while (n > 2 && mi.K < MAX_MG) {
        n /= 2;
        mi.g[mi.K++] = make_grid(cfg->dim, n, cfg->z_chunk, cfg->stencil_tile);
      }
    }
    if (cudaMalloc(&mi.table, sizeof(double) * (size_t)mi.n * m) != cudaSuccess) {
      mi.table = nullptr;
      cudaGetLastError();
      return fail(MLMC_ERR_OOM);
    }
    if (run(p, KID_TABLE, [&] { return launch_kle_table(p->stream, mi.n, m, p->d_omega, p->d_theta, p->d_even, mi.table); }) != cudaSuccess)
      return fail(MLMC_ERR_CUDA);
  }
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    p->cap_stream = nullptr;
    return fail(MLMC_ERR_CUDA);
  }
  for (int l = 0; l < cfg->n_levels; ++l) {
    cudaStream_t bs;
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return fail(MLMC_ERR_CUDA);
    p->branch.push_back(bs);
  }
  for (int l = 0; l <= cfg->n_levels; ++l) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(MLMC_ERR_CUDA);
    p->branch_ev.push_back(ev);
  }
  if (cudaEventCreateWithFlags(&p->round_done, cudaEventDisableTiming) != cudaSuccess) {
    p->round_done = nullptr;
    return fail(MLMC_ERR_CUDA);
  }
  size_t budget = cfg->workspace_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(MLMC_ERR_CUDA);
    budget = std::min<size_t>((size_t)(0.4 * (double)fr), (size_t)48 << 30);
  }
  p->ws_budget = budget;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return fail(MLMC_ERR_CUDA);
  *out = p;
  return MLMC_OK;
}

mlmc_status mlmc_plan_retarget(mlmc_plan p, const mlmc_config* cfg) {
  if (!p) return MLMC_ERR_INVALID;
  mlmc_status st = validate(cfg);
  if (st != MLMC_OK) return st;
  const mlmc_config& o = p->cfg;
  if (cfg->dim != o.dim || cfg->n_levels != o.n_levels || cfg->coarse_cells != o.coarse_cells ||
      cfg->modes_per_dim != o.modes_per_dim || cfg->solver != o.solver ||
      cfg->precision != o.precision || cfg->total_order != o.total_order ||
      cfg->z_chunk != o.z_chunk)
    return MLMC_ERR_INVALID;
  if (!p->round_count.empty()) return MLMC_ERR_INVALID;
  CK(cudaStreamSynchronize(p->stream));
  if (settle_graph_launches(p) != MLMC_OK) return MLMC_ERR_CUDA;
  clear_graphs(p);   // graphs bake field parameters, seeds and tolerances
  const int m = cfg->modes_per_dim;
  std::vector<double> omega, theta;
  std::vector<int32_t> even;
  kle_roots(cfg->corr_len, m, omega, theta, even);
  if (ensure_pin(p, sizeof(double) * 2 * m + sizeof(int32_t) * m) != MLMC_OK) return MLMC_ERR_OOM;
  double* hp = (double*)p->h_pin;
  std::memcpy(hp, omega.data(), sizeof(double) * m);
  std::memcpy(hp + m, theta.data(), sizeof(double) * m);
  std::memcpy(hp + 2 * m, even.data(), sizeof(int32_t) * m);
  CK(cudaMemcpyAsync(p->d_omega, hp, sizeof(double) * m, cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemcpyAsync(p->d_theta, hp + m, sizeof(double) * m, cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemcpyAsync(p->d_even, hp + 2 * m, sizeof(int32_t) * m, cudaMemcpyHostToDevice, p->stream));
  for (auto& mi : p->meshes)
    CK(run(p, KID_TABLE, [&] { return launch_kle_table(p->stream, mi.n, m, p->d_omega, p->d_theta, p->d_even, mi.table); }));
  p->cfg = *cfg;
  p->sqrt_sigma2 = std::sqrt(cfg->sigma2);
  if (cfg->workspace_bytes && !p->ws_borrowed) p->ws_budget = cfg->workspace_bytes;
  CK(cudaMemsetAsync(p->d_states, 0, sizeof(mlmc_level_state) * cfg->n_levels, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return MLMC_OK;
}

mlmc_status mlmc_plan_set_workspace(mlmc_plan p, void* ws, uint64_t bytes) {
  if (!p || (ws && (bytes == 0 || ((uintptr_t)ws & 255) != 0))) return MLMC_ERR_INVALID;
  if (!p->round_count.empty()) return MLMC_ERR_INVALID;
  CK(cudaStreamSynchronize(p->stream));
  if (settle_graph_launches(p) != MLMC_OK) return MLMC_ERR_CUDA;
  clear_graphs(p);   // graphs bake workspace addresses
  if (p->ws && !p->ws_borrowed) ws_release(p->ws, p->ws_bytes);
  p->ws = ws;
  p->ws_bytes = ws ? (size_t)bytes : 0;
  p->ws_borrowed = ws != nullptr;
  if (ws) p->ws_budget = (size_t)bytes;
  return MLMC_OK;
}

int64_t mlmc_round_bytes(const mlmc_config* cfg, const int64_t* count) {
  if (!cfg || !count || validate(cfg) != MLMC_OK) return -1;
  const int M = (int)coef_count(cfg);
  std::vector<MeshInfo> meshes(cfg->n_levels);
  for (int l = 0; l < cfg->n_levels; ++l) mesh_info_shape(*cfg, l, meshes[l]);
  std::vector<int64_t> f(cfg->n_levels, 0), c(count, count + cfg->n_levels);
  for (auto& x : c) x = std::max<int64_t>(x, 0);
  return (int64_t)round_chunks_of(*cfg, meshes.data(), M, f, c, nullptr);
}

mlmc_status mlmc_release_cached_memory(void) {
  std::vector<WsBlock> all;
  {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    all.swap(g_ws_cache);
  }
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return MLMC_ERR_CUDA;
  cudaError_t first = cudaSuccess;
  for (const WsBlock& w : all) {
    cudaError_t e = cudaSetDevice(w.dev);
    if (e == cudaSuccess) e = cudaFree(w.ptr);
    if (e != cudaSuccess && first == cudaSuccess) first = e;
  }
  if (cudaSetDevice(cur) != cudaSuccess || first != cudaSuccess) return MLMC_ERR_CUDA;
  return MLMC_OK;
}

mlmc_status mlmc_plan_destroy(mlmc_plan p) {
  if (!p) return MLMC_ERR_INVALID;
  cudaStreamSynchronize(p->stream);
  clear_graphs(p);
  if (p->group_graph.exec) cudaGraphExecDestroy(p->group_graph.exec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  for (auto bs : p->branch) cudaStreamDestroy(bs);
  for (auto ev : p->branch_ev) cudaEventDestroy(ev);
  if (p->round_done) cudaEventDestroy(p->round_done);
  for (auto& mi : p->meshes)
    if (mi.table) cudaFree(mi.table);
  cudaFree(p->d_omega);
  cudaFree(p->d_slot);
  cudaFree(p->d_theta);
  cudaFree(p->d_even);
  cudaFree(p->d_states);
  cudaFree(p->d_cost);
  cudaFree(p->d_small);
  cudaFree(p->d_N);
  cudaFree(p->d_prof);
  if (p->ws && !p->ws_borrowed) ws_release(p->ws, p->ws_bytes);
  if (p->d_fold) cudaFree(p->d_fold);
  if (p->h_pin) cudaFreeHost(p->h_pin);
  for (auto& e : p->pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : p->pool) cudaEventDestroy(e);
  delete p;
  return MLMC_OK;
}

mlmc_status mlmc_reset_stats(mlmc_plan p) {
  if (!p) return MLMC_ERR_INVALID;
  CK(cudaMemsetAsync(p->d_states, 0, sizeof(mlmc_level_state) * p->cfg.n_levels, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return MLMC_OK;
}

mlmc_status mlmc_draw_xi(mlmc_plan p, int level, int64_t first, int64_t count, double* xi) {
  if (!p || level < 0 || level >= p->cfg.n_levels || first < 0 || count < 0 ||
      first + count > (int64_t(1) << 32) || (count > 0 && !xi))
    return MLMC_ERR_INVALID;
  CK(run(p, KID_XI, [&] {
    return launch_draw_xi(p->stream, p->cfg.seed, p->cfg.stream_id, level, first, count, p->M, xi,
                          prof_for(p, KID_XI, p->M * 8.0));
  }));
  return MLMC_OK;
}

mlmc_status mlmc_kappa(mlmc_plan p, int mesh, const double* xi, int64_t count, double* kappa) {
  if (!p || mesh < 0 || mesh >= p->cfg.n_levels || count < 0 || (count > 0 && (!xi || !kappa)))
    return MLMC_ERR_INVALID;
  const Grid& g = p->meshes[mesh].g[0];
  for (int64_t off = 0; off < count; off += 65535) {
    const int64_t B = std::min<int64_t>(65535, count - off);
    mlmc_status st = make_kappa(p, mesh, xi + off * p->M, B, kappa + off * g.es);
    if (st != MLMC_OK) return st;
  }
  return MLMC_OK;
}

mlmc_status mlmc_kappa32(mlmc_plan p, int mesh, const double* xi, int64_t count, float* kappa32) {
  if (!p || mesh < 0 || mesh >= p->cfg.n_levels || count < 0 || (count > 0 && (!xi || !kappa32)))
    return MLMC_ERR_INVALID;
  const MeshInfo& mi = p->meshes[mesh];
  p->tc_used = true;
  for (int64_t off = 0; off < count; off += 65535) {
    const int64_t B = std::min<int64_t>(65535, count - off);
    CK(run(p, KID_KAPPA, [&] {
      return launch_kappa32_tc(p->stream, mi.g[0], p->cfg.modes_per_dim, p->sqrt_sigma2, mi.table,
                               xi + off * p->M, p->M, p->d_slot, B, kappa32 + off * mi.g[0].es);
    }));
  }
  return MLMC_OK;
}

mlmc_status mlmc_apply(mlmc_plan p, int mesh, const double* kappa, const double* x, double* y,
                       int64_t count) {
  if (!p || mesh < 0 || mesh >= p->cfg.n_levels || count < 0 ||
      (count > 0 && (!kappa || !x || !y)))
    return MLMC_ERR_INVALID;
  const Grid& g = p->meshes[mesh].g[0];
  for (int64_t off = 0; off < count; off += 65535) {
    const int64_t B = std::min<int64_t>(65535, count - off);
    CK(run(p, KID_APPLY, [&] {
      return op::apply(p->stream, g, kappa + off * g.es, x + off * g.ns, y + off * g.ns, B,
                       prof_for(p, KID_APPLY, (2 * nodes_of(g) + elems_of(g)) * 8));
    }));
  }
  return MLMC_OK;
}

mlmc_status mlmc_apply32(mlmc_plan p, int mesh, const float* kappa32, const float* x, float* y,
                         int64_t count) {
  if (!p || mesh < 0 || mesh >= p->cfg.n_levels || count < 0 ||
      (count > 0 && (!kappa32 || !x || !y)))
    return MLMC_ERR_INVALID;
  const Grid& g = p->meshes[mesh].g[0];
  if (g.dim == 3) p->zw_used = true;
  for (int64_t off = 0; off < count; off += 65535) {
    const int64_t B = std::min<int64_t>(65535, count - off);
    CK(run(p, KID_APPLY, [&] {
      return op::apply(p->stream, g, kappa32 + off * g.es, x + off * g.ns, y + off * g.ns, B,
                       prof_for(p, KID_APPLY, (2 * nodes_of(g) + elems_of(g)) * 4));
    }));
  }
  return MLMC_OK;
}

mlmc_status mlmc_solve(mlmc_plan p, int mesh, const double* kappa, int64_t count, double* u,
                       double* q, int32_t* iters) {
  if (!p || mesh < 0 || mesh >= p->cfg.n_levels || count < 0 || (count > 0 && (!kappa || !q)))
    return MLMC_ERR_INVALID;
  const MeshInfo& mi = p->meshes[mesh];
  const bool mixed = is_mixed(p);
  const int64_t Bmax = max_batch(p, [&](int64_t B) { return solve_bytes(mi, B, mixed); }, count);
  bool bad = false;
  for (int64_t off = 0; off < count; off += Bmax) {
    const int64_t B = std::min<int64_t>(Bmax, count - off);
    mlmc_status st = ensure_ws(p, solve_bytes(mi, B, mixed));
    if (st != MLMC_OK) return st;
    Carve c(p->ws);
    const double* kap = kappa + off * mi.g[0].es;
    int32_t* it_dev = nullptr;
    const double* x = nullptr;
    if (mixed) {
      MixedWs w;
      carve_mixed(c, mi, B, w);
      CK(cudaMemcpyAsync(w.kap64, kap, sizeof(double) * B * mi.g[0].es, cudaMemcpyDeviceToDevice, p->stream));
      st = solve_mixed(p, mesh, mi, w, B, q + off, iters ? iters + off : nullptr, Guess{});
      it_dev = w.outer.iters;
      x = w.u;
    } else {
      SolveWs<double> w;
      carve_solve(c, mi, B, false, w);
      w.kap[0] = const_cast<double*>(kap);
      st = solve_fp64(p, mesh, mi, w, B, q + off, iters ? iters + off : nullptr, Guess{});
      it_dev = w.sc.iters;
      x = w.x;
    }
    if (st != MLMC_OK) return st;
    if (u) CK(cudaMemcpyAsync(u + off * mi.g[0].ns, x, sizeof(double) * B * mi.g[0].ns, cudaMemcpyDeviceToDevice, p->stream));
    if (ensure_pin(p, sizeof(int32_t) * B) != MLMC_OK) return MLMC_ERR_OOM;
    CK(cudaMemcpyAsync(p->h_pin, it_dev, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (settle_graph_launches(p) != MLMC_OK) return MLMC_ERR_CUDA;
    const int32_t* it = (const int32_t*)p->h_pin;
    for (int64_t b = 0; b < B; ++b) bad |= (it[b] < 0);
  }
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}

mlmc_status mlmc_sample_level(mlmc_plan p, int level, int64_t first, int64_t count, double* q_fine,
                              double* q_coarse, int32_t* iters) {
  if (!p || level < 0 || level >= p->cfg.n_levels || first < 0 || count < 0 ||
      first + count > (int64_t(1) << 32))
    return MLMC_ERR_INVALID;
  if (count == 0) return MLMC_OK;
  const MeshInfo& mf = p->meshes[level];
  const int M = p->M;
  const bool mixed = is_mixed(p);
  const int64_t gns = guess_ns_of(p->cfg, level);
  const int64_t Bmax = max_batch(p, [&](int64_t B) { return coupled_bytes(mf, M, B, mixed, gns); }, count);
  const double cost = level_cost_cfg(&p->cfg, level);
  const int sides = level > 0 ? 2 : 1;
  bool bad = false;
  for (int64_t off = 0; off < count; off += Bmax) {
    const int64_t B = std::min<int64_t>(Bmax, count - off);
    mlmc_status st = ensure_ws(p, coupled_bytes(mf, M, B, mixed, gns));
    if (st != MLMC_OK) return st;
    for (int k = 0; k < sides; ++k) {
      // side 0: mesh `level` (fine), side 1: mesh `level - 1` (coarse); the
      // carve prefix (xi, q_f, q_c, iteration counts, guess) is identical for
      // both. With the nested guess the coarse mesh is solved first.
      const int side = gns > 0 ? sides - 1 - k : k;
      const int mesh = level - side;
      const MeshInfo& mi = p->meshes[mesh];
      Carve c(p->ws);
      CoupledWs w;
      carve_coupled(c, mi, M, B, mixed, gns, side, w);
      if (k == 0) {
        st = mlmc_draw_xi(p, level, first + off, B, w.xi);
        if (st != MLMC_OK) return st;
      }
      st = make_kappa(p, mesh, w.xi, B, w.kap);
      if (st != MLMC_OK) return st;
      double* qd = side == 0 ? w.qf : w.qc;
      int32_t* itd = side == 0 ? w.itf : w.itc;
      const Guess gs = guess_views(p, level, side, mixed, w);
      st = mixed ? solve_mixed(p, mesh, mi, w.mx, B, qd, itd, gs)
                 : solve_fp64(p, mesh, mi, w.s, B, qd, itd, gs);
      if (st != MLMC_OK) return st;
    }
    Carve c(p->ws);
    CoupledWs w;
    carve_coupled(c, mf, M, B, mixed, gns, 0, w);
    CK(run(p, KID_WELFORD, [&] {
      return launch_welford(p->stream, w.qf, level > 0 ? w.qc : nullptr, B, p->d_states + level, cost);
    }));
    const size_t need = sizeof(double) * 2 * B + sizeof(int32_t) * 2 * B;
    if (ensure_pin(p, need) != MLMC_OK) return MLMC_ERR_OOM;
    double* hq = (double*)p->h_pin;
    int32_t* hit = (int32_t*)(hq + 2 * B);
    CK(cudaMemcpyAsync(hq, w.qf, sizeof(double) * B, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(hq + B, w.qc, sizeof(double) * B, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(hit, w.itf, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(hit + B, w.itc, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    if (settle_graph_launches(p) != MLMC_OK) return MLMC_ERR_CUDA;
    for (int64_t b = 0; b < B; ++b) {
      if (hit[b] < 0 || (level > 0 && hit[B + b] < 0)) bad = true;
      if (q_fine) q_fine[off + b] = hq[b];
      if (q_coarse) q_coarse[off + b] = level > 0 ? hq[B + b] : 0.0;
      if (iters) iters[off + b] = hit[b];
    }
  }
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}

mlmc_status mlmc_level_fold(mlmc_plan p, int level, const double* qf, const double* qc, int64_t count) {
  if (!p || level < 0 || level >= p->cfg.n_levels || count < 0 || (count > 0 && !qf)) return MLMC_ERR_INVALID;
  if (count == 0) return MLMC_OK;
  if (count > p->fold_cap) {
    CK(cudaStreamSynchronize(p->stream));
    if (p->d_fold) cudaFree(p->d_fold);
    p->d_fold = nullptr;
    p->fold_cap = 0;
    if (cudaMalloc(&p->d_fold, sizeof(double) * 2 * (size_t)count) != cudaSuccess) {
      cudaGetLastError();
      return MLMC_ERR_OOM;
    }
    p->fold_cap = count;
  }
  double* dqf = p->d_fold;
  double* dqc = qc ? p->d_fold + count : nullptr;
  CK(cudaMemcpyAsync(dqf, qf, sizeof(double) * count, cudaMemcpyHostToDevice, p->stream));
  if (qc) CK(cudaMemcpyAsync(dqc, qc, sizeof(double) * count, cudaMemcpyHostToDevice, p->stream));
  const double cost = level_cost_cfg(&p->cfg, level);
  CK(run(p, KID_WELFORD, [&] { return launch_welford(p->stream, dqf, dqc, count, p->d_states + level, cost); }));
  CK(cudaStreamSynchronize(p->stream));
  return MLMC_OK;
}

mlmc_status mlmc_level_stats(mlmc_plan p, int level, mlmc_level_state* out) {
  if (!p || !out || level < 0 || level >= p->cfg.n_levels) return MLMC_ERR_INVALID;
  CK(cudaMemcpyAsync(out, p->d_states + level, sizeof(mlmc_level_state), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return MLMC_OK;
}

mlmc_status mlmc_estimate(mlmc_plan p, double* q_hat, double* stat_var) {
  if (!p) return MLMC_ERR_INVALID;
  CK(run(p, KID_ESTIMATE, [&] {
    return launch_estimate(p->stream, p->d_states, p->cfg.n_levels, p->d_cost, 0.0, p->d_small, nullptr);
  }));
  double h[2];
  CK(cudaMemcpyAsync(h, p->d_small, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (q_hat) *q_hat = h[0];
  if (stat_var) *stat_var = h[1];
  return MLMC_OK;
}

mlmc_status mlmc_allocate(const double* V, const double* C, int n_levels, double eps,
                          int64_t* N_out) {
  if (!V || !C || !N_out || n_levels < 1 || n_levels > 16 || !(eps > 0.0)) return MLMC_ERR_INVALID;
  for (int l = 0; l < n_levels; ++l)
    if (!(V[l] >= 0.0) || !(C[l] > 0.0)) return MLMC_ERR_INVALID;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 2 * 16 + sizeof(int64_t) * 16) != cudaSuccess) {
    cudaGetLastError();
    return MLMC_ERR_OOM;
  }
  int64_t* dN = (int64_t*)(d + 32);
  mlmc_status st = MLMC_OK;
  if (cudaMemcpy(d, V, sizeof(double) * n_levels, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d + 16, C, sizeof(double) * n_levels, cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_allocate(nullptr, d, d + 16, n_levels, eps, dN) != cudaSuccess ||
      cudaMemcpy(N_out, dN, sizeof(int64_t) * n_levels, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = MLMC_ERR_CUDA;
  cudaFree(d);
  return st;
}

mlmc_status mlmc_run(mlmc_plan p, double eps, int64_t pilot, const int64_t* N_fixed, double* q_hat,
                     double* stat_var, int64_t* N_out) {
  if (!p || (!N_fixed && !(eps > 0.0)) || pilot < 0) return MLMC_ERR_INVALID;
  const int L1 = p->cfg.n_levels;
  mlmc_status st = mlmc_reset_stats(p);
  if (st != MLMC_OK) return st;
  std::vector<int64_t> have(L1, 0), target(L1, pilot);
  if (N_fixed)
    for (int l = 0; l < L1; ++l) {
      if (N_fixed[l] < 0) return MLMC_ERR_INVALID;
      target[l] = N_fixed[l];
    }
  bool bad = false;
  for (int round = 0; round < 64; ++round) {
    st = sample_phase(p, have, target, &bad);
    if (st != MLMC_OK) return st;
    if (N_fixed) break;
    CK(run(p, KID_ESTIMATE, [&] {
      return launch_estimate(p->stream, p->d_states, L1, p->d_cost, eps, p->d_small, p->d_N);
    }));
    int64_t hN[16];
    CK(cudaMemcpyAsync(hN, p->d_N, sizeof(int64_t) * L1, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    bool more = false;
    for (int l = 0; l < L1; ++l) {
      if (hN[l] > target[l]) {
        target[l] = hN[l];
        more = true;
      }
    }
    if (!more) break;
  }
  st = mlmc_estimate(p, q_hat, stat_var);
  if (st != MLMC_OK) return st;
  if (N_out)
    for (int l = 0; l < L1; ++l) N_out[l] = have[l];
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}

mlmc_status mlmc_adapt(mlmc_plan p, int32_t L_active, double eps, int64_t* N_out, int32_t* L_out,
                       double* fit_out) {
  if (!p || !N_out || !L_out || !(eps > 0.0) || L_active < 0 || L_active >= p->cfg.n_levels)
    return MLMC_ERR_INVALID;
  CK(run(p, KID_ESTIMATE, [&] {
    return launch_adapt(p->stream, p->d_states, L_active, p->cfg.n_levels - 1, p->d_cost, eps,
                        p->d_N, p->d_small + 8);
  }));
  double h[3];
  CK(cudaMemcpyAsync(N_out, p->d_N, sizeof(int64_t) * (L_active + 1), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(h, p->d_small + 8, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  *L_out = (int32_t)h[0];
  if (fit_out) {
    fit_out[0] = h[1];
    fit_out[1] = h[2];
  }
  return MLMC_OK;
}

mlmc_status mlmc_run_adaptive(mlmc_plan p, double eps, int64_t pilot, int32_t L0, double* q_hat,
                              double* stat_var, int64_t* N_out, int32_t* L_out) {
  if (!p || !(eps > 0.0) || pilot < 1 || L0 < 0) return MLMC_ERR_INVALID;
  const int L1 = p->cfg.n_levels;
  int32_t L = std::min<int32_t>(L0, L1 - 1);
  mlmc_status st = mlmc_reset_stats(p);
  if (st != MLMC_OK) return st;
  std::vector<int64_t> have(L1, 0), target(L1, 0);
  for (int l = 0; l <= L; ++l) target[l] = pilot;
  bool bad = false;
  for (int round = 0; round < 64; ++round) {
    st = sample_phase(p, have, target, &bad);
    if (st != MLMC_OK) return st;
    if (round == 63) break;   // no more phases: keep L the last sampled level
    int64_t N[16];
    int32_t Lnew = L;
    st = mlmc_adapt(p, L, eps, N, &Lnew, nullptr);
    if (st != MLMC_OK) return st;
    bool more = false;
    for (int l = 0; l <= L; ++l)
      if (N[l] > target[l]) {
        target[l] = N[l];
        more = true;
      }
    if (Lnew > L) {
      for (int l = L + 1; l <= Lnew; ++l) target[l] = pilot;
      L = Lnew;
      more = true;
    }
    if (!more) break;
  }
  st = mlmc_estimate(p, q_hat, stat_var);
  if (st != MLMC_OK) return st;
  if (N_out)
    for (int l = 0; l < L1; ++l) N_out[l] = have[l];
  if (L_out) *L_out = L;
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}

// Rebuilds the grids of every mesh (after a change of cfg.z_chunk).
void regrid(mlmc_plan p) {
  for (auto& mi : p->meshes)
    for (int k = 0; k < mi.K; ++k) mi.g[k] = make_grid(p->cfg.dim, mi.g[k].n, p->cfg.z_chunk, p->cfg.stencil_tile);
}

mlmc_status mlmc_autotune(mlmc_plan p, int level, int64_t count, int flags, mlmc_tune_report* out) {
  if (!p || !out || level < 0 || level >= p->cfg.n_levels || count < 1 || count > 4096 ||
      !p->round_count.empty())
    return MLMC_ERR_INVALID;
  const int L1 = p->cfg.n_levels;
  std::vector<mlmc_level_state> saved(L1);
  CK(cudaMemcpyAsync(saved.data(), p->d_states, sizeof(mlmc_level_state) * L1, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  const bool mixed = is_mixed(p);
  std::vector<double> rtols = {p->cfg.inner_rtol};
  if (mixed && (flags & MLMC_TUNE_INNER_RTOL)) rtols = {1e-2, 3e-3, 1e-3, 3e-4, 1e-4};
  std::vector<double> omegas = {p->cfg.mg_omega};
  if (p->cfg.solver == MLMC_GMG_PCG && (flags & MLMC_TUNE_MG_OMEGA)) omegas = {0.7, 0.8, 0.9};
  std::vector<int> zcs = {p->cfg.z_chunk};
  if (p->cfg.dim == 3 && (flags & MLMC_TUNE_Z_CHUNK)) zcs = {0, 24, 32, 64};
  std::vector<int> tiles = {p->cfg.stencil_tile};
  if (p->cfg.dim == 3 && mixed && (flags & MLMC_TUNE_TILE)) tiles = {0, 1, 2};
  std::vector<int> widths = {p->cfg.batch_split};
  const bool tune_split = (flags & MLMC_TUNE_BATCH) && graphs_on(p);
  if (tune_split) {
    widths = {0};
    for (int k = 2; k <= 4 && count / k >= 2; k *= 2) widths.push_back(k);
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MLMC_ERR_CUDA;
  }
  const mlmc_config base = p->cfg;
  mlmc_tune_report r{};
  r.best_ms = -1.0;
  r.worst_ms = -1.0;
  mlmc_status st = MLMC_OK;
  // probe samples far from the indices a run uses; the level states are
  // restored afterwards. Each setting is timed twice (the faster counts), and
  // the plan's own setting is kept unless another one beats it by 2%: the
  // probe is a small sample of the iteration counts, so near-ties are noise.
  const int64_t first = (int64_t(1) << 32) - count;
  // one probe: the level's samples as one round (a graph with a branch per
  // batch; the batch width matters there) or, without graphs, one batched call
  const bool as_round = graphs_on(p);
  auto probe = [&]() -> mlmc_status {
    if (!as_round) return mlmc_sample_level(p, level, first, count, nullptr, nullptr, nullptr);
    std::vector<int64_t> f(L1, 0), c(L1, 0);
    for (int l = tune_split ? 0 : level; l <= level; ++l) {   // the split acts on every level of a round
      f[l] = first;
      c[l] = count;
    }
    mlmc_status s1 = round_launch(p, f, c);
    if (s1 != MLMC_OK) {
      p->round_count.clear();
      p->round_chunks.clear();
      return s1;
    }
    bool bad = false;
    s1 = round_finish(p, &bad);
    return s1 != MLMC_OK ? s1 : (bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK);
  };
  double base_ms = -1.0;
  for (double rt : rtols)
    for (double om : omegas)
      for (int zc : zcs)
        for (int tl : tiles)
          for (int bw : widths) {
            if (st != MLMC_OK) break;
            p->cfg.inner_rtol = rt;
            p->cfg.mg_omega = om;
            p->cfg.z_chunk = zc;
            p->cfg.stencil_tile = tl;
            p->cfg.batch_split = bw;
            if ((st = settle_graph_launches(p)) != MLMC_OK) break;
            clear_graphs(p);
            regrid(p);
            // the first call builds and caches the graphs; the next two are timed
            st = probe();
            if (st == MLMC_ERR_UNIMPLEMENTED) {   // the round does not fit the budget: skip
              st = MLMC_OK;
              continue;
            }
            if (st != MLMC_OK && st != MLMC_ERR_NOT_CONVERGED) break;
            float ms = -1.0f;
            mlmc_status st2 = MLMC_OK;
            for (int rep = 0; rep < 2; ++rep) {
              if (cudaEventRecord(e0, p->stream) != cudaSuccess) { st = MLMC_ERR_CUDA; break; }
              st2 = probe();
              if (cudaEventRecord(e1, p->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                st = MLMC_ERR_CUDA;
                break;
              }
              float t = 0.0f;
              cudaEventElapsedTime(&t, e0, e1);
              if (ms < 0.0f || t < ms) ms = t;
              if (st2 != MLMC_OK) break;
            }
            if (st == MLMC_ERR_CUDA) break;
            st = MLMC_OK;
            ++r.candidates;
            if (st2 == MLMC_ERR_NOT_CONVERGED) continue;   // a setting that fails is never chosen
            if (st2 != MLMC_OK) { st = st2; break; }
            if (rt == base.inner_rtol && om == base.mg_omega && zc == base.z_chunk && tl == base.stencil_tile &&
                bw == base.batch_split)
              base_ms = ms;
            if (r.best_ms < 0.0 || ms < r.best_ms) {
              r.best_ms = ms;
              r.inner_rtol = rt;
              r.mg_omega = om;
              r.z_chunk = zc;
              r.stencil_tile = tl;
              r.batch_split = bw;
            }
            if (ms > r.worst_ms) r.worst_ms = ms;
          }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (base_ms >= 0.0 && base_ms <= 1.02 * r.best_ms) {
    r.best_ms = base_ms;
    r.inner_rtol = base.inner_rtol;
    r.mg_omega = base.mg_omega;
    r.z_chunk = base.z_chunk;
    r.stencil_tile = base.stencil_tile;
    r.batch_split = base.batch_split;
  }
  // apply the best setting (or restore the original one on failure)
  p->cfg = base;
  if (st == MLMC_OK && r.best_ms >= 0.0) {
    p->cfg.inner_rtol = r.inner_rtol;
    p->cfg.mg_omega = r.mg_omega;
    p->cfg.z_chunk = r.z_chunk;
    p->cfg.stencil_tile = r.stencil_tile;
    p->cfg.batch_split = r.batch_split;
  }
  settle_graph_launches(p);
  clear_graphs(p);
  regrid(p);
  CK(cudaMemcpyAsync(p->d_states, saved.data(), sizeof(mlmc_level_state) * L1, cudaMemcpyHostToDevice, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (st != MLMC_OK) return st;
  if (r.best_ms < 0.0) return MLMC_ERR_NOT_CONVERGED;
  *out = r;
  return MLMC_OK;
}

mlmc_status mlmc_profile_enable(mlmc_plan p, int mask) {
  if (!p) return MLMC_ERR_INVALID;
  harvest(p);
  p->prof_mask = (uint32_t)mask;
  p->prof_on = mask != 0;
  return MLMC_OK;
}

mlmc_status mlmc_profile_reset(mlmc_plan p) {
  if (!p) return MLMC_ERR_INVALID;
  harvest(p);
  for (int k = 0; k < NUM_KERNELS; ++k) {
    p->ms[k] = 0.0;
    p->kl[k] = 0;
  }
  CK(cudaMemsetAsync(p->d_prof, 0, sizeof(double) * NUM_KERNELS, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return MLMC_OK;
}

mlmc_status mlmc_kernel_stats(mlmc_plan p, int kid, mlmc_kernel_stat* out) {
  if (!p || !out || kid < 0 || kid >= NUM_KERNELS) return MLMC_ERR_INVALID;
  harvest(p);
  double bytes = 0.0;
  CK(cudaMemcpyAsync(&bytes, p->d_prof + kid, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  out->launches = p->kl[kid];
  out->ms = p->ms[kid];
  out->bytes = bytes;
  return MLMC_OK;
}

mlmc_status mlmc_round_begin(mlmc_plan p, const int64_t* first, const int64_t* count) {
  if (!p || !first || !count) return MLMC_ERR_INVALID;
  if (!graphs_on(p)) return MLMC_ERR_UNIMPLEMENTED;
  if (!p->round_count.empty()) return MLMC_ERR_INVALID;   // a round is in flight
  const int L1 = p->cfg.n_levels;
  std::vector<int64_t> f(first, first + L1), c(count, count + L1);
  for (int l = 0; l < L1; ++l)
    if (f[l] < 0 || c[l] < 0 || f[l] + c[l] > (int64_t(1) << 32)) return MLMC_ERR_INVALID;
  mlmc_status st = round_launch(p, f, c);
  if (st != MLMC_OK) {
    p->round_count.clear();
    p->round_chunks.clear();
  }
  return st;
}

int mlmc_round_ready(mlmc_plan p) {
  if (!p) return -1;
  if (p->round_count.empty()) return 1;
  const cudaError_t e = cudaEventQuery(p->round_done);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  cudaGetLastError();
  return -1;
}

mlmc_status mlmc_round_end(mlmc_plan p) {
  if (!p) return MLMC_ERR_INVALID;
  if (p->round_count.empty()) return MLMC_OK;
  bool bad = false;
  mlmc_status st = round_finish(p, &bad);
  if (st != MLMC_OK) return st;
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}

mlmc_status mlmc_round_begin_group(mlmc_plan* plans, int nplans, const int64_t* first, const int64_t* count,
                                   void* ws, uint64_t ws_bytes) {
  if (!plans || nplans < 1 || nplans > 256 || !first || !count || !ws || ((uintptr_t)ws & 255)) return MLMC_ERR_INVALID;
  mlmc_plan p = plans[0];
  if (!p) return MLMC_ERR_INVALID;
  if (!graphs_on(p)) return MLMC_ERR_UNIMPLEMENTED;
  const int L1 = p->cfg.n_levels;
  for (int j = 0; j < nplans; ++j) {
    mlmc_plan q = plans[j];
    if (!q || !q->round_count.empty() || !q->group.empty() || !same_solve(p->cfg, q->cfg) || q->prof_on)
      return MLMC_ERR_INVALID;
    for (int k = 0; k < j; ++k)
      if (plans[k] == q) return MLMC_ERR_INVALID;
    for (int l = 0; l < L1; ++l) {
      const int64_t f = first[(size_t)j * L1 + l], c = count[(size_t)j * L1 + l];
      if (f < 0 || c < 0 || f + c > (int64_t(1) << 32)) return MLMC_ERR_INVALID;
    }
  }
  p->group.assign(plans, plans + nplans);
  p->group_count.assign(count, count + (size_t)nplans * L1);
  std::vector<int64_t> f(first, first + (size_t)nplans * L1);
  const mlmc_status st = group_launch(p, f, (char*)ws, ws_bytes);
  if (st != MLMC_OK) {
    if (p->group_graph.exec) cudaGraphExecDestroy(p->group_graph.exec);
    p->group_graph = GraphRec{};
    p->group.clear();
    p->group_count.clear();
    p->round_count.clear();
    p->round_chunks.clear();
    p->round_ws = (char*)p->ws;
    p->round_M = p->M;
  }
  return st;
}

int64_t mlmc_round_bytes_group(const mlmc_config* const* cfgs, int nplans, const int64_t* count) {
  if (!cfgs || nplans < 1 || !count) return -1;
  const mlmc_config* c0 = cfgs[0];
  if (!c0 || validate(c0) != MLMC_OK) return -1;
  int64_t Mmax = 1;
  for (int j = 0; j < nplans; ++j) {
    if (!cfgs[j] || validate(cfgs[j]) != MLMC_OK || !same_solve(*c0, *cfgs[j])) return -1;
    Mmax = std::max<int64_t>(Mmax, coef_count(cfgs[j]));
  }
  const int L1 = c0->n_levels;
  const bool mixed = c0->precision == MLMC_MIXED;
  size_t total = 0;
  for (int l = 0; l < L1; ++l) {
    int64_t B = 0;
    for (int j = 0; j < nplans; ++j) {
      if (count[(size_t)j * L1 + l] < 0) return -1;
      B += count[(size_t)j * L1 + l];
    }
    if (B <= 0) continue;
    MeshInfo mi{};
    mesh_info_shape(*c0, l, mi);
    total += (size_t)round_up((int64_t)coupled_bytes(mi, (int)Mmax, B, mixed, guess_ns_of(*c0, l)), 256);
  }
  return (int64_t)total;
}

mlmc_status mlmc_round_end_group(mlmc_plan p, int32_t* member_bad) {
  if (!p) return MLMC_ERR_INVALID;
  if (p->round_count.empty()) return MLMC_OK;
  bool bad = false;
  mlmc_status st = round_finish(p, &bad, member_bad);
  if (st != MLMC_OK) return st;
  return bad ? MLMC_ERR_NOT_CONVERGED : MLMC_OK;
}

mlmc_status mlmc_round_values(mlmc_plan p, int level, double* q_fine, double* q_coarse, int64_t count) {
  if (!p || level < 0 || level >= p->cfg.n_levels || count < 0 || (count > 0 && !q_fine))
    return MLMC_ERR_INVALID;
  if (!p->round_count.empty() || level >= (int)p->done_count.size() || p->done_count[level] != count)
    return MLMC_ERR_INVALID;
  if (count == 0) return MLMC_OK;
  Carve c((char*)p->ws + p->done_off[level]);
  CoupledWs w;
  carve_coupled(c, p->meshes[level], p->M, count, is_mixed(p), guess_ns_of(p->cfg, level), 0, w);
  CK(cudaMemcpyAsync(q_fine, w.qf, sizeof(double) * count, cudaMemcpyDeviceToHost, p->stream));
  if (q_coarse) {
    if (level > 0)
      CK(cudaMemcpyAsync(q_coarse, w.qc, sizeof(double) * count, cudaMemcpyDeviceToHost, p->stream));
  }
  CK(cudaStreamSynchronize(p->stream));
  if (q_coarse && level == 0)
    for (int64_t b = 0; b < count; ++b) q_coarse[b] = 0.0;
  return MLMC_OK;
}

mlmc_status mlmc_allocation(mlmc_plan p, double eps, int64_t* N_out) {
  if (!p || !N_out || !(eps > 0.0)) return MLMC_ERR_INVALID;
  const int L1 = p->cfg.n_levels;
  CK(run(p, KID_ESTIMATE, [&] {
    return launch_estimate(p->stream, p->d_states, L1, p->d_cost, eps, p->d_small, p->d_N);
  }));
  CK(cudaMemcpyAsync(N_out, p->d_N, sizeof(int64_t) * L1, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return MLMC_OK;
}

int64_t mlmc_launch_count(mlmc_plan p) {
  if (!p) return -1;
  cudaStreamSynchronize(p->stream);
  settle_graph_launches(p);
  return p->launches;
}

}  // extern "C"
