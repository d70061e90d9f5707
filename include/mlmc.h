/*
 * mlmc.h - C ABI of libmlmc, the GB300 (sm_103a) batched coupled MLMC
 * sample solve.
 *
 * Method: Badia, Hampton, Principe, "A massively parallel implementation of
 * multilevel Monte Carlo for finite element models" (arXiv 2111.11788).
 * For each level l and sample i the library draws KLE coefficients xi(l, i),
 * forms kappa = exp(Phi xi) on the level-l and level-(l-1) meshes, solves
 * -div(kappa grad u) = 1 (Eq. (model), Sec. 2.1) with preconditioned CG on
 * both meshes, and folds Y_l^i = Q_l - Q_{l-1} (Eq. (mlmc_average)) into
 * per-level Welford statistics (Eq. (sample_variance)) that drive the
 * estimator and the sample allocation (Eq. (mlmc_num_samples)).
 *
 * Conventions for every entry point:
 *  - Return codes only; nothing is thrown across the ABI. On error the
 *    outputs are unspecified.
 *  - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *    pointers are CUDA global memory on the current device, owned by the
 *    caller. The plan owns only its own tables and workspace.
 *  - `stream` arguments are borrowed cudaStream_t handles (NULL = legacy
 *    default stream). Device-pointer entry points are asynchronous on the
 *    plan's stream; host-pointer entry points return after the results are
 *    in host memory.
 *  - Mesh m has n_m = coarse_cells * 2^m cells per side (Sec. 2.2, s = 2),
 *    (n_m + 1)^dim nodes including the boundary, n_m^dim elements.
 *  - Node arrays hold (n+1)^dim doubles per sample, x fastest, boundary
 *    entries included (ignored on input, written as 0 on output), samples
 *    mlmc_node_stride(dim, n) doubles apart. Element arrays hold n^dim
 *    doubles per sample, x fastest, mlmc_elem_stride(dim, n) apart.
 *  - A plan is not thread-safe; distinct plans may be used concurrently.
 */
#ifndef MLMC_H
#define MLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mlmc_status {
  MLMC_OK = 0,
  MLMC_ERR_INVALID = -1,        /* bad argument or configuration */
  MLMC_ERR_OOM = -2,            /* device allocation failed */
  MLMC_ERR_NOT_CONVERGED = -3,  /* some sample hit max_iter (its iters = -1) */
  MLMC_ERR_CUDA = -4,           /* a CUDA runtime call or launch failed */
  MLMC_ERR_TIMEOUT = -5,        /* reserved: a bounded device wait expired */
  MLMC_ERR_UNIMPLEMENTED = -6   /* combination not built (e.g. dim 3 + mixed) */
} mlmc_status;

enum { MLMC_QOI_DOMAIN_MEAN = 0, MLMC_QOI_BOX_MEAN = 1 };
enum { MLMC_JACOBI_PCG = 0, MLMC_GMG_PCG = 1 };
enum { MLMC_FP64 = 0, MLMC_MIXED = 1 };

/* Problem and solver description. Fill with mlmc_config_default() first. */
typedef struct mlmc_config {
  int32_t dim;             /* 2 or 3 */
  int32_t n_levels;        /* L + 1, 1..16 */
  int32_t coarse_cells;    /* n_0 >= 2, cells per side of mesh 0 */
  int32_t modes_per_dim;   /* m; M = m^dim tensor KLE modes, 1..32 */
  double sigma2;           /* variance of the Gaussian log-field (> 0) */
  double corr_len;         /* exponential correlation length (> 0) */
  int32_t qoi;             /* MLMC_QOI_DOMAIN_MEAN | MLMC_QOI_BOX_MEAN */
  int32_t solver;          /* MLMC_JACOBI_PCG | MLMC_GMG_PCG */
  double box_lo, box_hi;   /* QoI box [lo, hi]^dim, node-aligned on every mesh */
  double rtol;             /* stop when ||r||_2 <= rtol ||b||_2 */
  int32_t max_iter;        /* CG iteration cap (> 0) */
  int32_t precision;       /* MLMC_FP64 | MLMC_MIXED (FP32 inner PCG + FP64 refinement) */
  uint64_t seed;           /* Philox key */
  uint32_t stream_id;      /* fourth Philox counter word (request id) */
  int32_t mg_smooth;       /* damped-Jacobi sweeps before and after each coarse correction */
  double mg_omega;         /* Jacobi damping in the smoother */
  int32_t mg_coarsest;     /* cells per side of the coarsest multigrid grid (>= 2) */
  int32_t check_every;     /* CG iterations between convergence polls (0 = auto) */
  uint64_t workspace_bytes;/* device workspace budget for batching (0 = auto) */
  double inner_rtol;       /* MLMC_MIXED: relative tolerance of each FP32 inner solve */
  int32_t inner_max_iter;  /* MLMC_MIXED: iteration cap of each inner solve */
  int32_t outer_max_iter;  /* MLMC_MIXED: cap on FP64 refinement steps */
  int32_t use_graphs;      /* 1: each batched solve runs as one CUDA graph whose
                              while-nodes iterate on the device (no host polls);
                              0: host-driven iterations. Same results either way. */
  int32_t total_order;     /* -1: full tensor basis, M = m^dim modes; K >= 0:
                              total-order truncation (Sec. 5.2): only modes with
                              k_x + k_y (+ k_z) <= K (each k < m), M of them, in
                              the full basis' flat order */
  int32_t z_chunk;         /* 3D: z-planes per stencil CTA (0 = built-in rule:
                              all planes up to 24, else 16); set by mlmc_autotune */
  int32_t nested_guess;    /* 1 (default): in a coupled batch of level l > 0 the
                              mesh l-1 solve runs first and its solution,
                              interpolated (bi/trilinear) to mesh l, is the
                              initial iterate of the mesh l solve; 0: both
                              solves start from u = 0. The stopping test
                              (||r|| <= rtol ||b||) is the same either way. */
  int32_t kle_tensor;      /* MLMC_MIXED: 1 = the FP32 kappa of the inner solves
                              is exp of the KLE contraction on the tensor cores
                              (tcgen05, split BF16 with FP32 accumulation, see
                              mlmc_kappa32); 0 (default) = the FP64 kappa rounded
                              to FP32. The FP64 outer residual uses the FP64
                              kappa either way, so results meet the same
                              tolerance; iterates differ in the last digits. */
  int32_t stencil_tile;    /* 3D FP32 stencils: 0 (default) = full-width tiles
                              staged by one TMA bulk copy per plane and array
                              where the mesh allows it (32..256 cells per side),
                              four node rows per thread; 2 = the same tiles with
                              two rows per thread; 1 = 32 x 16 column tiles
                              staged by cp.async. Same per-node arithmetic (the
                              per-tile partial sums differ in rounding only);
                              set by mlmc_autotune */
  int32_t batch_split;     /* rounds: each level's batch of coupled samples is
                              split into this many near-equal batches (at most
                              count of them), solved side by side as parallel
                              graph branches and folded in sample order
                              (0 or 1 = one batch per level, up to 64). Same
                              results; set by mlmc_autotune */
} mlmc_config;

/* Per-level Welford state (Eq. (sample_variance): V = m2 / n). */
typedef struct mlmc_level_state {
  int64_t n;
  double mean;
  double m2;
  double cost_sum;         /* sum of the per-sample cost model C_l */
} mlmc_level_state;

typedef struct mlmc_plan_s* mlmc_plan;

/* ---- configuration and layout -------------------------------------- */

/* Defaults: 2D, 3 levels, n_0 = 16, m = 4, sigma2 = 1, corr_len = 0.3,
 * domain-mean QoI, Jacobi-PCG, rtol 1e-10, FP64, seed 0, mg_omega 0.9,
 * CUDA graphs on, full tensor KLE basis (total_order -1), nested initial
 * guess on; mixed form: inner_rtol 3e-3, inner_max_iter 200,
 * outer_max_iter 40.
 *
 * MLMC_MIXED (iterative refinement, the precision pattern the method admits
 * on GB300): u = u0 (0, or the nested guess), r = b - A u; repeat { d = A32^-1 (r / s) by FP32 PCG with
 * kappa32 = (float) kappa to inner_rtol; u += s d; r = b - A(kappa) u in
 * FP64; s = ||r|| } until ||r||_2 <= rtol ||b||_2 (the FP64 true residual),
 * or until a refinement step no longer halves ||r|| while ||r|| is already
 * within 100 rtol ||b||: the FP64 evaluation of b - A u cannot resolve a
 * smaller residual there (for high-contrast kappa its rounding floor can sit
 * a few times above rtol ||b||). iters then counts all inner iterations; -1
 * if outer_max_iter was hit. */
void mlmc_config_default(mlmc_config* cfg);

/* Doubles between consecutive samples in node / element arrays. */
int64_t mlmc_node_stride(int dim, int n);
int64_t mlmc_elem_stride(int dim, int n);

/* Cells per side of mesh `mesh` (n_0 * 2^mesh), or -1 if out of range. */
int64_t mlmc_mesh_cells(const mlmc_config* cfg, int mesh);

/* KLE coefficients per sample (the length of one xi): m^dim, or the number
 * of modes kept by the total-order truncation (Sec. 5.2); -1 for an
 * invalid configuration. */
int64_t mlmc_coef_count(const mlmc_config* cfg);

/* Deterministic level cost C_l = interior DOFs of mesh l + of mesh l-1
 * (the paper measures CPU time per Y_l, Sec. 2.3). */
double mlmc_level_cost(const mlmc_config* cfg, int level);

const char* mlmc_status_str(mlmc_status s);

/* ---- plan ----------------------------------------------------------- */

/* Validates cfg, solves the 1D KLE eigenproblems (Sec. 5.2 exponential
 * covariance; Ghanem & Spanos closed form), builds the per-mesh tables on
 * the device and zeroes the level states. `stream` is borrowed for the
 * plan's lifetime. Errors: INVALID, OOM, CUDA. */
mlmc_status mlmc_plan_create(const mlmc_config* cfg, void* stream, mlmc_plan* out);
/* Destroys the plan after its stream's work has completed. The plan's own
 * workspace (not one set by mlmc_plan_set_workspace) is kept by the library
 * for the next plan on the same device that needs at most its size (up to
 * four blocks, the oldest freed first; a failed allocation frees this
 * device's kept blocks and retries), so creating plans in a loop does not
 * unmap and map gigabytes each time. */
mlmc_status mlmc_plan_destroy(mlmc_plan plan);
/* Returns the workspaces kept from destroyed plans to the driver (call it
 * before handing the memory to another allocator). Errors: CUDA. */
mlmc_status mlmc_release_cached_memory(void);

/* Re-target an idle plan to a configuration of the same shape (dim,
 * n_levels, coarse_cells, modes_per_dim, solver, precision, total_order,
 * z_chunk): field
 * parameters, seed, stream id, tolerances and QoI may change. Rebuilds the
 * KLE tables in place, drops cached graphs and resets the level states;
 * allocates nothing (no device synchronisation from cudaFree). A nonzero
 * workspace_bytes sets the batching budget unless the workspace is
 * borrowed. INVALID for a different shape or while a round is in flight. */
mlmc_status mlmc_plan_retarget(mlmc_plan plan, const mlmc_config* cfg);

/* Give the plan a caller-owned device workspace of `bytes` bytes at `ws`
 * (256-byte aligned) for its batches and rounds; the plan then never
 * allocates or grows a workspace, and the batching budget becomes `bytes`.
 * A plan's own previous workspace is freed; cached graphs are dropped. `ws`
 * must stay valid until the plan is destroyed or given another workspace;
 * NULL returns the plan to its own (lazily allocated) workspace. INVALID
 * while a round is in flight or for a misaligned pointer. */
mlmc_status mlmc_plan_set_workspace(mlmc_plan plan, void* ws, uint64_t bytes);

/* Device workspace bytes of one round with count[l] samples per level
 * (host array of n_levels entries), or -1 for an invalid configuration. */
int64_t mlmc_round_bytes(const mlmc_config* cfg, const int64_t* count);

/* Reset all level states to n = 0. */
mlmc_status mlmc_reset_stats(mlmc_plan plan);

/* Coupled samples first..first+count-1 of `level` (Eq. (mlmc_average)):
 * one xi(level, i) per sample, solved on mesh `level` and, for level > 0,
 * on mesh level-1 (with nested_guess, mesh level-1 first, its solution
 * seeding the mesh `level` solve); Y = Q_f - Q_c is folded into the level
 * state in sample order. Optional host outputs (each `count` long, may be NULL): q_fine,
 * q_coarse (0 for level 0), iters (fine-mesh CG iterations, -1 if not
 * converged). Returns NOT_CONVERGED if any solve hit max_iter (its Y is
 * still folded). Samples must satisfy 0 <= i < 2^32. */
mlmc_status mlmc_sample_level(mlmc_plan plan, int level, int64_t first, int64_t count,
                              double* q_fine, double* q_coarse, int32_t* iters);

/* Fold coupled sample values computed elsewhere (e.g. on other GPUs) into
 * the level's device Welford state (Eq. (sample_variance)), in the order
 * given: Y = qf[s] - qc[s] (qc NULL: Y = qf[s]), each sample adding the
 * level cost C_l to cost_sum. qf, qc: host arrays of `count` doubles. Folding
 * a level's samples in index order reproduces bit for bit the state that
 * mlmc_sample_level builds. Synchronous; may allocate a staging buffer. */
mlmc_status mlmc_level_fold(mlmc_plan plan, int level, const double* qf, const double* qc, int64_t count);

/* Host copy of one level state. */
mlmc_status mlmc_level_stats(mlmc_plan plan, int level, mlmc_level_state* out);

/* Eq. (mlmc_average) and Sec. 2.2: q_hat = sum_l mean_l and
 * stat_var = sum_l (m2_l / n_l) / n_l over levels with n_l > 0 (host outputs). */
mlmc_status mlmc_estimate(mlmc_plan plan, double* q_hat, double* stat_var);

/* Eq. (mlmc_num_samples): N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_i sqrt(V_i C_i)).
 * V, C, N_out are host arrays of n_levels entries; evaluated on the device. */
mlmc_status mlmc_allocate(const double* V, const double* C, int n_levels, double eps,
                          int64_t* N_out);

/* Adaptive MLMC with L fixed (Sec. 2.3, Algorithm 2): `pilot` samples per
 * level, then repeat {N_l from Eq. (mlmc_num_samples) with the current
 * V_l and the cost model; draw the missing samples} until every level has
 * its N_l. With N_fixed (host, n_levels entries) the counts are fixed and
 * eps is ignored. Outputs q_hat, stat_var (host, may be NULL); N_out (host,
 * n_levels, may be NULL) receives the final sample counts. */
mlmc_status mlmc_run(mlmc_plan plan, double eps, int64_t pilot, const int64_t* N_fixed,
                     double* q_hat, double* stat_var, int64_t* N_out);

/* Adaptive MLMC with the number of levels adapted as well (Sec. 2.3,
 * Algorithm 2): start on levels 0..L0 with `pilot` (>= 1) samples each;
 * after every sampling phase run mlmc_adapt and take its sample counts
 * (never lowering one) and its level (new levels get `pilot` samples), until
 * neither changes. The plan's n_levels - 1 is the largest level it may
 * reach; L0 >= 1 is needed for the level to move (the fit needs a level
 * difference). Outputs: estimate and sum_l V_l / N_l over the active levels,
 * N_out (host, n_levels entries, 0 beyond the final level), *L_out the final
 * level. NOT_CONVERGED as for mlmc_run. */
mlmc_status mlmc_run_adaptive(mlmc_plan plan, double eps, int64_t pilot, int32_t L0,
                              double* q_hat, double* stat_var, int64_t* N_out, int32_t* L_out);

/* One adaptive step at a phase boundary, from the device level states of
 * levels 0..L_active: N_out[0..L_active] (host) per Eq. (mlmc_num_samples)
 * and *L_out per Eq. (mlmc_num_levels) with s = 2 and the bias model
 * |E(Q_l - Q)| = c 2^(-alpha l), alpha and c fitted by least squares on
 * log2 |mean(Y_l)| over l = 1..L_active (levels with a zero mean skipped;
 * one level: alpha = 2; alpha clamped to [0.5, 4]). *L_out lies in
 * [L_active, n_levels - 1]; it equals L_active when no level l >= 1 has a
 * nonzero mean. fit_out (host, nullable) receives {alpha, c}. */
mlmc_status mlmc_adapt(mlmc_plan plan, int32_t L_active, double eps, int64_t* N_out,
                       int32_t* L_out, double* fit_out);

/* ---- asynchronous allocation rounds ----------------------------------- */

/* Launch samples first[l] .. first[l] + count[l] - 1 of every level l
 * (host arrays of n_levels entries; count 0 skips a level) as one CUDA
 * graph with a branch per level, asynchronously on the plan's stream. The
 * level states are updated when the round completes; at most one round per
 * plan is in flight. Returns UNIMPLEMENTED when graphs are off (use_graphs
 * = 0 or tracing on) or the batches do not fit the workspace budget
 * together (the caller then uses mlmc_sample_level level by level). */
mlmc_status mlmc_round_begin(mlmc_plan plan, const int64_t* first, const int64_t* count);
/* 1 when the launched round (if any) has completed, 0 if not yet, -1 on error. */
int mlmc_round_ready(mlmc_plan plan);
/* Waits for the round; NOT_CONVERGED if a solve hit its iteration cap. */
mlmc_status mlmc_round_end(mlmc_plan plan);
/* Eq. (mlmc_num_samples) from the current level states (V_l = m2_l / n_l)
 * and the cost model: N_out (host, n_levels entries). */
mlmc_status mlmc_allocation(mlmc_plan plan, double eps, int64_t* N_out);
/* Cross-request batching: one allocation round over `nplans` plans whose
 * coupled solves can share launches (same dim, levels, coarse cells, solver,
 * precision, tolerances, iteration caps, multigrid and QoI settings,
 * z_chunk, nested_guess, and kle_tensor 0; their fields sigma2 and
 * corr_len, KLE modes, total order, seeds and stream ids may differ; INVALID
 * otherwise). first and count are host arrays of nplans x n_levels entries
 * (plan k's level l at [k * n_levels + l]): plan k contributes the coupled
 * samples first .. first + count - 1 of level l (Eq. (mlmc_average)). For
 * every level the samples of all plans form ONE batch: each plan draws its
 * xi and forms kappa with its own KLE tables into its range of the batch,
 * the solves on both meshes run once for the whole batch, and each plan's
 * Y_l are folded into its own level state in sample order. The result of
 * every sample, hence every plan's level states, is bit for bit what the
 * plan's own rounds give (the solves are per sample; a converged sample is
 * frozen while the batch finishes). The round is one CUDA graph with a
 * branch per level, launched on plans[0]'s stream and driven by plans[0]:
 * poll it with mlmc_round_ready(plans[0]) and end it with
 * mlmc_round_end_group(plans[0], ...); no plan of the group may be used
 * until then. ws: caller-owned device workspace (256-byte aligned) of at
 * least mlmc_round_bytes_group bytes, held until the round ends.
 * Errors: INVALID, OOM (ws too small), UNIMPLEMENTED (graphs off, tracing on,
 * or more than 65535 samples on a level), CUDA. */
mlmc_status mlmc_round_begin_group(mlmc_plan* plans, int nplans, const int64_t* first, const int64_t* count,
                                   void* ws, uint64_t ws_bytes);
/* Device workspace bytes of mlmc_round_begin_group for plans of these
 * configurations (host array of nplans pointers) and counts (nplans x
 * n_levels); -1 if a configuration is invalid or they cannot share a round. */
int64_t mlmc_round_bytes_group(const mlmc_config* const* cfgs, int nplans, const int64_t* count);
/* Waits for the group round driven by `plan`; member_bad (host, nplans
 * entries, may be NULL) receives 1 for a plan one of whose solves hit its
 * iteration cap. NOT_CONVERGED if any did. */
mlmc_status mlmc_round_end_group(mlmc_plan plan, int32_t* member_bad);

/* Per-sample values of the last finished round (after mlmc_round_end) for
 * one level: q_fine[s] = Q_l and q_coarse[s] = Q_{l-1} (0 for level 0) of
 * sample first[l] + s, s < count, where count must equal the round's count
 * for the level (0: nothing to copy). Host arrays; q_coarse may be NULL.
 * These are the Y_l = Q_l - Q_{l-1} terms of Eq. (mlmc_average) that the
 * round folded into the level state; ranks that split a phase's samples
 * exchange them (16 bytes per sample) and fold them in index order with
 * mlmc_level_fold. Valid until the next call that uses the plan's workspace
 * (a round, mlmc_sample_level, mlmc_solve, mlmc_autotune); INVALID after
 * that, while a round is in flight or for a count that does not match.
 * Synchronous. */
mlmc_status mlmc_round_values(mlmc_plan plan, int level, double* q_fine, double* q_coarse,
                              int64_t count);

/* ---- autotuning ------------------------------------------------------ */

enum { MLMC_TUNE_INNER_RTOL = 1, MLMC_TUNE_MG_OMEGA = 2, MLMC_TUNE_Z_CHUNK = 4, MLMC_TUNE_TILE = 8,
       MLMC_TUNE_BATCH = 16 };

typedef struct mlmc_tune_report {
  int32_t candidates;   /* settings timed */
  int32_t z_chunk;      /* chosen z-planes per 3D stencil CTA (0 = built-in rule) */
  double inner_rtol;    /* chosen inner tolerance (mixed form) */
  double mg_omega;      /* chosen Jacobi damping of the multigrid smoother */
  double best_ms;       /* time of one coupled batch with the chosen setting */
  double worst_ms;      /* slowest setting */
  int32_t stencil_tile; /* chosen 3D FP32 stencil tile shape (mlmc_config.stencil_tile) */
  int32_t batch_split;  /* chosen batches per level in rounds (0 = one) */
} mlmc_tune_report;

/* Time `count` (1..4096) coupled samples of `level` under every setting of
 * the selected knobs (flags: MLMC_TUNE_*; mixed-form inner tolerance
 * 1e-2..1e-4, multigrid damping 0.7..0.9, 3D z-planes per stencil CTA, the
 * 3D FP32 stencil tile shape, and the batch split of rounds: 1, 2 or 4
 * batches per level; with that knob the probe is a round of `count`
 * samples on every level up to `level`) and keep the fastest in the plan's configuration (inner_rtol, mg_omega,
 * z_chunk, stencil_tile, batch_split; each setting is timed twice and the
 * faster time counts; the
 * plan's current setting stays unless another is more than 2% faster;
 * cached graphs are rebuilt; a setting whose
 * solves hit the iteration cap is never chosen). Probe samples use indices
 * just below 2^32; the level states are restored. Solves then stop at the
 * same rtol but their iterates, hence results in the last digits, depend on
 * the chosen setting, and the choice on the measured times. NOT_CONVERGED if
 * no setting converged. */
mlmc_status mlmc_autotune(mlmc_plan plan, int level, int64_t count, int flags, mlmc_tune_report* out);

/* ---- device-level steps (device pointers, asynchronous on the plan's stream) */

/* xi[s * M + k] = xi_k(level, first + s), s < count (the plan's seed and
 * stream_id; Philox4x32-10 counter (k/2, i, level, stream_id)); M = m^dim,
 * or the number of modes kept by the total-order truncation, coefficient k
 * belonging to the k-th kept mode in the full basis' flat order. */
mlmc_status mlmc_draw_xi(mlmc_plan plan, int level, int64_t first, int64_t count, double* xi);

/* kappa = exp(Phi xi) at the element centroids of mesh `mesh` for `count`
 * coefficient vectors xi (count x M, contiguous; Phi restricted to the kept
 * modes under total-order truncation). Output element arrays. */
mlmc_status mlmc_kappa(mlmc_plan plan, int mesh, const double* xi, int64_t count, double* kappa);

/* The FP32 kappa of the mixed form from the tensor cores: kappa32 =
 * exp(Phi xi) at the element centroids of mesh `mesh` (Sec. 5.2 KLE, the
 * dense contraction of the plan's per-axis tables, full or total-order
 * basis, with `count` coefficient vectors xi: device, count x M doubles,
 * contiguous). Phi and xi are each split into two BF16 terms and the three
 * leading products are accumulated in FP32 (tcgen05 MMAs, tensor-memory
 * accumulators): about 1e-5 relative error in kappa32. kappa32: device
 * float element arrays (count x mlmc_elem_stride(dim, n)); asynchronous on
 * the plan's stream. Errors: INVALID, CUDA; TIMEOUT (reported at the next
 * sync point of the plan) if a bounded wait of the kernel gave up. */
mlmc_status mlmc_kappa32(mlmc_plan plan, int mesh, const double* xi, int64_t count, float* kappa32);

/* y = A(kappa) x on mesh `mesh` (Q1 stiffness, homogeneous Dirichlet):
 * node arrays in and out, `count` samples. */
mlmc_status mlmc_apply(mlmc_plan plan, int mesh, const double* kappa, const double* x,
                       double* y, int64_t count);

/* The same operator in FP32, as the mixed form's inner solve applies it
 * (the 3D kernel is the one the plan's stencil_tile selects): y = A(kappa32)
 * x with FP32 arithmetic (error of order 2^-24 times sum |A_ij x_j|). Node
 * and element arrays as in mlmc_apply, in floats; asynchronous on the
 * plan's stream. Errors: INVALID, CUDA; TIMEOUT (at the next sync point)
 * if a bounded wait of the 3D kernel gave up. */
mlmc_status mlmc_apply32(mlmc_plan plan, int mesh, const float* kappa32, const float* x, float* y,
                         int64_t count);

/* Solve A(kappa) u = b (b_i = h^dim) with the configured PCG for `count`
 * samples; u (node arrays, may be NULL), q (QoI, count doubles), iters
 * (count int32, may be NULL; -1 = not converged). */
mlmc_status mlmc_solve(mlmc_plan plan, int mesh, const double* kappa, int64_t count,
                       double* u, double* q, int32_t* iters);

/* ---- solve without device allocation -------------------------------- */

/* Bytes of the static device scratch used by mlmc_solve_noalloc. */
#define MLMC_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* The batched PCG solve of mlmc_solve (the same algorithm: Jacobi- or
 * GMG-PCG with the same stopping test; the QoIs agree with mlmc_solve's to
 * rounding, within 1e-9 relative, and the iteration counts can differ by
 * one) for callers that must not allocate device memory: code living inside
 * another framework's memory arena, latency-critical loops that cannot
 * afford the device synchronisation of cudaMalloc/cudaFree, and hosts that
 * forbid device allocation. It runs the kappa-form 2D kernels with separate
 * coarse levels, where mlmc_solve's FP64 form uses precomputed operator
 * coefficients and a fused V-cycle bottom. The paper has no counterpart; it
 * is a deployment convenience of this library.
 *  - No plan is needed and nothing is allocated: the scratch is a static
 *    device array of MLMC_NOALLOC_SCRATCH_BYTES inside the library, held by
 *    every GPU that loads it until the process exits.
 *  - cfg: dim 2, FP64, Jacobi- or GMG-PCG (as for mlmc_plan_create); mesh
 *    m has n = coarse_cells * 2^m cells per side.
 *  - kappa: device element arrays (count x mlmc_elem_stride(2, n));
 *    q: device, count doubles (QoI per sample); iters: device, count int32
 *    (may be NULL; -1 = not converged). stream: borrowed cudaStream_t.
 *  - Returns MLMC_ERR_INVALID, before launching anything, when count
 *    samples of this mesh need more scratch than MLMC_NOALLOC_SCRATCH_BYTES
 *    (e.g. about 40 GMG samples of 128^2 cells, 10 of 256^2), or
 *    count > 65535; NOT_CONVERGED if a sample hit max_iter.
 *  - The call blocks: it waits on `stream` between convergence checks and
 *    returns once q and iters hold the results.
 *  - The first call on a device looks up the array's device address on
 *    that device; make that first call before any stream capture.
 *  - Every call shares the one array, and the array keeps the last call's
 *    contents (each call writes every scratch entry it reads before reading
 *    it). Calls that overlap on the GPU (other streams, other host threads)
 *    race on it: the caller must serialise them. */
mlmc_status mlmc_solve_noalloc(const mlmc_config* cfg, int mesh, const double* kappa,
                               int64_t count, double* q, int32_t* iters, void* stream);

/* ---- tracing: per-kernel CUDA-event timing -------------------------- */

typedef struct mlmc_kernel_stat {
  int64_t launches;
  double ms;              /* summed event time of the recorded launches */
  double bytes;           /* summed algorithmic DRAM bytes of those launches */
} mlmc_kernel_stat;

int mlmc_kernel_count(void);
const char* mlmc_kernel_name(int kernel_id);
/* `mask` selects kernels by bit (1 << kernel_id; -1 = all, 0 = off). Every
 * launch of a selected kernel is bracketed by CUDA events on the plan's
 * stream and its algorithmic bytes are accumulated on the device; stats
 * accumulate until mlmc_profile_reset. */
mlmc_status mlmc_profile_enable(mlmc_plan plan, int mask);
mlmc_status mlmc_profile_reset(mlmc_plan plan);
mlmc_status mlmc_kernel_stats(mlmc_plan plan, int kernel_id, mlmc_kernel_stat* out);
/* Number of kernel launches issued by this plan since creation. */
int64_t mlmc_launch_count(mlmc_plan plan);

/* ---- measurement ------------------------------------------------------ */

/* Measured FP64 FMA rate of the current device, the peak that FP64-bound
 * kernels are reported against (no passage of the paper; a measurement
 * aid): independent FMA chains on every SM (4 CTAs of 256 threads per SM,
 * 16 chains per thread), timed with CUDA events on `stream` (borrowed; NULL =
 * legacy default stream), best of three launches after a warm-up; synchronous.
 * tflops (host): FP64 TFLOP/s with an FMA counted as 2 flops; ms_out (host,
 * may be NULL): the best launch time. Errors: INVALID (tflops NULL), CUDA. */
mlmc_status mlmc_probe_fp64_rate(void* stream, double* tflops, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_H */
