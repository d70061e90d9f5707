/*
 * mlmc_server.h - continuous-batching MLMC estimation server on top of the
 * plan API of mlmc.h.
 *
 * A request is one adaptive MLMC estimation (Sec. 2.3): a problem description (mlmc_config: field parameters,
 * hierarchy, solver, precision, seed) and a target RMSE eps. The server runs
 * it exactly like mlmc_run(plan, eps, pilot, NULL, ...): pilot samples on
 * every level, then the sample counts of Eq. (mlmc_num_samples) from the
 * request's own device-resident Welford variances (Eq. (sample_variance)),
 * then the missing samples, until no level needs more; or, with adapt_from
 * = k >= 1, like mlmc_run_adaptive(plan, eps, pilot, k, ...), which also
 * raises the number of levels by Eq. (mlmc_num_levels). Its estimate and
 * variance are bitwise those of that plan call with the same configuration
 * and pilot, whatever other requests run beside it: a sample's result depends
 * only on (config, level, sample index) and every level folds its samples
 * into its Welford state in sample order.
 *
 * Continuous batching: one worker thread owns the GPU work. It admits
 * queued requests in arrival order while a slot is free and the request's
 * round workspace fits the HBM budget, gives each admitted request a plan
 * and a stream of its own (plans of the same shape are pooled and
 * re-targeted, so a warm server allocates nothing), and keeps one round of
 * every admitted request in flight at once: each round is one CUDA graph
 * with a branch per level, so coupled solves of every mesh size from every
 * request overlap on the device. A finished round is followed at once by the
 * request's next one (or its allocation step); a finished request frees its
 * slot and workspace for the next queued one. Requests that want a round at
 * the same moment and can share solves are launched as one group round
 * (mlmc_round_begin_group): same-size levels of different requests are then
 * solved by the same batched launches.
 *
 * The paper has no server; its closest counterpart is the dynamic scheduler
 * of Sec. 3-4 that feeds processor groups with sample batches.
 *
 * Thread safety: submit, poll, drain and clock may be called from any
 * thread; create and destroy from one.
 */
#ifndef MLMC_SERVER_H
#define MLMC_SERVER_H

#include "mlmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlmc_server_s* mlmc_server;

typedef struct mlmc_server_config {
  uint64_t hbm_budget;   /* bytes of round workspace admitted at once
                            (0 = 60% of the device's free memory at create) */
  int32_t max_slots;     /* requests in flight at once, 1..256 */
  int32_t pilot;         /* pilot samples per level (>= 2) */
  int32_t device;        /* CUDA device ordinal */
  int32_t max_rounds;    /* cap on allocation rounds per request (0 = 64) */
  int32_t adapt_from;    /* 0: every request samples all its levels (L fixed,
                            as mlmc_run); k >= 1: requests start on levels
                            0..k and adapt L (as mlmc_run_adaptive, L0 = k) */
  int32_t solo_rounds;   /* 0 (default): cross-request batching - requests
                            whose coupled solves can share launches (same
                            meshes, solver, precision, tolerances; see
                            mlmc_round_begin_group) and want a round at the
                            same moment run it as ONE group round: per level
                            their samples form one batch, solved by one set
                            of launches. 1: every request runs its own
                            rounds. Results are the same either way. */
} mlmc_server_config;

typedef struct mlmc_request_result {
  uint64_t id;
  int32_t status;        /* mlmc_status of the request (OK, NOT_CONVERGED, ...) */
  int32_t rounds;        /* rounds of sampling launched */
  int32_t levels;        /* levels sampled: final L + 1 */
  int32_t group_rounds;  /* of those, rounds run together with other requests */
  double q_hat;          /* Eq. (mlmc_average) */
  double stat_var;       /* sum_l V_l / N_l */
  double t_submit;       /* seconds on the server clock */
  double t_admit;
  double t_done;
  double dof_solves;     /* sum_l N_l C_l: interior DOFs of both meshes per sample */
  int64_t N[16];         /* samples taken per level */
} mlmc_request_result;

/* Start a server (and its worker thread) on cfg->device. */
mlmc_status mlmc_server_create(const mlmc_server_config* cfg, mlmc_server* out);

/* Queue one request. `cfg` is copied; cfg->workspace_bytes and
 * cfg->use_graphs are overridden by the server. Returns INVALID for an
 * invalid configuration or eps <= 0, and the request id in *id. */
mlmc_status mlmc_server_submit(mlmc_server s, const mlmc_config* cfg, double eps, uint64_t* id);

/* *done = 1 and *out filled (out may be NULL) when request `id` has
 * finished; *done = 0 while it is queued or running. INVALID for an
 * unknown id. */
mlmc_status mlmc_server_poll(mlmc_server s, uint64_t id, int* done, mlmc_request_result* out);

/* Block until every submitted request has finished, or `timeout_s` seconds
 * passed (TIMEOUT). */
mlmc_status mlmc_server_drain(mlmc_server s, double timeout_s);

/* Seconds since the server was created (the clock of the result times). */
double mlmc_server_clock(mlmc_server s);

/* Stop the worker after the requests in flight finish, then free every
 * pooled plan and stream. Queued requests that were not admitted are
 * dropped. */
mlmc_status mlmc_server_destroy(mlmc_server s);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_SERVER_H */
