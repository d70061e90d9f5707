/*
 * mlmc_sched.h - host-side scheduling of sample batches (libmlmc).
 *
 * Two pieces of the paper's scheduler, kept for the multi-GPU sample
 * dispenser and for simulation; both run on the host and touch no GPU.
 *
 *  - The dynamic batch size of Eq. (batch) (Sec. 4): the next batch of a
 *    level is a contiguous range of sample indices whose size follows the
 *    unassigned share of the level, bounded below and above by fractions of
 *    the per-partition share.
 *  - Algorithm 1 (incremental greedy scheduling, Sec. 3) on known task
 *    times, optionally dispensed in batches by a serial coordinator with a
 *    fixed cost per message (the role of the master in Sec. 4, stressed by
 *    the "Pause" model of Sec. 5.1). Theorem 3.1: with q_0 | q_1 | ... |
 *    q_L | p the greedy makespan is below twice the optimum.
 */
#ifndef MLMC_SCHED_H
#define MLMC_SCHED_H

#include "mlmc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. (batch) with the paper's defaults as parameters. Reading of the
 * garbled formula: the batch is the unassigned share spread over the
 * partitions, b = ceil((N - n) / parts), clamped to
 * [max(1, ceil(min_frac * s)), max(1, floor(max_frac * s))] with
 * s = ceil(N / parts) the per-partition share (paper: min_frac = 0.01,
 * max_frac = 1/phi ~ 0.618), and never more than the N - n samples left.
 * Returns 0 when n >= N, -1 for N < 0, n < 0, parts < 1 or fractions
 * outside 0 < min_frac <= max_frac <= 1. */
int64_t mlmc_batch_size(int64_t N, int64_t n, int64_t parts, double min_frac, double max_frac);

typedef struct mlmc_sched_result {
  double makespan;          /* W: last finish time */
  double work_total;        /* W_T = sum_l q_l sum_j w_lj (levels, then tasks, in index order) */
  double work_lb;           /* W_LB = max(W_T / p, largest task or batch time) */
  double last_start;        /* start time of the last task (batch) to start */
  double idle_before_last;  /* processor-time idle in [0, last_start] */
  int64_t batches;          /* dispatches (tasks when batching is off) */
} mlmc_sched_result;

/* Simulate Algorithm 1. Level l has n_tasks[l] tasks needing q[l]
 * processors each, task times w (host, levels one after the other in index
 * order, tasks in index order). Levels are scheduled finest first (l =
 * n_levels - 1 .. 0); at level l the p processors form p / q[l] aligned
 * groups, and the next task (or batch) goes to the group that becomes free
 * first (ties: lowest group), starting when the group is free and the
 * coordinator has dispatched it: each dispatch occupies the coordinator for
 * dispatch_cost seconds, dispatches served in request order. batch != 0
 * dispenses contiguous task ranges sized by mlmc_batch_size(n_tasks[l],
 * assigned, p / q[l], min_frac, max_frac), run back to back on one group;
 * batch == 0 dispenses single tasks. start (host, nullable, one per task in
 * w's order) receives each task's start time. INVALID unless 1 <= q[0],
 * q[l] divides q[l + 1], q[n_levels - 1] divides p, n_tasks >= 0 and
 * w >= 0. */
mlmc_status mlmc_schedule_greedy(int n_levels, const int64_t* q, const int64_t* n_tasks,
                                 const double* w, int64_t p, int batch, double min_frac,
                                 double max_frac, double dispatch_cost, mlmc_sched_result* out,
                                 double* start);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_SCHED_H */
