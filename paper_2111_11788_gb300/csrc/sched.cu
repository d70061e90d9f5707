// Host-side scheduling pieces (include/mlmc_sched.h): the dynamic batch size
// of Eq. (batch) and a simulator of Algorithm 1 (incremental greedy
// scheduling, Sec. 3) with an optional serial coordinator (Sec. 4).
#include "mlmc.h"
#include "mlmc_sched.h"

#include <algorithm>
#include <cmath>
#include <vector>

extern "C" {

int64_t mlmc_batch_size(int64_t N, int64_t n, int64_t parts, double min_frac, double max_frac) {
  if (N < 0 || n < 0 || parts < 1 || !(min_frac > 0.0) || !(min_frac <= max_frac) || !(max_frac <= 1.0))
    return -1;
  if (n >= N) return 0;
  const int64_t share = (N + parts - 1) / parts;          // samples per partition
  int64_t b = (N - n + parts - 1) / parts;                 // unassigned share per partition
  const int64_t lo = std::max<int64_t>(1, (int64_t)std::ceil(min_frac * (double)share));
  const int64_t hi = std::max<int64_t>(1, (int64_t)std::floor(max_frac * (double)share));
  b = std::min(std::max(b, lo), hi);
  return std::min(b, N - n);
}

mlmc_status mlmc_schedule_greedy(int n_levels, const int64_t* q, const int64_t* n_tasks,
                                 const double* w, int64_t p, int batch, double min_frac,
                                 double max_frac, double dispatch_cost, mlmc_sched_result* out,
                                 double* start) {
  if (n_levels < 1 || !q || !n_tasks || !out || p < 1 || !(dispatch_cost >= 0.0)) return MLMC_ERR_INVALID;
  if (q[0] < 1) return MLMC_ERR_INVALID;
  for (int l = 0; l < n_levels; ++l) {
    if (n_tasks[l] < 0) return MLMC_ERR_INVALID;
    if (l + 1 < n_levels && q[l + 1] % q[l] != 0) return MLMC_ERR_INVALID;
  }
  if (p % q[n_levels - 1] != 0) return MLMC_ERR_INVALID;
  if (batch && mlmc_batch_size(1, 0, 1, min_frac, max_frac) < 0) return MLMC_ERR_INVALID;
  std::vector<int64_t> off(n_levels + 1, 0);
  for (int l = 0; l < n_levels; ++l) off[l + 1] = off[l] + n_tasks[l];
  if (off[n_levels] > 0 && !w) return MLMC_ERR_INVALID;
  for (int64_t t = 0; t < off[n_levels]; ++t)
    if (!(w[t] >= 0.0) || !std::isfinite(w[t])) return MLMC_ERR_INVALID;

  mlmc_sched_result r{};
  for (int l = 0; l < n_levels; ++l) {
    double s = 0.0;
    for (int64_t j = 0; j < n_tasks[l]; ++j) s += w[off[l] + j];
    r.work_total += (double)q[l] * s;
  }
  std::vector<double> fin((size_t)p, 0.0);   // finish time of each processor
  double idle = 0.0, coord = 0.0, big = 0.0, last = 0.0;
  for (int l = n_levels - 1; l >= 0; --l) {
    const int64_t G = p / q[l];
    int64_t assigned = 0;
    while (assigned < n_tasks[l]) {
      // the group that becomes free first (its processors finish together
      // except right after a level change, hence the max)
      int64_t g_best = 0;
      double ready_best = 0.0;
      for (int64_t g = 0; g < G; ++g) {
        double ready = 0.0;
        for (int64_t k = g * q[l]; k < (g + 1) * q[l]; ++k) ready = std::max(ready, fin[(size_t)k]);
        if (g == 0 || ready < ready_best) {
          ready_best = ready;
          g_best = g;
        }
      }
      const int64_t b = batch ? mlmc_batch_size(n_tasks[l], assigned, G, min_frac, max_frac) : 1;
      coord = std::max(coord, ready_best) + dispatch_cost;
      const double s = coord;
      double t = s;
      for (int64_t j = assigned; j < assigned + b; ++j) {
        if (start) start[off[l] + j] = t;
        t += w[off[l] + j];
      }
      big = std::max(big, t - s);
      last = std::max(last, s);
      for (int64_t k = g_best * q[l]; k < (g_best + 1) * q[l]; ++k) {
        idle += s - fin[(size_t)k];
        fin[(size_t)k] = t;
      }
      assigned += b;
      ++r.batches;
    }
  }
  for (int64_t k = 0; k < p; ++k) {
    r.makespan = std::max(r.makespan, fin[(size_t)k]);
    if (fin[(size_t)k] < last) idle += last - fin[(size_t)k];
  }
  r.last_start = last;
  r.idle_before_last = idle;
  r.work_lb = std::max(r.work_total / (double)p, big);
  *out = r;
  return MLMC_OK;
}

}  // extern "C"
