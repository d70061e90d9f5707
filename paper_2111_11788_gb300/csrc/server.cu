// Continuous-batching MLMC estimation server (include/mlmc_server.h).
//
// Built only on the public plan API of mlmc.h: every request runs the
// adaptive loop of Sec. 2.3 (pilot samples, the allocation of
// Eq. (mlmc_num_samples) from the request's device-resident Welford states,
// the missing samples, repeat) as a chain of asynchronous rounds, and one
// worker thread interleaves the rounds of every admitted request, so their
// CUDA graphs (one branch per level) run side by side on the device.
#include "mlmc.h"
#include "mlmc_server.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxLevels = 16;

// Plans of one shape can be re-targeted to each other's configurations.
using ShapeKey = std::tuple<int, int, int, int, int, int, int, int>;

ShapeKey shape_of(const mlmc_config& c) {
  return ShapeKey(c.dim, c.n_levels, c.coarse_cells, c.modes_per_dim, c.solver, c.precision,
                  c.total_order, c.z_chunk);
}

struct Slot {
  mlmc_plan plan = nullptr;
  cudaStream_t stream = nullptr;
};

struct Request {
  mlmc_config cfg{};
  double eps = 0.0;
  mlmc_request_result res{};
  // running state
  std::unique_ptr<Slot> slot;
  uint64_t reserve = 0;   // bytes of the server's workspace arena held
  uint64_t offset = 0;
  int64_t have[kMaxLevels] = {};
  int64_t target[kMaxLevels] = {};
  int64_t inflight[kMaxLevels] = {};
  int phases = 0;   // completed sampling phases (each ends with an allocation)
  int L = 0;        // highest active level
  bool bad = false;
  bool finished = false;
  bool pending = false;        // its next round (inflight counts) waits for launch
  Request* driver = nullptr;   // in a group round: the member whose plan drives it
  std::vector<Request*> members;                // driver only: the group, driver first
  uint64_t group_off = 0, group_bytes = 0;      // driver only: the group's arena block
};

constexpr int kMaxGroup = 32;   // requests per group round

}  // namespace

struct mlmc_server_s {
  mlmc_server_config cfg{};
  Clock::time_point t0;
  std::thread worker;

  std::mutex mu;                      // guards inbox, results, counters, stop
  std::condition_variable cv_work;    // worker: new request or stop
  std::condition_variable cv_done;    // drain: a request finished
  std::deque<std::unique_ptr<Request>> inbox;
  std::unordered_map<uint64_t, mlmc_request_result> results;
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0;
  bool stop = false;

  // worker-only state
  std::deque<std::unique_ptr<Request>> queue;
  std::vector<std::unique_ptr<Request>> active;
  std::map<ShapeKey, std::vector<std::unique_ptr<Slot>>> pool;
  // round workspaces of the admitted requests are carved from one arena of
  // hbm_budget bytes (first fit, free blocks coalesced)
  char* arena = nullptr;
  std::map<uint64_t, uint64_t> free_blocks;   // offset -> bytes

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  void run();
  bool admit();
  void advance(Request& r);
  void launch_pending();
  void end_group(Request& d);
  void finish(Request& r, mlmc_status st);
  uint64_t reservation(const mlmc_config& c) const;
  void chunk(const Request& r, const int64_t* want, int64_t* out) const;
  std::unique_ptr<Slot> acquire(const mlmc_config& c, mlmc_status* st);
  void release(Request& r, bool keep);
  void drop_pool();
  bool arena_alloc(uint64_t bytes, uint64_t* off);
  void arena_free(uint64_t off, uint64_t bytes);
};

namespace {

void destroy_slot(Slot& s) {
  if (s.plan) mlmc_plan_destroy(s.plan);
  if (s.stream) cudaStreamDestroy(s.stream);
  s.plan = nullptr;
  s.stream = nullptr;
}

}  // namespace

// Round workspace a request may hold: its pilot round, capped at an equal
// share of the budget per slot (larger rounds are split into chunks), but
// never below one sample on every level.
uint64_t mlmc_server_s::reservation(const mlmc_config& c) const {
  int64_t cnt[kMaxLevels];
  for (int l = 0; l < c.n_levels; ++l) cnt[l] = cfg.pilot;
  const int64_t pilot_bytes = mlmc_round_bytes(&c, cnt);
  for (int l = 0; l < c.n_levels; ++l) cnt[l] = 1;
  const int64_t one = mlmc_round_bytes(&c, cnt);
  const uint64_t share = cfg.hbm_budget / (uint64_t)cfg.max_slots;
  const uint64_t r = std::max<uint64_t>((uint64_t)one, std::min<uint64_t>((uint64_t)pilot_bytes, share));
  const uint64_t grain = (uint64_t)1 << 20;
  return (r + grain - 1) / grain * grain;
}

bool mlmc_server_s::arena_alloc(uint64_t bytes, uint64_t* off) {
  for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
    if (it->second < bytes) continue;
    *off = it->first;
    const uint64_t rest = it->second - bytes;
    free_blocks.erase(it);
    if (rest) free_blocks[*off + bytes] = rest;
    return true;
  }
  return false;
}

void mlmc_server_s::arena_free(uint64_t off, uint64_t bytes) {
  auto it = free_blocks.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != free_blocks.end() && it->first + it->second == next->first) {
    it->second += next->second;
    free_blocks.erase(next);
  }
  if (it != free_blocks.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      free_blocks.erase(it);
    }
  }
}

// The next round of `want[l]` missing samples per level that fits the
// request's workspace: the level holding most bytes is halved until it fits.
// Samples left out run in the following rounds; the sample index ranges stay
// contiguous, so the result does not depend on the split.
void mlmc_server_s::chunk(const Request& r, const int64_t* want, int64_t* out) const {
  const int L1 = r.cfg.n_levels;
  for (int l = 0; l < L1; ++l) out[l] = std::min<int64_t>(want[l], 65535);
  for (;;) {
    if ((uint64_t)mlmc_round_bytes(&r.cfg, out) <= r.reserve) return;
    int big = -1;
    int64_t big_bytes = -1;
    int64_t one[kMaxLevels];
    for (int l = 0; l < L1; ++l) {
      if (out[l] <= 0) continue;
      for (int k = 0; k < L1; ++k) one[k] = k == l ? out[l] : 0;
      const int64_t b = mlmc_round_bytes(&r.cfg, one);
      if (b > big_bytes) {
        big_bytes = b;
        big = l;
      }
    }
    if (big < 0) return;
    if (out[big] == 1) {
      // one sample per level always fits (reservation); drop to the finest
      // level holding a sample so that some level progresses
      for (int l = 0; l < L1; ++l) out[l] = (l == big) ? 1 : 0;
      return;
    }
    out[big] = (out[big] + 1) / 2;
  }
}

// A plan for configuration `c`: an idle pooled plan of the same shape,
// re-targeted, or a new one with a stream of its own.
std::unique_ptr<Slot> mlmc_server_s::acquire(const mlmc_config& c, mlmc_status* st) {
  auto& idle = pool[shape_of(c)];
  if (!idle.empty()) {
    std::unique_ptr<Slot> s = std::move(idle.back());
    idle.pop_back();
    *st = mlmc_plan_retarget(s->plan, &c);
    if (*st != MLMC_OK) {
      destroy_slot(*s);
      return nullptr;
    }
    return s;
  }
  std::unique_ptr<Slot> s(new Slot());
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    s->stream = nullptr;
    *st = MLMC_ERR_CUDA;
    return nullptr;
  }
  *st = mlmc_plan_create(&c, s->stream, &s->plan);
  if (*st != MLMC_OK) {
    destroy_slot(*s);
    return nullptr;
  }
  return s;
}

void mlmc_server_s::release(Request& r, bool keep) {
  if (!r.slot) return;
  if (keep) pool[shape_of(r.cfg)].push_back(std::move(r.slot));
  else destroy_slot(*r.slot);
  r.slot.reset();
  if (r.reserve) arena_free(r.offset, r.reserve);
  r.reserve = 0;
}

void mlmc_server_s::drop_pool() {
  for (auto& kv : pool)
    for (auto& s : kv.second) destroy_slot(*s);
  pool.clear();
}

void mlmc_server_s::finish(Request& r, mlmc_status st) {
  const int L1 = r.cfg.n_levels;
  if (st == MLMC_OK) {
    double q = 0.0, v = 0.0;
    st = mlmc_estimate(r.slot->plan, &q, &v);
    r.res.q_hat = q;
    r.res.stat_var = v;
    if (st == MLMC_OK && r.bad) st = MLMC_ERR_NOT_CONVERGED;
  }
  double dofs = 0.0;
  for (int l = 0; l < L1; ++l) {
    r.res.N[l] = r.have[l];
    dofs += (double)r.have[l] * mlmc_level_cost(&r.cfg, l);
  }
  r.res.dof_solves = dofs;
  r.res.levels = r.L + 1;
  r.res.status = st;
  r.res.t_done = now();
  // a plan whose last call failed is not reused
  release(r, st == MLMC_OK || st == MLMC_ERR_NOT_CONVERGED);
  r.finished = true;
  {
    std::lock_guard<std::mutex> g(mu);
    results[r.res.id] = r.res;
    ++completed;
  }
  cv_done.notify_all();
}

// Launches the request's next round, or runs its allocation step and then
// the next round, or finishes it: the control flow of mlmc_run.
void mlmc_server_s::advance(Request& r) {
  const int L1 = r.cfg.n_levels;
  for (;;) {
    int64_t want[kMaxLevels];
    bool any = false;
    for (int l = 0; l < L1; ++l) {
      want[l] = std::max<int64_t>(0, r.target[l] - r.have[l]);
      any = any || want[l] > 0;
    }
    if (any) {
      // launched by launch_pending, together with the requests it can share solves with
      chunk(r, want, r.inflight);
      r.pending = true;
      return;
    }
    // every level holds its target: one sampling phase is complete
    ++r.phases;
    if (r.phases >= cfg.max_rounds) {
      finish(r, MLMC_OK);
      return;
    }
    int64_t N[kMaxLevels];
    int32_t Lnew = r.L;
    const mlmc_status st = cfg.adapt_from > 0 ? mlmc_adapt(r.slot->plan, r.L, r.eps, N, &Lnew, nullptr)
                                              : mlmc_allocation(r.slot->plan, r.eps, N);
    if (st != MLMC_OK) {
      finish(r, st);
      return;
    }
    bool more = false;
    for (int l = 0; l <= r.L; ++l)
      if (N[l] > r.target[l]) {
        r.target[l] = N[l];
        more = true;
      }
    if (Lnew > r.L) {
      for (int l = r.L + 1; l <= Lnew; ++l) r.target[l] = cfg.pilot;
      r.L = Lnew;
      more = true;
    }
    if (!more) {
      finish(r, MLMC_OK);
      return;
    }
  }
}

// Launches the rounds that requests want now. Requests whose solves can share
// launches (mlmc_round_bytes_group accepts them together) form groups of up to
// kMaxGroup; a group of two or more whose round workspace fits a free block
// of the arena runs as one group round driven by its first member's plan.
// The others (and groups that do not fit) run their own rounds.
void mlmc_server_s::launch_pending() {
  std::vector<std::vector<Request*>> groups;
  for (auto& a : active) {
    Request& r = *a;
    if (!r.pending || r.finished) continue;
    bool placed = false;
    if (!cfg.solo_rounds) {
      for (auto& g : groups) {
        if ((int)g.size() >= kMaxGroup || g[0]->cfg.n_levels != r.cfg.n_levels) continue;
        const mlmc_config* pair[2] = {&g[0]->cfg, &r.cfg};
        int64_t one[2 * kMaxLevels];
        for (int l = 0; l < 2 * r.cfg.n_levels; ++l) one[l] = 1;
        if (mlmc_round_bytes_group(pair, 2, one) < 0) continue;
        g.push_back(&r);
        placed = true;
        break;
      }
    }
    if (!placed) groups.push_back({&r});
  }
  for (auto& g : groups) {
    const int n = (int)g.size();
    if (n >= 2) {
      const int L1 = g[0]->cfg.n_levels;
      std::vector<const mlmc_config*> cfgs(n);
      std::vector<mlmc_plan> plans(n);
      std::vector<int64_t> first((size_t)n * L1), count((size_t)n * L1);
      for (int k = 0; k < n; ++k) {
        cfgs[k] = &g[k]->cfg;
        plans[k] = g[k]->slot->plan;
        for (int l = 0; l < L1; ++l) {
          first[(size_t)k * L1 + l] = g[k]->have[l];
          count[(size_t)k * L1 + l] = g[k]->inflight[l];
        }
      }
      const int64_t bytes = mlmc_round_bytes_group(cfgs.data(), n, count.data());
      uint64_t off = 0;
      if (bytes > 0 && arena_alloc((uint64_t)bytes, &off)) {
        const mlmc_status st =
            mlmc_round_begin_group(plans.data(), n, first.data(), count.data(), arena + off, (uint64_t)bytes);
        if (st == MLMC_OK) {
          Request* d = g[0];
          d->members = g;
          d->group_off = off;
          d->group_bytes = (uint64_t)bytes;
          for (Request* m : g) {
            m->driver = d;
            m->pending = false;
            ++m->res.rounds;
            ++m->res.group_rounds;
          }
          continue;
        }
        arena_free(off, (uint64_t)bytes);
      }
    }
    for (Request* m : g) {
      m->pending = false;
      const mlmc_status st = mlmc_round_begin(m->slot->plan, m->have, m->inflight);
      if (st != MLMC_OK) {
        finish(*m, st);
        continue;
      }
      ++m->res.rounds;
    }
  }
}

// The group round driven by d has completed: every member takes its samples
// and moves on (its next round, allocation step or end).
void mlmc_server_s::end_group(Request& d) {
  std::vector<Request*> g = d.members;
  std::vector<int32_t> bad(g.size(), 0);
  const mlmc_status st = mlmc_round_end_group(d.slot->plan, bad.data());
  arena_free(d.group_off, d.group_bytes);
  d.members.clear();
  d.group_bytes = 0;
  for (size_t k = 0; k < g.size(); ++k) {
    Request& m = *g[k];
    m.driver = nullptr;
    if (st != MLMC_OK && st != MLMC_ERR_NOT_CONVERGED) {
      finish(m, st);
      continue;
    }
    if (bad[k]) m.bad = true;
    for (int l = 0; l < m.cfg.n_levels; ++l) m.have[l] += m.inflight[l];
    advance(m);
  }
}

// Admits queued requests in arrival order while a slot is free and the
// head's round workspace fits a free block of the arena.
bool mlmc_server_s::admit() {
  bool any = false;
  while (!queue.empty() && (int)active.size() < cfg.max_slots) {
    Request& r = *queue.front();
    const uint64_t bytes = reservation(r.cfg);
    uint64_t off = 0;
    mlmc_status st = MLMC_OK;
    if (bytes > cfg.hbm_budget) st = MLMC_ERR_OOM;   // one sample per level does not fit
    else if (!arena_alloc(bytes, &off)) break;       // wait for a request to finish
    if (st == MLMC_OK) {
      r.cfg.workspace_bytes = bytes;
      r.cfg.use_graphs = 1;
      r.slot = acquire(r.cfg, &st);
      if (!r.slot) arena_free(off, bytes);
    }
    if (st == MLMC_OK) {
      r.reserve = bytes;
      r.offset = off;
      st = mlmc_plan_set_workspace(r.slot->plan, arena + off, bytes);
    }
    if (st == MLMC_OK) st = mlmc_reset_stats(r.slot->plan);
    r.res.t_admit = now();
    std::unique_ptr<Request> owned = std::move(queue.front());
    queue.pop_front();
    any = true;
    if (st != MLMC_OK) {
      finish(*owned, st);
      continue;
    }
    const int Lmax = owned->cfg.n_levels - 1;
    owned->L = cfg.adapt_from > 0 ? std::min(cfg.adapt_from, Lmax) : Lmax;
    for (int l = 0; l <= Lmax; ++l) {
      owned->have[l] = 0;
      owned->target[l] = l <= owned->L ? cfg.pilot : 0;
    }
    advance(*owned);
    if (!owned->finished) active.push_back(std::move(owned));
  }
  return any;
}

void mlmc_server_s::run() {
  cudaSetDevice(cfg.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> g(mu);
      while (!inbox.empty()) {
        queue.push_back(std::move(inbox.front()));
        inbox.pop_front();
      }
      if (stop && active.empty()) break;
    }
    bool progressed = stop ? false : admit();
    for (auto& a : active) {
      Request& r = *a;
      if (r.finished || r.pending) continue;
      if (r.driver && r.driver != &r) continue;   // a group member: its driver is polled
      const int ready = mlmc_round_ready(r.slot->plan);
      if (ready == 0) continue;
      progressed = true;
      if (r.driver == &r) {
        if (ready < 0) {
          for (Request* m : std::vector<Request*>(r.members)) {
            m->driver = nullptr;
            finish(*m, MLMC_ERR_CUDA);
          }
          arena_free(r.group_off, r.group_bytes);
          r.members.clear();
          continue;
        }
        end_group(r);
        continue;
      }
      if (ready < 0) {
        finish(r, MLMC_ERR_CUDA);
        continue;
      }
      const mlmc_status st = mlmc_round_end(r.slot->plan);
      if (st == MLMC_ERR_NOT_CONVERGED) r.bad = true;
      else if (st != MLMC_OK) {
        finish(r, st);
        continue;
      }
      for (int l = 0; l < r.cfg.n_levels; ++l) r.have[l] += r.inflight[l];
      advance(r);
    }
    launch_pending();
    active.erase(std::remove_if(active.begin(), active.end(),
                                [](const std::unique_ptr<Request>& a) { return a->finished; }),
                 active.end());
    if (!progressed) {
      std::unique_lock<std::mutex> g(mu);
      if (inbox.empty() && !stop) {
        if (active.empty()) cv_work.wait(g, [&] { return !inbox.empty() || stop; });
        else cv_work.wait_for(g, std::chrono::microseconds(20));
      }
    }
  }
  // requests never admitted are dropped
  for (auto& q : queue) {
    q->res.status = MLMC_ERR_INVALID;
    q->res.t_done = now();
  }
  queue.clear();
  drop_pool();
}

extern "C" {

mlmc_status mlmc_server_create(const mlmc_server_config* cfg, mlmc_server* out) {
  if (!out) return MLMC_ERR_INVALID;
  *out = nullptr;
  if (!cfg || cfg->max_slots < 1 || cfg->max_slots > 256 || cfg->pilot < 2 || cfg->device < 0 ||
      cfg->max_rounds < 0 || cfg->adapt_from < 0)
    return MLMC_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device >= ndev) {
    cudaGetLastError();
    return MLMC_ERR_CUDA;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) return MLMC_ERR_CUDA;
  mlmc_server s = new mlmc_server_s();
  s->cfg = *cfg;
  if (s->cfg.max_rounds == 0) s->cfg.max_rounds = 64;
  if (s->cfg.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return MLMC_ERR_CUDA;
    }
    s->cfg.hbm_budget = (uint64_t)(0.6 * (double)fr) & ~(uint64_t)((1 << 20) - 1);
  }
  if (cudaMalloc((void**)&s->arena, s->cfg.hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return MLMC_ERR_OOM;
  }
  s->free_blocks[0] = s->cfg.hbm_budget;
  s->t0 = Clock::now();
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return MLMC_OK;
}

mlmc_status mlmc_server_submit(mlmc_server s, const mlmc_config* cfg, double eps, uint64_t* id) {
  if (!s || !cfg || !id || !(eps > 0.0)) return MLMC_ERR_INVALID;
  if (cfg->n_levels < 1 || cfg->n_levels > kMaxLevels) return MLMC_ERR_INVALID;
  int64_t cnt[kMaxLevels];
  for (int l = 0; l < cfg->n_levels; ++l) cnt[l] = 1;
  if (mlmc_round_bytes(cfg, cnt) < 0) return MLMC_ERR_INVALID;
  std::unique_ptr<Request> r(new Request());
  r->cfg = *cfg;
  r->eps = eps;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return MLMC_ERR_INVALID;
    r->res.id = s->next_id++;
    r->res.t_submit = s->now();
    r->res.status = MLMC_OK;
    *id = r->res.id;
    ++s->submitted;
    s->inbox.push_back(std::move(r));
  }
  s->cv_work.notify_one();
  return MLMC_OK;
}

mlmc_status mlmc_server_poll(mlmc_server s, uint64_t id, int* done, mlmc_request_result* out) {
  if (!s || !done) return MLMC_ERR_INVALID;
  std::lock_guard<std::mutex> g(s->mu);
  if (id == 0 || id >= s->next_id) return MLMC_ERR_INVALID;
  auto it = s->results.find(id);
  if (it == s->results.end()) {
    *done = 0;
    return MLMC_OK;
  }
  *done = 1;
  if (out) *out = it->second;
  return MLMC_OK;
}

mlmc_status mlmc_server_drain(mlmc_server s, double timeout_s) {
  if (!s || !(timeout_s >= 0.0)) return MLMC_ERR_INVALID;
  std::unique_lock<std::mutex> g(s->mu);
  const bool ok = s->cv_done.wait_for(g, std::chrono::duration<double>(timeout_s),
                                      [&] { return s->completed == s->submitted; });
  return ok ? MLMC_OK : MLMC_ERR_TIMEOUT;
}

double mlmc_server_clock(mlmc_server s) { return s ? s->now() : -1.0; }

mlmc_status mlmc_server_destroy(mlmc_server s) {
  if (!s) return MLMC_ERR_INVALID;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->cfg.device);
  cudaFree(s->arena);
  delete s;
  return MLMC_OK;
}

}  // extern "C"
