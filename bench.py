"""Benchmark: MLMC to RMSE eps on the 2D-at-scale workload, one JSON line.

Workload (default): 2D -div(kappa grad u) = 1 on the unit square, Q1 on
32^2..1024^2 elements (6 levels), lognormal KLE field sigma^2 = 1,
correlation length 0.1, M = 64 tensor modes, GMG-preconditioned CG rtol
1e-10, domain-mean QoI, adaptive sample counts for RMSE eps = 1e-3 from 100
pilot samples per level. One step = one whole MLMC run to eps (pilot,
allocation rounds, estimate) through mlmc_run.

Metric: coupled DOF-solves/s = sum over completed coupled samples of the
interior DOFs of both meshes, per second (higher is better); the step time
is the time to RMSE eps.

--impl reference times the CPU FP64 oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import serving_request, serving_stream, workload  # noqa: E402

WORKLOAD = "2d-scale"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-level", type=int, default=None,
                    help="profiling case: only run this level's coupled batch twice, then exit")
    ap.add_argument("--profile-batch", type=int, default=64)
    ap.add_argument("--stencil-tile", type=int, default=None,
                    help="profile case: 3D FP32 stencil tile shape (mlmc_config.stencil_tile)")
    ap.add_argument("--profile-kle", action="store_true",
                    help="profiling case: the KLE contraction of the finest level's batch "
                         "(--profile-batch samples), FP64 and tensor-core kernels, twice each")
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed"],
                    help="form of the headline line (the other form is measured alongside)")
    ap.add_argument("--single-form", action="store_true")
    ap.add_argument("--serve", type=float, default=5.0,
                    help="also run the serving stream for this many seconds of Poisson arrivals "
                         "(0: skip)")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=24)
    ap.add_argument("--serve-pilot", type=int, default=32)
    ap.add_argument("--serve-adapt", type=int, default=2,
                    help="requests start on levels 0..K and adapt L (0: all levels, L fixed)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the autotuner (by default inner tolerance, MG damping and the 3D "
                         "z-chunk are tuned on the finest level before the warm-up, outside the "
                         "timed region)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="host-driven solver loops (same kernels; ncu cannot profile kernels "
                         "inside graphs with conditional nodes)")
    return ap.parse_args()


def interior_dofs(dim, n):
    return (n - 1) ** dim


def coupled_dofs(wl, level):
    n = wl["n0"] << level
    d = interior_dofs(wl["dim"], n)
    if level > 0:
        d += interior_dofs(wl["dim"], n // 2)
    return d


def workload_desc(wl):
    nf = wl["n0"] << (wl["levels"] - 1)
    if wl.get("N") is not None:
        tail = "fixed N=%s" % (list(wl["N"]),)
    else:
        tail = "eps=%g, pilot %d" % (wl["eps"], wl["pilot"])
    return ("%dD Q1 %d^%d..%d^%d elements (%d levels), sigma2=%g, corr_len=%g, M=%d, %s-PCG "
            "rtol %g, %s QoI, %s" % (
                wl["dim"], wl["n0"], wl["dim"], nf, wl["dim"], wl["levels"], wl["sigma2"],
                wl["corr_len"], wl["m"] ** wl["dim"], wl["solver"].upper(), wl["rtol"],
                wl["qoi"], tail))


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle
#
# The oracle runs in a pool of spawned worker processes (never forked after
# the first CUDA call), each with single-threaded BLAS. A task is one coupled
# sample (level, i): the worker returns (Q_l, Q_{l-1}, its own elapsed time).

_ORACLE_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_task(args):
    name, level, i = args
    sys.path.insert(0, ROOT)
    from oracle import mlmc as omlmc
    from synth import workload as wlf
    t = time.perf_counter()
    qf, qc = omlmc.coupled_sample(wlf(name), level, i)
    return level, i, qf, qc, time.perf_counter() - t


class OraclePool:
    """nproc single-threaded oracle workers (spawn start method)."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or (os.cpu_count() or 1)
        for k, v in _ORACLE_ENV.items():
            os.environ.setdefault(k, v)
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_noop, range(self.procs))      # workers up and importable

    def run(self, tasks):
        t = time.perf_counter()
        out = self.pool.map(_oracle_task, tasks, chunksize=1)
        return out, time.perf_counter() - t

    def close(self):
        self.pool.close()
        self.pool.join()


def _noop(_):
    sys.path.insert(0, ROOT)
    import oracle.mlmc  # noqa: F401
    return os.getpid()


def cpu_baseline(name, N, pool):
    """The oracle on the host cores, reported beside the GPU number.

    single thread: one coupled sample (sample 0) of every level, each in its
    own worker at the same time (one core each), giving the per-sample time
    t_l; all cores: nproc coupled samples of one level at once, giving the
    speed-up S of the host over one core. Both are extrapolated to the GPU
    run's sample counts N_l: time to eps T1 = sum N_l t_l single-threaded and
    T1 / S on all cores. Returns (line, oracle values of sample 0 per level)."""
    wl = workload(name)
    L = wl["levels"]
    res, _ = pool.run([(name, l, 0) for l in range(L)])
    t1 = {l: dt for l, _, _, _, dt in res}
    ref = {l: (qf, qc) for l, _, qf, qc, _ in res}
    la = min(4, L - 1)
    par, wall = pool.run([(name, la, 1 + k) for k in range(pool.procs)])
    speedup = pool.procs * t1[la] / wall
    T1 = sum(N[l] * t1[l] for l in range(L))
    dofs = sum(N[l] * coupled_dofs(wl, l) for l in range(L))
    line = {"value": dofs / (T1 / speedup), "unit": "coupled DOF-solves/s", "cores": pool.procs,
            "kind": "oracle", "nproc": os.cpu_count(), "extrapolated": True,
            "time_to_eps_s": T1 / speedup,
            "single_thread": {"value": dofs / T1, "cores": 1, "time_to_eps_s": T1},
            "per_sample_s": [round(t1[l], 3) for l in range(L)],
            "all_core_speedup": round(speedup, 2),
            "sample": ("measured: one coupled sample (sample 0) of each of levels 0..%d of the %s "
                       "workload, single-threaded, one worker per level; %d coupled samples of "
                       "level %d on %d workers at once (%.1f s wall); extrapolated to the GPU run's "
                       "N = %s. Oracle: dense KLE, assembled Q1 matrix, sparse LU (or Jacobi-PCG "
                       "to 1e-13 above its size limit)" % (L - 1, name, pool.procs, la, pool.procs,
                                                          wall, list(N)))}
    return line, ref


def result_errors(m, wl, cfg, stream, ref):
    """Per-result relative error of one GPU form against the oracle: Q_l and
    Q_{l-1} of sample 0 of every level (a fresh plan, one coupled sample per
    call)."""
    import torch
    per, worst = [], 0.0
    with torch.cuda.stream(stream):
        with m.Plan(cfg, stream.cuda_stream) as plan:
            for l in sorted(ref):
                qf, qc, _ = plan.sample_level(l, 0, 1)
                rf, rc = ref[l]
                ef = abs(float(qf[0]) - rf) / abs(rf)
                per.append([l, "fine", ef])
                worst = max(worst, ef)
                if l > 0:
                    ec = abs(float(qc[0]) - rc) / abs(rc)
                    per.append([l, "coarse", ec])
                    worst = max(worst, ec)
    return {"max_rel": worst, "per_result": per,
            "sample": "Q_l and Q_(l-1) of sample 0 of levels %s against the FP64 oracle"
                      % sorted(ref)}


def bench_reference(args):
    """The oracle as the reference arm: each step runs nproc coupled samples
    at once on the host cores (levels 0..min(4, L-1) in turn, one per
    worker); value = coupled DOFs of the step / its wall time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload)
    levels = list(range(min(wl["levels"], 5)))
    pool = OraclePool()
    try:
        def tasks(step):
            return [(args.workload, levels[k % len(levels)], 1000 * step + k) for k in range(pool.procs)]
        for w in range(min(args.warmup, 2)):
            pool.run(tasks(10 ** 4 + w))
        t_dofs, t_sec = 0, 0.0
        for st in range(args.steps):
            out, wall = pool.run(tasks(st))
            t_dofs += sum(coupled_dofs(wl, l) for l, _, _, _, _ in out)
            t_sec += wall
    finally:
        pool.close()
    value = t_dofs / t_sec
    line = {"impl": "reference", "metric": "coupled DOF-solves/s", "value": value,
            "unit": "coupled DOF-solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload + ": " + workload_desc(wl),
                       "sample": "per step %d coupled samples on %d workers, levels %s in turn"
                                 % (pool.procs, pool.procs, levels)},
            "cpu_baseline": {"value": value, "unit": "coupled DOF-solves/s", "cores": pool.procs,
                             "kind": "oracle",
                             "sample": "per step one coupled sample per host core, levels %s in "
                                       "turn (levels above 4 are left out to bound the step)"
                                       % levels},
            "e2e": {"value": value, "unit": "coupled DOF-solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU

def tuned_config(m, cfg, tune):
    """The tuned settings are configuration fields: a user's plan takes them directly."""
    cfg2 = m.Config.from_buffer_copy(cfg)
    if tune is not None:
        cfg2.inner_rtol, cfg2.mg_omega, cfg2.z_chunk = (tune["inner_rtol"], tune["mg_omega"],
                                                        tune["z_chunk"])
        cfg2.stencil_tile, cfg2.batch_split = tune["stencil_tile"], tune["batch_split"]
    return cfg2


def mlmc_step(plan, wl, rank, world, gather):
    """One MLMC estimate: mlmc_run on one GPU; on several, the same estimate
    with each phase's samples split over the ranks (distributed.run_rounds)."""
    fixed = list(wl["N"]) if wl.get("N") is not None else None
    if world == 1:
        if fixed is not None:
            return plan.run(N=fixed)
        return plan.run(eps=wl["eps"], pilot=wl["pilot"])
    from paper_2111_11788_gb300.distributed import run_rounds
    N, q, v = run_rounds(plan, rank, world, gather, eps=wl.get("eps"), pilot=wl.get("pilot", 0),
                         N_fixed=fixed)
    return q, v, N


def measure_form(m, wl, cfg, stream, args, world, barrier, with_e2e, rank=0, gather=None):
    """Warm up, trace one run, then time args.steps MLMC runs of one form."""
    import torch
    sh = stream.cuda_stream
    with torch.cuda.stream(stream):
        tune = None
        if args.autotune:
            # tuned on rank 0 and shared, so that every rank solves with the same settings
            if rank == 0:
                with m.Plan(cfg, sh) as tp:
                    # solver knobs on the finest level, then the tile shape and the
                    # batch split on a round over every level (from the tuned settings)
                    cnt = 32 if wl["dim"] == 2 else 16
                    tune = tp.autotune(wl["levels"] - 1, cnt, 7)
                    t2 = tp.autotune(wl["levels"] - 1, cnt, 8 | 16)
                    tune.update(stencil_tile=t2["stencil_tile"], batch_split=t2["batch_split"],
                                candidates=tune["candidates"] + t2["candidates"],
                                round_best_ms=t2["best_ms"], round_worst_ms=t2["worst_ms"])
            if world > 1:
                import torch.distributed as dist
                box = [tune]
                dist.broadcast_object_list(box, src=0)
                tune = box[0]
        cfg = tuned_config(m, cfg, tune)
        plan = m.Plan(cfg, sh)
        N = None
        def one_run():
            return mlmc_step(plan, wl, rank, world, gather)
        for _ in range(max(args.warmup, 1)):
            q, v, N = one_run()
        dofs_step = sum(int(N[l]) * coupled_dofs(wl, l) for l in range(wl["levels"]))
        # pick the dominant kernel from a traced run
        plan.profile(-1)
        plan.profile_reset()
        one_run()
        stats = plan.kernel_stats()
        plan.profile(0)
        total_ms = sum(st[1] for st in stats.values())
        dom = max(stats, key=lambda k: stats[k][1])
        shares = {k: round(st[1] / total_ms, 4) for k, st in stats.items() if st[1] > 0}
        # per kernel: launches, traced time, algorithmic GB/s (event-timed launch by launch)
        per_kernel = {k: {"launches": int(st[0]), "ms": round(st[1], 3),
                          "gbs": round(st[2] / (st[1] / 1e3) / 1e9, 1) if st[1] > 0 and st[2] > 0 else None}
                      for k, st in stats.items() if st[1] > 0}
        # timed region: device events around whole MLMC runs (solves run as CUDA graphs)
        clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        l0 = plan.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            q, v, N = one_run()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        launches = plan.launch_count() - l0
        ms = ev0.elapsed_time(ev1)
        # the dominant kernel, timed launch by launch with CUDA events on the plan's
        # stream, over a repeat of the same step (host-driven launches of the same kernels)
        plan.profile_reset()
        plan.profile(1 << m.Plan.kernel_id(dom))
        one_run()
        dstat = plan.kernel_stats()[dom]
        plan.profile(0)
        wall = []
        if with_e2e:
            # end to end through the public API: plan creation (host KLE roots,
            # table upload), the run, results back to host, plan destruction
            for _ in range(args.steps):
                barrier()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                p2 = m.Plan(cfg, sh)
                mlmc_step(p2, wl, rank, world, gather)
                p2.close()
                torch.cuda.synchronize()
                wall.append(time.perf_counter() - t0)
        plan.close()
    return dict(ms=ms, N=[int(x) for x in N], dofs_step=dofs_step, q=q, v=v, dom=dom, tune=tune,
                dstat=dstat, shares=shares, per_kernel=per_kernel, clocks=clk, launches=launches,
                wall=wall)


def serving_both(m, args, device=0):
    """The serving stream with adaptive levels (headline) and with every level
    of the ranges sampled (L fixed)."""
    res = serving_run(m, args, device, args.serve_adapt)
    if args.serve_adapt > 0:
        fixed = serving_run(m, args, device, 0)
        keep = ("p50_time_to_eps_s", "p99_time_to_eps_s", "mean_time_to_eps_s",
                "aggregate_dof_solves_per_s", "span_s", "max_in_flight", "failed", "failed_requests",
                "rounds", "group_rounds")
        res["fixed_levels"] = {k: fixed[k] for k in keep}
    return res


def serving_run(m, args, device=0, adapt=0):
    """The serving stream: Poisson arrivals submitted at their arrival times to
    one server; returns latency percentiles and aggregate throughput."""
    import numpy as np
    import torch
    n_req = max(1, int(round(args.serve * args.serve_rate)))
    stream = serving_stream(n_req, rate=args.serve_rate, seed=1)
    srv = m.Server(max_slots=args.serve_slots, pilot=args.serve_pilot, device=device,
                   adapt_from=adapt)
    try:
        # warm-up: every plan shape the stream can ask for, a slot's worth each
        warm = []
        for dim, modes in ((2, (5, 6, 7, 8)), (3, (5, 6, 7))):
            for mm in modes:
                for j in range(3):
                    wl = serving_request(dim, 1.0, 1.5 / (mm - 0.5), 10 ** 6 + len(warm))
                    warm.append(srv.submit(m.config_from_workload(wl), 5e-3))
        srv.drain(timeout=900.0)
        clocks = ClockSampler(device)
        torch.cuda.synchronize()
        clocks.start()
        t0 = srv.clock()
        ids = []
        for (ta, wl, eps) in stream:
            delay = t0 + ta - srv.clock()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(m.config_from_workload(wl), eps))
        srv.drain(timeout=3600.0)
        clk = clocks.stop()
        res = [srv.poll(i) for i in ids]
    finally:
        srv.close()
    bad = [r for r in res if r["status"] not in (0,)]
    bad_info = [dict(status=r["status"], dim=wl["dim"], sigma2=round(wl["sigma2"], 3),
                     corr_len=round(wl["corr_len"], 3), m=wl["m"], eps=round(eps, 6), N=r["N"][:wl["levels"]])
                for (ta, wl, eps), r in zip(stream, res) if r["status"] != 0]
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    wait = np.array([r["t_admit"] - r["t_submit"] for r in res])
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    dofs = sum(r["dof_solves"] for r in res)
    by_dim = {}
    for (ta, wl, eps), r in zip(stream, res):
        by_dim.setdefault(wl["dim"], []).append(r["t_done"] - r["t_submit"])
    # most requests in flight at once
    ev = sorted([(r["t_admit"], 1) for r in res] + [(r["t_done"], -1) for r in res])
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    return {"requests": n_req, "rate_per_s": args.serve_rate, "arrival_seed": 1,
            "slots": args.serve_slots, "pilot": args.serve_pilot, "failed": len(bad),
            "failed_requests": bad_info,
            "levels": ("adaptive from levels 0..%d (Eq. mlmc_num_levels)" % adapt
                       if adapt > 0 else "all levels of the range"),
            "levels_used_hist": {str(k): sum(1 for r in res if r["levels"] == k)
                                 for k in sorted(set(r["levels"] for r in res))},
            "p50_time_to_eps_s": float(np.percentile(lat, 50)),
            "p99_time_to_eps_s": float(np.percentile(lat, 99)),
            "mean_time_to_eps_s": float(lat.mean()),
            "p50_by_dim_s": {str(d): float(np.percentile(v, 50)) for d, v in sorted(by_dim.items())},
            "p99_admission_wait_s": float(np.percentile(wait, 99)),
            "aggregate_dof_solves_per_s": dofs / span, "span_s": span,
            "max_in_flight": peak, "rounds": int(sum(r["rounds"] for r in res)),
            "group_rounds": int(sum(r["group_rounds"] for r in res)),
            "clocks": clk,
            "mix": "eps~U[5e-4,5e-3], dim 2|3 (p=1/2), sigma2~U[0.5,2], corr_len~U[0.05,0.3]; "
                   "2D 32^2..1024^2 domain-mean QoI, 3D 8^3..128^3 box QoI; m=ceil(1.5/corr_len) "
                   "capped 8 (2D) / 7 (3D); GMG-PCG rtol 1e-10, FP32 inner + FP64 refinement"}


# FP64 work of the FP64 stencil kernels per output node, counted off the
# kernels as built (the halo lanes and rows a strip or tile also computes are
# not counted: they show up as lost efficiency), with the algorithmic bytes
# per node that the byte counters use (nn ~ ne, nc ~ nn / 2^d).
# 2D (coefficient form): the operator is 1 multiply + 8 FMAs, or 9 FMAs when
# a residual f - A x is accumulated from f; mg_post adds the streamed
# prolongation (1 add on every other row for the coarse row sums, 1 add on
# odd rows, 1 FMA), the smoothing FMA and the dot (13 instructions, 25
# flops); mg_pre the W b multiply and the residual stencil (10, 19); pcg_pq
# the direction FMA, the stencil and the dot (11, 21); resid64 the residual
# stencil and its square (10, 20).
# 3D (element-sum z-march on precomputed kappa sums, k_zm3q): per element
# position 3 adds (plane sum of its 4 nodes), 1 add and 1 multiply (Q =
# kappa S); per node 1.5 adds (x pairs of Q, shared by the two rows of a
# thread) + 1 add (2 x 2 sum of Q) + 1 multiply and 5 FMAs (six face
# neighbours) + 1 multiply and 1 FMA (5 u K_n) + 2 adds (minus the two
# layers' sums): 17.5 instructions, 23.5 flops for the operator. Loaders and
# epilogues: A p: z + beta p (1 FMA), q = h/12 t (1 multiply), p.q (1 FMA);
# pre-smoother: W b (1 multiply), b - h/12 t (1 FMA); post-smoother: b -
# h/12 t, e + W r and b.out (3 FMAs); residual: f - h/12 t and r.r (2 FMAs).
# The 4 kappa-sum arrays, read per node, are precomputed once per solve and,
# like the 2D coefficient arrays, not in the algorithmic bytes.
#   (instructions per node, flops per node, bytes per node)
FP64_WORK = {
    (2, "mg_post"): (13.0, 25.0, 42.0), (2, "mg_pre"): (10.0, 19.0, 40.0),
    (2, "pcg_pq"): (11.0, 21.0, 40.0), (2, "resid64"): (10.0, 20.0, 24.0),
    (3, "mg_post"): (20.5, 29.5, 41.0), (3, "mg_pre"): (19.5, 26.5, 40.0),
    (3, "pcg_pq"): (20.5, 28.5, 40.0), (3, "resid64"): (19.5, 27.5, 24.0),
}
# DRAM bytes per output node measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch whose arrays exceed L2), for the
# dominant kernels whose capture matches the kernel as built; a launch's
# traffic is scaled from it by the nodes the launch processes (its
# algorithmic bytes / the per-node byte model).
#   (dim, kernel, fp64 form?): (DRAM bytes per node, capture)
DRAM_PER_NODE = {
    (2, "mg_post", True): ((498.484224e6 + 59.262976e6) / (513 * 513 * 32),
                           "ncu, k_mgpost2<double, 1>, 512^2 elements x 32 samples"),
}

GB300_SMS = 152
DFMA_PER_SM_CLK = 2


def roofline_of(res, peaks, fp64_alu, dim=2, fp64_probe=None):
    d_launches, d_ms, d_bytes = res["dstat"]
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    gbs = (d_bytes / (d_ms / 1e3)) / 1e9 if d_ms > 0 else 0.0
    r = {"kernel": res["dom"], "traffic": None, "launches": d_launches,
         "avg_launch_us": round(1e3 * d_ms / max(d_launches, 1), 2),
         "time_shares": res["shares"], "per_kernel": res["per_kernel"]}
    work = FP64_WORK.get((dim, res["dom"]))
    dram = DRAM_PER_NODE.get((dim, res["dom"], bool(fp64_alu)))
    if dram is not None and work is not None and d_launches > 0:
        nodes_per_launch = d_bytes / work[2] / d_launches
        r["traffic"] = round(nodes_per_launch * dram[0])
        r["traffic_source"] = ("%s: %.1f B/node (algorithmic %.0f), scaled to the average launch "
                               "(%.3g nodes)" % (dram[1], dram[0], work[2], nodes_per_launch))
    # the FP64 kernels (every stencil of the FP64 form; the outer residual of
    # the mixed form) are bound by the FP64 pipe
    if (fp64_alu or res["dom"] == "resid64") and work is not None:
        # FP64-pipe bound: algorithmic FP64 flops/s (FMA = 2) against 2 DFMA per
        # SM per cycle at the median SM clock of the timed region; the same as
        # FP64 instructions/s against the pipe's 2 instructions per SM per cycle
        ins, flops, nbytes = work
        mhz = (res.get("clocks") or {}).get("sm_mhz") or 2070.0
        derived = DFMA_PER_SM_CLK * 2 * GB300_SMS * mhz * 1e6 / 1e12
        achieved = gbs * flops / nbytes / 1e3
        ipeak = DFMA_PER_SM_CLK * GB300_SMS * mhz * 1e6 / 1e12
        iach = gbs * ins / nbytes / 1e3
        if fp64_probe:
            peak = fp64_probe["tflops"]
            psrc = ("measured: FP64 FMA-chain probe (mlmc_probe_fp64_rate, %.3f ms per launch) run "
                    "by this bench before the timed region; derived %d SMs x %d DFMA/cycle x 2 "
                    "flops x %.0f MHz = %.4f TFLOP/s" % (fp64_probe["ms"], GB300_SMS,
                                                         DFMA_PER_SM_CLK, mhz, derived))
        else:
            peak = derived
            psrc = ("derived: %d SMs x %d DFMA/cycle x 2 flops x %.0f MHz (median under load)"
                    % (GB300_SMS, DFMA_PER_SM_CLK, mhz))
        r.update({"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4),
                  "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "peak_source": psrc,
                  "fp64_instructions": {"achieved": round(iach, 4), "peak": round(ipeak, 4),
                                        "unit": "T instr/s", "frac": round(iach / ipeak, 4)},
                  # the same launches against HBM, in algorithmic bytes
                  "hbm": {"achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                          "frac": round(gbs / hbm_peak, 4), "peak_source": src,
                          "bytes_per_node": nbytes}})
    else:
        r.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                  "frac": round(gbs / hbm_peak, 4), "peak_source": src})
    return r


def kle_compare(m, wl, stream, peaks, batch=None, reps=10):
    """The KLE contraction of one coupled batch of the finest mesh: the FP64
    sum-factorised kernel (mlmc_kappa, the kappa of the FP64 residual) and the
    tensor-core kernel (mlmc_kappa32, split BF16 on tcgen05, the FP32 kappa of
    the inner solves), each timed with CUDA events on the plan's stream.
    Tensor roofline: the dense contraction's flops 2 ne M B and the flops the
    MMAs issue (three BF16 products on tiles padded to 128 elements x 64
    modes x 16 samples) against the measured BF16 peak."""
    import torch
    L = wl["levels"] - 1
    n = wl["n0"] << L
    d = wl["dim"]
    B = batch or (100 if d == 2 else 16)
    cfg = m.config_from_workload(wl, precision="mixed")
    M = m.coef_count(cfg)
    ne = n ** d
    es = m.elem_stride(d, n)
    res = {"mesh": "%d^%d" % (n, d), "samples": B, "modes": M}
    with torch.cuda.stream(stream):
        with m.Plan(cfg, stream.cuda_stream) as plan:
            xi = torch.zeros(B * M, dtype=torch.float64, device="cuda")
            plan.draw_xi(L, 0, B, xi.data_ptr())
            k64 = torch.empty(B * es, dtype=torch.float64, device="cuda")
            k32 = torch.empty(B * es, dtype=torch.float32, device="cuda")
            for name, fn in (("fp64_sum_factorised",
                              lambda: plan.kappa(L, xi.data_ptr(), B, k64.data_ptr())),
                             ("tensor_cores_split_bf16",
                              lambda: plan.kappa32(L, xi.data_ptr(), B, k32.data_ptr()))):
                fn()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    fn()
                e1.record(stream)
                torch.cuda.synchronize()
                res[name] = {"ms": e0.elapsed_time(e1) / reps}
    dense = 2.0 * ne * M * B
    issued = 3 * 2.0 * ((ne + 127) // 128 * 128) * ((M + 63) // 64 * 64) * ((min(B, 256) + 15) // 16 * 16) \
        * ((B + 255) // 256)
    t = res["tensor_cores_split_bf16"]["ms"] / 1e3
    peak = peaks.get("bf16_tflops")
    tens = {"bound": "tensor", "achieved": round(issued / t / 1e12, 2), "unit": "TFLOP/s",
            "dense_contraction_tflops": round(dense / t / 1e12, 2),
            "peak": peak, "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops)" if peak else None,
            "frac": round(issued / t / 1e12 / peak, 4) if peak else None,
            "kappa32_write_gbs": round(4.0 * ne * B / t / 1e9, 1)}
    res["tensor_roofline"] = tens
    res["faster"] = min(("fp64_sum_factorised", "tensor_cores_split_bf16"), key=lambda k: res[k]["ms"])
    return res


def bench_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as m

    def barrier():
        if world > 1:
            dist.barrier()

    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": serving_both(m, args, local)}), flush=True)
        return
    wl = workload(args.workload)
    stream = torch.cuda.Stream()
    # the FP64 peak of this device, measured (the FP64 form is bound by it)
    tf, pms = m.probe_fp64_rate(stream.cuda_stream)
    fp64_probe = {"tflops": tf, "ms": pms}
    # several GPUs share one MLMC estimate: every phase's samples are split
    # over the ranks and their values all-gathered (NCCL) and folded in order
    gather = None
    if world > 1:
        from paper_2111_11788_gb300.distributed import tensor_gather
        gather = tensor_gather(dist, "cuda")
    forms = {}
    for form in (args.form, "mixed" if args.form == "fp64" else "fp64"):
        if form != args.form and args.single_form:
            continue
        cfg = m.config_from_workload(wl, precision=form)
        forms[form] = measure_form(m, wl, cfg, stream, args, world, barrier,
                                   with_e2e=(form == args.form), rank=rank, gather=gather)

    def reduce_max(x):
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    # the mixed form with its FP32 kappa from the tensor cores (kle_tensor = 1)
    kle_tc = None
    if not args.single_form and "mixed" in forms:
        cfg = m.config_from_workload(wl, precision="mixed", kle_tensor=1)
        kle_tc = measure_form(m, wl, cfg, stream, args, world, barrier, with_e2e=False, rank=rank,
                              gather=gather)
    main = forms[args.form]
    ms = reduce_max(main["ms"])
    e2e_s = reduce_max(sum(main["wall"]))
    # one estimate per step whatever the number of GPUs (strong scaling)
    value = main["dofs_step"] * args.steps / (ms / 1e3)
    e2e_value = main["dofs_step"] * args.steps / e2e_s
    h2d = 8 * 2 * wl["m"] + 4 * wl["m"] + 8 * wl["levels"]
    d2h = 8 * 2 + 8 * wl["levels"]
    other = {}
    for form, res in forms.items():
        if form == args.form:
            continue
        oms = reduce_max(res["ms"])
        other[form] = {"value": res["dofs_step"] * args.steps / (oms / 1e3),
                       "unit": "coupled DOF-solves/s", "ms_per_step": oms / args.steps,
                       "time_to_eps_s": oms / args.steps / 1e3,
                       "samples_per_level": res["N"], "q_hat": res["q"], "stat_var": res["v"],
                       "gpu_launches": int(res["launches"]), "clocks": res["clocks"],
                       "autotune": res["tune"],
                       "roofline": roofline_of(res, peaks, fp64_alu=(form == "fp64"), dim=wl["dim"],
                                               fp64_probe=fp64_probe)}
    if kle_tc is not None:
        oms = reduce_max(kle_tc["ms"])
        other["mixed+kle_tensor"] = {
            "value": kle_tc["dofs_step"] * args.steps / (oms / 1e3), "unit": "coupled DOF-solves/s",
            "ms_per_step": oms / args.steps, "samples_per_level": kle_tc["N"],
            "q_hat": kle_tc["q"], "stat_var": kle_tc["v"], "gpu_launches": int(kle_tc["launches"]),
            "kappa_share": kle_tc["shares"].get("kappa"), "autotune": kle_tc["tune"]}
    if rank == 0:
        names = {"fp64": "plain FP64", "mixed": "mixed: FP32 inner PCG + FP64 refinement",
                 "mixed+kle_tensor": "mixed, FP32 kappa from the tensor-core KLE"}
        line = {"metric": "coupled DOF-solves/s", "value": value, "unit": "coupled DOF-solves/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "time_to_eps_s": ms / args.steps / 1e3,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64" if args.form == "fp64" else "f32+f64", "data": "synthetic",
                "config": {"workload": args.workload + ": " + workload_desc(wl),
                           "form": names[args.form],
                           "samples_per_level": main["N"],
                           "q_hat": main["q"], "stat_var": main["v"],
                           "l2": "working set of the 512^2/1024^2 levels (GBs) exceeds the 129 MB L2",
                           "parallelism": ("one estimate over %d GPUs: each phase's samples "
                                           "split by Eq. (batch), values all-gathered (NCCL) "
                                           "and folded in index order" % world)
                                          if world > 1 else "single GPU"},
                "roofline": roofline_of(main, peaks, fp64_alu=(args.form == "fp64"), dim=wl["dim"],
                                        fp64_probe=fp64_probe),
                "clocks": main["clocks"], "gpu_launches": int(main["launches"]),
                "autotune": main["tune"],
                "e2e": {"value": e2e_value, "unit": "coupled DOF-solves/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "other_forms": {names[k]: v for k, v in other.items()}}
        line["kle"] = kle_compare(m, wl, stream, peaks)
        if args.serve > 0:
            line["serving"] = serving_both(m, args, local)
        if not args.no_cpu_baseline:
            pool = OraclePool()
            try:
                line["cpu_baseline"], ref = cpu_baseline(args.workload, main["N"], pool)
            finally:
                pool.close()
            # error of every form against the oracle, result by result
            for form in forms:
                cfgf = m.config_from_workload(wl, precision=form)
                err = result_errors(m, wl, cfgf, stream, ref)
                if form == args.form:
                    line["error_vs_oracle"] = err
                else:
                    line["other_forms"][names[form]]["error_vs_oracle"] = err
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def profile_case(args):
    """Small case for ncu: one level's coupled batch, twice, no timing."""
    import torch
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as m
    wl = workload(args.workload)
    cfg = m.config_from_workload(wl, precision=args.form, use_graphs=0 if args.no_graphs else 1,
                                 stencil_tile=args.stencil_tile)
    with m.Plan(cfg, torch.cuda.current_stream().cuda_stream) as plan:
        for rep in range(2):
            plan.sample_level(args.profile_level, rep * args.profile_batch, args.profile_batch,
                              want=False)
    torch.cuda.synchronize()
    print("profile case done: level %d, batch %d" % (args.profile_level, args.profile_batch))


def profile_kle(args):
    """Small case for ncu: the two KLE kernels on one batch of the finest mesh."""
    import torch
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as m
    wl = workload(args.workload)
    L = wl["levels"] - 1
    n = wl["n0"] << L
    B = args.profile_batch
    cfg = m.config_from_workload(wl, precision="mixed")
    M = m.coef_count(cfg)
    es = m.elem_stride(wl["dim"], n)
    with m.Plan(cfg, torch.cuda.current_stream().cuda_stream) as plan:
        xi = torch.zeros(B * M, dtype=torch.float64, device="cuda")
        plan.draw_xi(L, 0, B, xi.data_ptr())
        k64 = torch.empty(B * es, dtype=torch.float64, device="cuda")
        k32 = torch.empty(B * es, dtype=torch.float32, device="cuda")
        for _ in range(2):
            plan.kappa(L, xi.data_ptr(), B, k64.data_ptr())
            plan.kappa32(L, xi.data_ptr(), B, k32.data_ptr())
    torch.cuda.synchronize()
    print("profile case done: KLE of %d samples on %d^%d" % (B, n, wl["dim"]))


def main():
    args = parse()
    if args.profile_kle:
        profile_kle(args)
    elif args.profile_level is not None:
        profile_case(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
