"""The multi-rank sample dispenser (paper_2111_11788_gb300/distributed.py)
on CPU ranks over gloo (world size 2) and in one process.

Checks: the ranges claimed by all ranks are disjoint and cover every
level's missing samples in every phase; both ranks end with the level
states of the single-process run bit for bit (values gathered and folded in
index order), hence the same sample counts; the batches follow Eq. (batch).
The samples are synthetic values keyed by (level, index), the states and
the allocation the oracle's (Welford, Eq. (mlmc_num_samples)).
"""
import json
import os
import socket
import time

import numpy as np
import pytest

from oracle import mlmc as omlmc
from oracle import sched as osched

torch = pytest.importorskip("torch")

L1 = 4
COST = [1.0, 5.0, 25.0, 125.0]


def synthetic(level, i):
    r = np.random.default_rng([7, level, i]).standard_normal(2)
    qf = 1.0 + 0.5 ** level * r[0] + 0.1 * r[1]
    qc = 0.0 if level == 0 else 1.0 + 0.5 ** level * r[0] + 0.1 * 2 * r[1] * 0.5 ** level
    return qf, qc


class Local:
    """Rank-local callables over oracle Welford states."""

    def __init__(self, delay=0.0):
        self.states = [omlmc.Welford() for _ in range(L1)]
        self.delay = delay

    def sample(self, level, first, count):
        if self.delay:
            time.sleep(self.delay)
        vals = [synthetic(level, i) for i in range(first, first + count)]
        return [a for a, _ in vals], [b for _, b in vals]

    def reset(self):
        self.states = [omlmc.Welford() for _ in range(L1)]

    def fold(self, level, qf, qc):
        for a, b in zip(qf, qc):
            self.states[level].add(a - b)

    def allocate(self, eps):
        return omlmc.allocate([s.var() for s in self.states], COST, eps)


class DictStore:
    def __init__(self):
        self.d = {}

    def add(self, key, amount):
        self.d[key] = self.d.get(key, 0) + amount
        return self.d[key]


def single(eps=3e-2, pilot=20):
    from paper_2111_11788_gb300.build import build_library
    build_library()
    from paper_2111_11788_gb300.distributed import RangeDispenser, run_sharded
    loc = Local()
    N, claimed = run_sharded(L1, loc.sample, loc.fold, loc.reset, loc.allocate, lambda o: [o],
                             RangeDispenser(DictStore(), 1), eps=eps, pilot=pilot)
    return N, [(s.n, s.mean, s.m2) for s in loc.states], claimed


def _rank_main(rank, world, port, out_dir, eps, pilot):
    import torch.distributed as dist
    from paper_2111_11788_gb300.distributed import RangeDispenser, run_sharded
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)

    def gather(obj):
        out = [None] * world
        dist.all_gather_object(out, obj)
        return out

    loc = Local(delay=0.002)
    N, claimed = run_sharded(L1, loc.sample, loc.fold, loc.reset, loc.allocate, gather,
                             RangeDispenser(store, world, prefix="t"), eps=eps, pilot=pilot)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"N": N, "states": [(s.n, s.mean, s.m2) for s in loc.states],
                   "claimed": claimed}, f)
    dist.barrier()
    dist.destroy_process_group()


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_single_process_run_matches_a_direct_sequential_run():
    N, states, claimed = single()
    ref = [omlmc.Welford() for _ in range(L1)]
    for l in range(L1):
        for i in range(N[l]):
            a, b = synthetic(l, i)
            ref[l].add(a - b)
    assert states == [(s.n, s.mean, s.m2) for s in ref]
    # one rank: the batches of each phase are exactly Eq. (batch)'s cuts
    phase0 = [(l, f, c) for (ph, l, f, c) in claimed if ph == 0 and l == 0]
    assert [(f, c) for (_, f, c) in phase0] == osched.batches(20, 1)


def test_two_gloo_ranks_share_the_work_and_match_one_process(tmp_path):
    import torch.multiprocessing as mp
    eps, pilot = 3e-2, 20
    port = free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path), eps, pilot), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    N1, states1, _ = single(eps, pilot)
    for r in res:
        assert r["N"] == N1
        assert [tuple(s) for s in r["states"]] == [tuple(s) for s in states1]
    # ranges: disjoint, covering every phase's missing samples of every level
    ranges = [tuple(c) for r in res for c in r["claimed"]]
    by = {}
    for ph, l, f, c in ranges:
        by.setdefault((ph, l), []).append((f, c))
    for key, rs in by.items():
        rs.sort()
        for (f0, c0), (f1, _) in zip(rs, rs[1:]):
            assert f1 == f0 + c0, key
    for l in range(L1):
        covered = sum(c for (ph, ll, f, c) in ranges if ll == l)
        assert covered == N1[l]
    assert all(len(r["claimed"]) > 0 for r in res)


class FakePlan:
    """The plan calls run_rounds makes, over oracle Welford states and the
    synthetic sample values: a round solves its samples (values kept for
    round_values) and folds them, like mlmc_round_begin/end."""

    class _Cfg:
        n_levels = L1

    def __init__(self):
        self.cfg = self._Cfg()
        self.loc = Local()
        self.last = {}
        self.rounds = []

    def round(self, first, count):
        self.rounds.append((list(first), list(count)))
        self.last = {}
        for l in range(L1):
            if count[l]:
                qf, qc = self.loc.sample(l, first[l], count[l])
                self.last[l] = (np.array(qf), np.array(qc))
                self.loc.fold(l, qf, qc)

    def round_values(self, level, count):
        qf, qc = self.last[level]
        assert qf.size == count
        return qf, qc

    def reset_stats(self):
        self.loc.reset()

    def level_fold(self, level, qf, qc=None):
        self.loc.fold(level, qf, np.zeros_like(qf) if qc is None else qc)

    def allocation(self, eps):
        return self.loc.allocate(eps)

    def estimate(self):
        q = sum(s.mean for s in self.loc.states)
        v = sum(s.var() / s.n for s in self.loc.states if s.n)
        return q, v


def _rounds_rank_main(rank, world, port, out_dir, eps, pilot):
    import torch.distributed as dist
    from paper_2111_11788_gb300.distributed import run_rounds, tensor_gather
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    plan = FakePlan()
    N, q, v = run_rounds(plan, rank, world, tensor_gather(dist, "cpu"), eps=eps, pilot=pilot)
    with open(os.path.join(out_dir, "rounds%d.json" % rank), "w") as f:
        json.dump({"N": N, "q": q, "v": v, "rounds": plan.rounds,
                   "states": [(s.n, s.mean, s.m2) for s in plan.loc.states]}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_shares_split_each_level_contiguously():
    from paper_2111_11788_gb300.distributed import shares
    for missing in (0, 1, 5, 64, 101):
        for world in (1, 2, 3, 8):
            sh = shares(missing, world)
            assert len(sh) == world
            assert sh[0][0] == 0
            for (a, n), (b, _) in zip(sh, sh[1:]):
                assert b == a + n
            assert sum(n for _, n in sh) == missing
            assert max(n for _, n in sh) == (-(-missing // world) if missing else 0)


def test_round_sharded_run_over_two_gloo_ranks_matches_one_rank(tmp_path):
    """run_rounds with the tensor all-gather: two CPU ranks (gloo) end with the
    level states, sample counts and estimate of one rank, bit for bit, and
    their rounds cover each phase's missing samples without overlap."""
    import torch.multiprocessing as mp
    from paper_2111_11788_gb300.build import build_library
    build_library()
    from paper_2111_11788_gb300.distributed import run_rounds

    eps, pilot = 3e-2, 20
    one = FakePlan()
    N1, q1, v1 = run_rounds(one, 0, 1, lambda counts, vals: [vals], eps=eps, pilot=pilot)
    # one rank: the same as drawing every level's samples in index order
    ref = [omlmc.Welford() for _ in range(L1)]
    for l in range(L1):
        for i in range(N1[l]):
            a, b = synthetic(l, i)
            ref[l].add(a - b)
    assert [(s.n, s.mean, s.m2) for s in one.loc.states] == [(s.n, s.mean, s.m2) for s in ref]
    port = free_port()
    mp.spawn(_rounds_rank_main, args=(2, port, str(tmp_path), eps, pilot), nprocs=2, join=True)
    res = [json.load(open(tmp_path / ("rounds%d.json" % r))) for r in range(2)]
    for r in res:
        assert r["N"] == N1 and (r["q"], r["v"]) == (q1, v1)
        assert [tuple(s) for s in r["states"]] == [(s.n, s.mean, s.m2) for s in one.loc.states]
    # phase by phase the two ranks' rounds tile each level's new samples
    assert len(res[0]["rounds"]) == len(res[1]["rounds"]) == len(one.rounds)
    for (f0, c0), (f1, c1), (fo, co) in zip(res[0]["rounds"], res[1]["rounds"], one.rounds):
        for l in range(L1):
            assert f0[l] == fo[l] and f1[l] == f0[l] + c0[l] and c0[l] + c1[l] == co[l]
