"""Scheduling: Eq. (batch) and Algorithm 1 (host code, no GPU).

Oracle pins (oracle/sched.py): the batch rule cuts [0, N) into contiguous
ranges within its bounds; Algorithm 1 meets Theorem 3.1 (no idling before
the last start, makespan <= W_bar + max task <= 2 W_LB) on random divisible
instances, reaches the tight ratio 2p / (p + 1) on the text's example of p^2
unit tasks followed by one of length p, and stays within twice a brute-force
optimum; the "Pause" model shows the benefit of batching when dispatches
cost time (Sec. 5.1). Parity: the library's mlmc_batch_size and
mlmc_schedule_greedy equal the oracle exactly (integers and the same
floating-point sums in the same order).
"""
import random

import numpy as np
import pytest

from oracle import sched as osched


# ------------------------------------------------------------ oracle pins

@pytest.mark.parametrize("N,parts", [(1, 1), (7, 3), (100, 4), (1024, 16), (4096, 600), (65, 64),
                                     (100000, 7)])
def test_batches_partition_the_level(N, parts):
    bs = osched.batches(N, parts)
    assert bs[0][0] == 0
    for (f0, c0), (f1, _) in zip(bs, bs[1:]):
        assert f1 == f0 + c0
    assert sum(c for _, c in bs) == N
    share = -(-N // parts)
    lo = max(1, int(np.ceil(0.01 * share)))
    hi = max(1, int(np.floor(osched.PHI_INV * share)))
    sizes = [c for _, c in bs]
    assert all(lo <= c <= hi for c in sizes[:-1])
    assert sizes[-1] <= hi
    # guided: sizes never grow
    assert all(a >= b for a, b in zip(sizes, sizes[1:]))
    # the first batch is the 1/phi cap of the share once N is large
    if N >= 10 * parts:
        assert sizes[0] == hi


def test_batch_follows_unassigned_share():
    N, parts = 10000, 10
    prev = None
    for n in range(0, N, 500):
        b = osched.batch_size(N, n, parts)
        expect = min(max(-(-(N - n) // parts), 10), 618)
        assert b == expect
        if prev is not None:
            assert b <= prev
        prev = b


def random_instance(rng, levels=3, p_groups=4):
    q = [1]
    for _ in range(levels - 1):
        q.append(q[-1] * rng.choice([1, 2, 4]))
    p = q[-1] * p_groups
    n = [rng.randint(0, 12) for _ in range(levels)]
    w = [[rng.uniform(0.1, 3.0) for _ in range(n[l])] for l in range(levels)]
    return q, n, w, p


def test_theorem_3_1_on_random_divisible_instances():
    rng = random.Random(0)
    for _ in range(300):
        q, n, w, p = random_instance(rng, levels=rng.randint(1, 4), p_groups=rng.randint(1, 5))
        if sum(n) == 0:
            continue
        r, _ = osched.greedy(q, n, w, p)
        wmax = max(x for lvl in w for x in lvl)
        assert r["idle_before_last"] < 1e-12
        assert r["makespan"] <= r["work_total"] / p + wmax + 1e-12
        assert r["makespan"] <= 2 * r["work_lb"] + 1e-12
        assert r["makespan"] >= r["work_lb"] - 1e-12


@pytest.mark.parametrize("p", [2, 3, 4, 8])
def test_tight_example_of_the_text(p):
    # p^2 unit tasks, then one task p times longer, one processor each
    w = [[1.0] * (p * p) + [float(p)]]
    r, _ = osched.greedy([1], [p * p + 1], w, p)
    assert r["makespan"] == 2 * p
    if p <= 3:
        assert osched.optimal_makespan(w[0], p) == p + 1


def test_greedy_within_twice_brute_force_optimum():
    rng = random.Random(1)
    for _ in range(60):
        p = rng.randint(2, 3)
        n = rng.randint(1, 7)
        w = [rng.choice([1.0, 2.0, 3.0, 5.0]) for _ in range(n)]
        r, _ = osched.greedy([1], [n], [w], p)
        opt = osched.optimal_makespan(w, p)
        assert opt - 1e-12 <= r["makespan"] < 2 * opt


def test_batched_dispatch_keeps_the_bound_and_helps_under_dispatch_cost():
    rng = random.Random(2)
    # Sec. 5.1 shape: q = 8, 64, 512 cores, N = C (1024, 64, 4), short tasks
    q, C = [8, 64, 512], 2
    n = [1024 * C, 64 * C, 4 * C]
    p = 512 * 4
    w = [osched.pause_times(rng, 1e-4, 1e-10, n[l]) for l in range(3)]
    free_single, _ = osched.greedy(q, n, w, p)
    free_batch, _ = osched.greedy(q, n, w, p, batch=True)
    for r in (free_single, free_batch):
        assert r["idle_before_last"] < 1e-12
        assert r["makespan"] <= 2 * r["work_lb"] + 1e-15
    cost = 2e-5
    single, _ = osched.greedy(q, n, w, p, dispatch_cost=cost)
    batched, _ = osched.greedy(q, n, w, p, batch=True, dispatch_cost=cost)
    eff = lambda r: r["work_total"] / (p * r["makespan"])
    assert batched["batches"] < single["batches"]
    assert eff(batched) > eff(single)


# ------------------------------------------------------ library parity

@pytest.fixture(scope="module")
def m():
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as mod
    mod.lib()
    return mod


def test_library_batch_size_equals_oracle(m):
    for N in (0, 1, 5, 64, 100, 1023, 4096, 99991):
        for parts in (1, 2, 7, 64, 600):
            for n in sorted({0, 1, N // 3, N // 2, max(N - 1, 0), N}):
                assert m.batch_size(N, n, parts, 0.01, osched.PHI_INV) == osched.batch_size(N, n, parts)
    assert m.batch_size(10, 0, 0, 0.01, 0.6) == -1
    assert m.batch_size(10, 0, 2, 0.7, 0.6) == -1


@pytest.mark.parametrize("batch,cost", [(False, 0.0), (True, 0.0), (False, 0.3), (True, 0.05)])
def test_library_schedule_equals_oracle(m, batch, cost):
    rng = random.Random(5)
    for _ in range(40):
        q, n, w, p = random_instance(rng, levels=rng.randint(1, 4), p_groups=rng.randint(1, 5))
        ref, starts = osched.greedy(q, n, w, p, batch=batch, dispatch_cost=cost)
        flat = [x for lvl in w for x in lvl]
        got, st = m.schedule_greedy(q, n, flat, p, batch=batch, min_frac=0.01,
                                    max_frac=osched.PHI_INV, dispatch_cost=cost, want_starts=True)
        assert got == ref
        assert list(st) == [x for lvl in starts for x in lvl]


def test_library_schedule_rejects_non_divisible_groups(m):
    with pytest.raises(m.MLMCError):
        m.schedule_greedy([2, 3], [1, 1], [1.0, 1.0], 6)
    with pytest.raises(m.MLMCError):
        m.schedule_greedy([1, 2], [1, 1], [1.0, 1.0], 3)
    with pytest.raises(m.MLMCError):
        m.schedule_greedy([1], [1], [-1.0], 2)
