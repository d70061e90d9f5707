"""GPU parity of the adaptive number of levels (Sec. 2.3, Eq. (mlmc_num_levels)).

* mlmc_adapt on the device's own level states against the oracle's fit,
  level rule and allocation applied to those same states: the decisions
  (level, sample counts) are identical and (alpha, c) agree to 1e-12
  relative (both sides in FP64; log2/exp2 may differ by an ulp).
* mlmc_run_adaptive against the oracle's run_adaptive_levels on the same
  configuration: same final level, same sample counts, estimate within
  1e-9 relative (the plain FP64 per-sample tolerance).
* The server with adapt_from = k equals mlmc_run_adaptive(L0 = k) bit for
  bit, alone and in a mix.
"""
import functools

import numpy as np
import pytest

from oracle import mlmc as omlmc
from synth import small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as mod
    mod.lib()
    return mod


def stream():
    return torch.cuda.current_stream().cuda_stream


def case(dim=2, **over):
    if dim == 2:
        wl = small_case(2, n0=4, levels=5, m=4, solver="gmg", rtol=1e-11)
    else:
        wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", rtol=1e-11)
    wl.update(over)
    return wl


@pytest.mark.parametrize("La,counts,eps", [(1, (40, 20), 1e-3), (2, (60, 30, 15), 3e-4),
                                           (3, (50, 25, 12, 6), 1e-4), (2, (30, 30, 30), 5e-2)])
def test_adapt_step_matches_oracle_on_device_states(m, La, counts, eps):
    wl = case()
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        for l, n in enumerate(counts):
            plan.sample_level(l, 0, n, want=False)
        N, L, (alpha, c) = plan.adapt(La, eps)
        states = [plan.level_stats(l) for l in range(La + 1)]
    V = [m2 / n for (n, _, m2, _) in states]
    C = [omlmc.level_cost(wl, l) for l in range(La + 1)]
    assert list(N) == omlmc.allocate(V, C, eps)
    ra, rc = omlmc.fit_bias([mean for (_, mean, _, _) in states])
    assert abs(alpha - ra) <= 1e-12 * ra and abs(c - rc) <= 1e-12 * rc
    rL = min(max(omlmc.num_levels(ra, rc, eps), La), wl["levels"] - 1)
    assert L == rL


def test_adapt_without_difference_levels_keeps_level(m):
    cfg = m.config_from_workload(case())
    with m.Plan(cfg, stream()) as plan:
        plan.sample_level(0, 0, 10, want=False)
        N, L, _ = plan.adapt(0, 1e-3)
    assert L == 0 and N[0] > 0


@functools.lru_cache(maxsize=None)
def oracle_adaptive(dim, eps, pilot, L0):
    wl = case(dim)
    q, v, states, L = omlmc.run_adaptive_levels(wl, eps, pilot, L0, max_rounds=64)
    return q, v, [s.n for s in states], L


@pytest.mark.parametrize("dim,eps,pilot,L0", [(2, 2e-3, 10, 1), (2, 4e-4, 10, 1), (2, 4e-4, 8, 2),
                                              (3, 3e-4, 8, 1)])
def test_run_adaptive_matches_oracle(m, dim, eps, pilot, L0):
    wl = case(dim)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        q, v, N, L = plan.run_adaptive(eps, pilot, L0)
    rq, rv, rN, rL = oracle_adaptive(dim, eps, pilot, L0)
    assert L == rL
    assert [int(x) for x in N] == rN
    assert abs(q - rq) <= 1e-9 * abs(rq)
    assert abs(v - rv) <= 1e-6 * rv
    assert v <= eps ** 2 / 2 * (1 + 1e-9)


def test_level_grows_when_eps_shrinks(m):
    cfg = m.config_from_workload(case())
    Ls = []
    with m.Plan(cfg, stream()) as plan:
        for eps in (5e-3, 1e-3, 2e-4, 4e-5):
            Ls.append(plan.run_adaptive(eps, 10, 1)[3])
    assert Ls == sorted(Ls) and Ls[-1] > Ls[0]


@pytest.mark.parametrize("adapt_from", [1, 2])
def test_server_adaptive_equals_plan_call(m, adapt_from):
    reqs = []
    for k in range(6):
        dim = 2 if k % 2 == 0 else 3
        wl = case(dim, sigma2=0.5 + 0.2 * k, corr_len=0.15 + 0.03 * k, seed=5 + k, stream_id=k,
                  precision="mixed" if k % 3 == 1 else "fp64")
        reqs.append((wl, 2e-3 / (1 + k)))
    alone = []
    for wl, eps in reqs:
        with m.Plan(m.config_from_workload(wl, use_graphs=1), stream()) as plan:
            q, v, N, L = plan.run_adaptive(eps, 8, adapt_from)
        alone.append((q, v, [int(x) for x in N], L))
    with m.Server(max_slots=3, pilot=8, adapt_from=adapt_from) as srv:
        ids = [srv.submit(m.config_from_workload(wl), eps) for wl, eps in reqs]
        srv.drain(600.0)
        got = [srv.poll(i) for i in ids]
    for (q, v, N, L), r in zip(alone, got):
        assert r["status"] == 0
        assert r["levels"] == L + 1
        assert r["N"][:len(N)] == N
        assert (r["q_hat"], r["stat_var"]) == (q, v)
