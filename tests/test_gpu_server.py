"""GPU tests of the continuous-batching server (include/mlmc_server.h).

The server's contract is that a request's result does not depend on what
else is being served: every request below is run alone through mlmc_run on
its own plan and then in a mix of 2D/3D, FP64/mixed requests that arrive
while others are on the device, with a workspace budget small enough that
rounds are split into chunks and requests wait for admission. Estimates,
variances and sample counts must agree bit for bit. One FP64 request is also
checked against the oracle on the same samples (tolerance 1e-9 relative, as
for the MLMC mean of the plan API).
"""
import functools
import time

import numpy as np
import pytest

from oracle import mlmc as omlmc
from synth import small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PILOT = 8


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as mod
    mod.lib()
    return mod


def mix():
    """(workload, eps) pairs: both dimensions, both forms, varied fields and seeds."""
    out = []
    for k in range(10):
        dim = 2 if k % 2 == 0 else 3
        prec = "mixed" if k % 3 else "fp64"
        if dim == 2:
            wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision=prec)
        else:
            wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", precision=prec)
        wl.update(sigma2=0.5 + 0.15 * k, corr_len=0.1 + 0.02 * k, seed=11 + k, stream_id=k)
        out.append((wl, 4e-3 - 2.5e-4 * k))
    return out


@functools.lru_cache(maxsize=None)
def alone(m):
    res = []
    for wl, eps in mix():
        cfg = m.config_from_workload(wl, use_graphs=1)
        with m.Plan(cfg, torch.cuda.current_stream().cuda_stream) as plan:
            q, v, N = plan.run(eps=eps, pilot=PILOT)
        res.append((q, v, [int(x) for x in N]))
    return res


def serve(m, budget, slots, stagger, solo=0):
    out = {}
    with m.Server(hbm_budget=budget, max_slots=slots, pilot=PILOT, solo_rounds=solo) as srv:
        ids = []
        for k, (wl, eps) in enumerate(mix()):
            ids.append(srv.submit(m.config_from_workload(wl), eps))
            if stagger:
                time.sleep(0.002 * (k % 3))
        srv.drain(timeout=600.0)
        for k, rid in enumerate(ids):
            out[k] = srv.poll(rid)
    return out


@pytest.mark.parametrize("budget,slots,stagger,solo", [(0, 16, False, 0), (48 << 20, 3, True, 0),
                                                     (4 << 20, 2, False, 0), (0, 16, False, 1)])
def test_result_same_alone_and_in_mix(m, budget, slots, stagger, solo):
    """Bit for bit: alone through mlmc_run, and served in the mix, with
    requests that can share solves batched into group rounds (solo 0) or
    each in its own rounds (solo 1)."""
    ref = alone(m)
    got = serve(m, budget, slots, stagger, solo)
    if solo:
        assert all(r["group_rounds"] == 0 for r in got.values())
    for k, (q, v, N) in enumerate(ref):
        r = got[k]
        assert r is not None and r["status"] == 0, (k, r)
        L1 = len(N)
        assert r["N"][:L1] == N, k
        assert r["q_hat"] == q and r["stat_var"] == v, k
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        assert r["dof_solves"] > 0
        eps = mix()[k][1]
        assert v <= eps ** 2 / 2 * (1 + 1e-9)


def test_requests_overlap_and_chunk(m):
    """With several slots, admitted requests run at the same time; with a tiny
    budget a request's phase is split into several rounds."""
    got = serve(m, 0, 16, False)
    spans = sorted((r["t_admit"], r["t_done"]) for r in got.values())
    overlaps = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
    assert overlaps >= 1
    tiny = serve(m, 4 << 20, 2, False)
    assert sum(r["rounds"] for r in tiny.values()) > sum(r["rounds"] for r in got.values())


def test_served_fp64_request_matches_oracle(m):
    wl, eps = mix()[0]
    assert wl["dim"] == 2 and wl.get("precision", "fp64") == "fp64"
    r = serve(m, 0, 4, False)[0]
    ref = []
    for l in range(wl["levels"]):
        st = omlmc.Welford()
        for i in range(r["N"][l]):
            a, b = omlmc.coupled_sample(wl, l, i)
            st.add(a - b)
        ref.append(st)
    q, v = omlmc.estimate(ref)
    assert abs(r["q_hat"] - q) <= 1e-9 * abs(q)
    assert abs(r["stat_var"] - v) <= 1e-6 * v


def test_invalid_requests_rejected(m):
    with m.Server(max_slots=2, pilot=PILOT) as srv:
        cfg = m.config_from_workload(small_case(2))
        with pytest.raises(m.MLMCError):
            srv.submit(cfg, 0.0)
        cfg.dim = 5
        with pytest.raises(m.MLMCError):
            srv.submit(cfg, 1e-3)
        with pytest.raises(m.MLMCError):
            srv.poll(12345)


def test_requests_that_arrive_together_share_group_rounds(m):
    """Requests admitted at the same moment whose solves can share launches
    (same dimension, form, meshes and tolerances; different fields, modes and
    seeds) run their rounds as group rounds: same-size levels of different
    requests are solved by one batched set of launches."""
    got = serve(m, 0, 16, False, 0)
    assert sum(r["group_rounds"] for r in got.values()) >= 4
    assert all(r["group_rounds"] <= r["rounds"] for r in got.values())
