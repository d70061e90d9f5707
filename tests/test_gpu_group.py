"""Cross-request batching at the plan level (mlmc_round_begin_group): one
round over several plans with different fields (sigma2, corr_len), KLE
modes, seeds and stream ids but the same meshes, solver and tolerances.
Per level their samples form one batch solved by one set of launches; each
plan's level states must equal, bit for bit, what the plan's own rounds give
on the same samples (every result depends only on its own sample)."""
import numpy as np
import pytest

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


def members(dim, precision):
    out = []
    for k, (s2, lam, mm) in enumerate(((0.7, 0.15, 3), (1.4, 0.25, 4), (1.0, 0.1, 5))):
        if dim == 2:
            wl = small_case(2, n0=8, levels=3, m=mm + 2, solver="gmg", precision=precision)
        else:
            wl = small_case(3, n0=4, levels=3, m=mm, solver="gmg", qoi="box", precision=precision)
        wl.update(sigma2=s2, corr_len=lam, seed=3 + k, stream_id=40 + k)
        out.append(wl)
    return out


def states(plan, L1):
    return [tuple(plan.level_stats(l)) for l in range(L1)]


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (2, "mixed"), (3, "fp64"), (3, "mixed")])
def test_group_round_equals_own_rounds(m, dim, precision):
    wls = members(dim, precision)
    L1 = 3
    first = np.array([[0, 5, 2], [3, 0, 0], [7, 1, 4]], dtype=np.int64)
    count = np.array([[6, 3, 2], [4, 0, 5], [2, 2, 1]], dtype=np.int64)
    s = torch.cuda.current_stream().cuda_stream
    ref = []
    for k, wl in enumerate(wls):
        with m.Plan(m.config_from_workload(wl), s) as plan:
            plan.round(first[k], count[k])
            ref.append(states(plan, L1))
    cfgs = [m.config_from_workload(wl) for wl in wls]
    plans = [m.Plan(c, s) for c in cfgs]
    try:
        nbytes = m.round_bytes_group(cfgs, count)
        assert nbytes > 0
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (ws.data_ptr() + 255) // 256 * 256
        st, bad = m.round_group(plans, first, count, base, nbytes)
        assert st == m.MLMC_OK and not bad.any()
        for k, plan in enumerate(plans):
            assert states(plan, L1) == ref[k], k
        # a plan of another solve shape cannot join; a workspace too small is refused
        other = m.config_from_workload(dict(wls[0], rtol=1e-9))
        assert m.round_bytes_group([cfgs[0], other], count[:2]) == -1
        with pytest.raises(m.MLMCError):
            m.round_group(plans, first, count, base, nbytes // 2)
    finally:
        for p in plans:
            p.close()
