"""mlmc_autotune: times the settings of the selected knobs on a probe batch,
keeps the fastest, restores the level states; the tuned plan still meets the
oracle parity of its form (the knobs change iterates, not the stopping rule)."""
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


@pytest.mark.parametrize("dim,precision,flags,n_cand", [(2, "mixed", 3, 15), (3, "mixed", 7, 60),
                                                        (3, "fp64", 6, 12), (2, "fp64", 1, 1)])
def test_autotune_keeps_a_candidate_and_parity(m, dim, precision, flags, n_cand):
    if dim == 2:
        wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", rtol=1e-11, precision=precision)
    else:
        wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", rtol=1e-11,
                        precision=precision)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, torch.cuda.current_stream().cuda_stream) as plan:
        rep = plan.autotune(2, 8, flags)
        assert rep["candidates"] == n_cand
        assert 0 < rep["best_ms"] <= rep["worst_ms"]
        if precision == "mixed" and flags & 1:
            assert rep["inner_rtol"] in (1e-2, 3e-3, 1e-3, 3e-4, 1e-4)
        if flags & 2:
            assert rep["mg_omega"] in (0.7, 0.8, 0.9)
        if dim == 3 and flags & 4:
            assert rep["z_chunk"] in (0, 24, 32, 64)
        assert all(plan.level_stats(l)[0] == 0 for l in range(3))
        qf, qc, _ = plan.sample_level(2, 0, 3)
    for s in range(3):
        rf, rc = omlmc.coupled_sample(wl, 2, s)
        assert abs(qf[s] - rf) <= 1e-9 * abs(rf)
        assert abs(qc[s] - rc) <= 1e-9 * abs(rc)


def test_autotune_tile_shape_and_batch_split(m):
    """The 3D FP32 stencil tile shape (full-width TMA tiles with four or two
    rows per thread, or 32 x 16 cp.async tiles) and the batch width of rounds are tuned on a round of the
    level; the tuned plan keeps the oracle parity."""
    wl = small_case(3, n0=8, levels=3, m=3, solver="gmg", qoi="box", rtol=1e-11, precision="mixed")
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, torch.cuda.current_stream().cuda_stream) as plan:
        rep = plan.autotune(2, 16, m.TUNE_TILE | m.TUNE_BATCH)
        assert rep["candidates"] == 9              # 3 tiles x splits (1, 2, 4)
        assert rep["stencil_tile"] in (0, 1, 2) and rep["batch_split"] in (0, 2, 4)
        qf, qc, _ = plan.sample_level(2, 0, 2)
    for s in range(2):
        rf, rc = omlmc.coupled_sample(wl, 2, s)
        assert abs(qf[s] - rf) <= 1e-9 * abs(rf)
        assert abs(qc[s] - rc) <= 1e-9 * abs(rc)


@pytest.mark.parametrize("dim", [2, 3])
def test_batch_split_splits_rounds_without_changing_results(m, dim):
    """A round whose levels are each split into batch_split batches (parallel
    graph branches, folded in sample order) gives the same estimate, variance
    and sample counts as one batch per level, bit for bit."""
    if dim == 2:
        wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision="fp64")
    else:
        wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", precision="mixed")
    s = torch.cuda.current_stream().cuda_stream
    out = []
    for bw in (0, 3, 7):
        with m.Plan(m.config_from_workload(wl, batch_split=bw), s) as plan:
            q, v, N = plan.run(eps=1e-3, pilot=10)
        out.append((q, v, [int(x) for x in N]))
    assert out[1] == out[0] and out[2] == out[0]


def test_stencil_tiles_agree(m):
    """The three 3D FP32 stencil tile shapes compute the same per-node
    arithmetic (their per-tile partial sums differ in rounding only): the
    mixed-form QoIs agree within the parity tolerance."""
    wl = small_case(3, n0=8, levels=3, m=3, solver="gmg", qoi="box", rtol=1e-11, precision="mixed")
    s = torch.cuda.current_stream().cuda_stream
    got = []
    for tile in (0, 1, 2):
        with m.Plan(m.config_from_workload(wl, stencil_tile=tile), s) as plan:
            qf, qc, _ = plan.sample_level(2, 0, 4)
        got.append((qf, qc))
    import numpy as np
    for other in got[1:]:
        for a, b in zip(got[0], other):
            assert np.all(np.abs(a - b) <= 1e-9 * np.abs(b))
