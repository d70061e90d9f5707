"""The sample dispenser driving a real plan (one rank on one GPU): the
sharded run (ranges claimed by Eq. (batch), values gathered and folded in
index order into the level states) equals mlmc_run on the same plan bit for
bit: estimate, variance, sample counts. The multi-rank exchange itself is
covered by the gloo tests (tests/test_distributed.py)."""
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


class DictStore:
    def __init__(self):
        self.d = {}

    def add(self, key, amount):
        self.d[key] = self.d.get(key, 0) + amount
        return self.d[key]


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (2, "mixed"), (3, "mixed")])
def test_sharded_run_equals_plan_run(m, dim, precision):
    from paper_2111_11788_gb300.distributed import RangeDispenser, plan_callables, run_sharded
    if dim == 2:
        wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision=precision)
    else:
        wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", precision=precision)
    eps, pilot = 1e-3, 10
    cfg = m.config_from_workload(wl)
    s = torch.cuda.current_stream().cuda_stream
    with m.Plan(cfg, s) as plan:
        q_ref, v_ref, N_ref = plan.run(eps=eps, pilot=pilot)
    with m.Plan(cfg, s) as plan:
        sample, fold, reset, allocate = plan_callables(plan)
        N, claimed = run_sharded(3, sample, fold, reset, allocate, lambda o: [o],
                                 RangeDispenser(DictStore(), 1), eps=eps, pilot=pilot)
        q, v = plan.estimate()
    assert N == [int(x) for x in N_ref]
    assert (q, v) == (q_ref, v_ref)
    assert len(claimed) > 3


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (3, "mixed")])
def test_round_sharded_run_equals_plan_run(m, dim, precision):
    """run_rounds on one rank (one graph-captured round per phase, values read
    back with mlmc_round_values and refolded in index order) equals mlmc_run
    bit for bit; the multi-rank exchange is covered on CPU ranks."""
    from paper_2111_11788_gb300.distributed import run_rounds
    if dim == 2:
        wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision=precision)
    else:
        wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", precision=precision)
    eps, pilot = 1e-3, 10
    cfg = m.config_from_workload(wl)
    s = torch.cuda.current_stream().cuda_stream
    with m.Plan(cfg, s) as plan:
        q_ref, v_ref, N_ref = plan.run(eps=eps, pilot=pilot)
    with m.Plan(cfg, s) as plan:
        N, q, v = run_rounds(plan, 0, 1, lambda counts, vals: [vals], eps=eps, pilot=pilot)
        # the values of the last round can no longer be read once the workspace is reused
        plan.sample_level(0, 10 ** 6, 1)
        with pytest.raises(m.MLMCError):
            plan.round_values(0, 1)
    assert N == [int(x) for x in N_ref]
    assert (q, v) == (q_ref, v_ref)
