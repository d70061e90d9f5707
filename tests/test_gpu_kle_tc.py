"""The KLE contraction on the tensor cores (tcgen05, split BF16, FP32
accumulation) that gives the mixed form its FP32 kappa, through the C ABI.

kappa32 from mlmc_kappa32 is compared element by element with the oracle's
exp(Phi xi) (dense FP64 KLE of Sec. 5.2): the split-BF16 products carry about
16 significant bits, so the bound is 1e-4 relative. The mixed-form solves
that take their FP32 kappa from it still meet the FP64 parity tolerance
against the oracle (1e-9 per QoI): the outer FP64 residual uses the FP64
kappa, the tensor-core kappa only shapes the inner FP32 iterations."""
import numpy as np
import pytest

from oracle import kle, mlmc as omlmc
from synth import small_case, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_K32 = 1e-4
RTOL_Q = 1e-9


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


@pytest.mark.parametrize("dim,n0,levels,mpd,lam,sigma2,order,count", [
    (2, 8, 3, 4, 0.3, 1.0, -1, 5),        # M = 16, one 64-mode chunk, 8^2..32^2 (ragged tiles)
    (2, 32, 2, 8, 0.1, 1.0, -1, 100),     # M = 64, 32^2 and 64^2, 100 samples (N tile 112)
    (2, 16, 2, 8, 0.1, 1.5, -1, 300),     # 300 samples: two sample tiles of the CTA grid
    (3, 4, 3, 5, 0.2, 1.0, -1, 7),        # M = 125: two chunks, 4^3..16^3
    (3, 8, 2, 7, 0.1, 1.0, -1, 4),        # the 3D mixed workload's M = 343 (6 chunks)
    (3, 8, 2, 16, 0.25, 0.0625, 14, 3),   # total order 14 of 16 per axis: M = 680 (11 chunks)
])
def test_kappa32_tensor_cores_against_oracle(m, dim, n0, levels, mpd, lam, sigma2, order, count):
    cfg = m.config(dim=dim, n_levels=levels, coarse_cells=n0, modes_per_dim=mpd, corr_len=lam,
                   sigma2=sigma2, seed=5, total_order=order, precision="mixed")
    M = kle.n_modes(dim, mpd, None if order < 0 else order)
    with m.Plan(cfg, stream()) as plan:
        xi = torch.zeros(count * M, dtype=torch.float64, device="cuda")
        plan.draw_xi(levels - 1, 0, count, xi.data_ptr())
        xin = xi.cpu().numpy().reshape(count, M)
        for mesh in range(levels):
            n = n0 << mesh
            es = m.elem_stride(dim, n)
            k32 = torch.full((count * es,), float("nan"), dtype=torch.float32, device="cuda")
            plan.kappa32(mesh, xi.data_ptr(), count, k32.data_ptr())
            torch.cuda.synchronize()
            got = k32.cpu().numpy().astype(np.float64).reshape(count, es)[:, :n ** dim]
            ref = kle.kappa(dim, n, lam, sigma2, mpd, xin, None if order < 0 else order)
            err = np.max(np.abs(got - ref) / ref)
            assert err <= RTOL_K32, (mesh, err)
            # the contraction is not a plain rounding of kappa: it carries its own error
            assert err > 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_form_with_tensor_core_kappa_meets_fp64_tolerance(m, dim):
    if dim == 2:
        wl = small_case(2, n0=16, levels=3, m=8, corr_len=0.1, solver="gmg", rtol=1e-11,
                        precision="mixed")
    else:
        wl = small_case(3, n0=8, levels=2, m=5, corr_len=0.2, qoi="box", solver="gmg",
                        rtol=1e-11, precision="mixed")
    cfg = m.config_from_workload(wl, kle_tensor=1)
    L = wl["levels"] - 1
    with m.Plan(cfg, stream()) as plan:
        qf, qc, it = plan.sample_level(L, 0, 6)
    assert np.all(it > 0)
    for i in range(6):
        rf, rc = omlmc.coupled_sample(wl, L, i)
        assert abs(qf[i] - rf) <= RTOL_Q * abs(rf)
        assert abs(qc[i] - rc) <= RTOL_Q * abs(rc)


def test_3d_mixed_workload_level_with_tensor_core_kappa(m):
    """The 3D mixed workload (M = 343) on its 64^3/32^3 level with the FP32
    kappa from the tensor cores, in graph-captured rounds: QoIs against the
    oracle, and the same QoIs (to rounding) as the plan that casts kappa."""
    wl = workload("3d-mixed")
    got = {}
    for tc in (1, 0):
        cfg = m.config_from_workload(wl, kle_tensor=tc)
        with m.Plan(cfg, stream()) as plan:
            qf, qc, it = plan.sample_level(2, 0, 4)
        assert np.all(it > 0)
        got[tc] = (qf, qc)
    rf, rc = omlmc.coupled_sample(wl, 2, 0)
    assert abs(got[1][0][0] - rf) <= RTOL_Q * abs(rf)
    assert abs(got[1][1][0] - rc) <= RTOL_Q * abs(rc)
    for a, b in zip(got[1], got[0]):
        assert np.all(np.abs(a - b) <= 2 * RTOL_Q * np.abs(b))
