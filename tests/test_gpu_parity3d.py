"""GPU parity of the 3D path (trilinear Q1, box QoI, 3D multigrid) against the
CPU oracle, through the C ABI. Tolerances as in test_gpu_parity.py."""
import functools

import numpy as np
import pytest

from oracle import fem, kle, mlmc as omlmc
from synth import random_element_field, random_node_vectors, small_case, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def to_dev(arrs, stride):
    out = torch.zeros((arrs.shape[0], stride), dtype=torch.float64)
    out[:, :arrs.shape[1]] = torch.from_numpy(arrs)
    return out.reshape(-1).cuda()


@pytest.mark.parametrize("n0,levels,mpd,lam", [(2, 3, 3, 0.2), (4, 2, 5, 0.1), (3, 2, 4, 0.3)])
def test_kappa3d_parity(m, n0, levels, mpd, lam):
    cfg = m.config(dim=3, n_levels=levels, coarse_cells=n0, modes_per_dim=mpd, corr_len=lam, seed=2)
    M = mpd ** 3
    count = 5
    with m.Plan(cfg, stream()) as plan:
        xi = torch.zeros(count * M, dtype=torch.float64, device="cuda")
        plan.draw_xi(levels - 1, 0, count, xi.data_ptr())
        xin = xi.cpu().numpy().reshape(count, M)
        for mesh in range(levels):
            n = n0 << mesh
            es = m.elem_stride(3, n)
            kap = torch.zeros(count * es, dtype=torch.float64, device="cuda")
            plan.kappa(mesh, xi.data_ptr(), count, kap.data_ptr())
            got = kap.cpu().numpy().reshape(count, es)[:, :n ** 3]
            ref = kle.kappa(3, n, lam, 1.0, mpd, xin)
            assert np.max(np.abs(got - ref) / ref) <= 1e-12


@pytest.mark.parametrize("n", [2, 3, 5, 8, 16])
def test_apply3d_parity(m, n):
    cfg = m.config(dim=3, n_levels=1, coarse_cells=n)
    count = 3
    x = random_node_vectors(3, n, count, seed=n)
    kap = random_element_field(3, n, count, seed=50 + n)
    ns = m.node_stride(3, n)
    with m.Plan(cfg, stream()) as plan:
        xd = to_dev(x, ns)
        kd = to_dev(kap, m.elem_stride(3, n))
        yd = torch.full_like(xd, np.nan)
        plan.apply(0, kd.data_ptr(), xd.data_ptr(), yd.data_ptr(), count)
        y = yd.cpu().numpy().reshape(count, ns)[:, :(n + 1) ** 3]
    for s in range(count):
        A = fem.assemble(3, n, kap[s]) if n <= 5 else fem.assemble_fast(3, n, kap[s])
        xi_ = fem.from_node_grid(3, n, x[s])
        ref = A @ xi_
        scale = abs(A) @ np.abs(xi_)
        got = fem.from_node_grid(3, n, y[s])
        assert np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300)
        full = y[s].reshape((n + 1,) * 3)
        assert np.all(full[0] == 0) and np.all(full[-1] == 0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("solver,n,qoi", [("jacobi", 8, "domain"), ("gmg", 8, "box"),
                                          ("gmg", 16, "box"), ("gmg", 4, "domain"),
                                          ("jacobi", 2, "domain")])
def test_solve3d_parity(m, solver, n, qoi, precision):
    count = 4
    cfg = m.config(dim=3, n_levels=1, coarse_cells=n, solver=solver, rtol=1e-11, qoi=qoi,
                   precision=precision)
    kap = random_element_field(3, n, count, seed=9 * n, spread=0.7)
    ns = m.node_stride(3, n)
    with m.Plan(cfg, stream()) as plan:
        kd = to_dev(kap, m.elem_stride(3, n))
        u = torch.zeros(count * ns, dtype=torch.float64, device="cuda")
        q = torch.zeros(count, dtype=torch.float64, device="cuda")
        it = torch.zeros(count, dtype=torch.int32, device="cuda")
        plan.solve(0, kd.data_ptr(), count, u.data_ptr(), q.data_ptr(), it.data_ptr())
        qh = q.cpu().numpy()
        iters = it.cpu().numpy()
    assert np.all(iters > 0)
    b = fem.load_vector(3, n)
    w = fem.qoi_weights(3, n, qoi)
    for s in range(count):
        uref = fem.solve_direct(fem.assemble_fast(3, n, kap[s]), b)
        qref = w @ uref
        assert abs(qh[s] - qref) <= RTOL_Q * abs(qref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coupled_samples_3d(m, precision):
    wl = small_case(3, n0=4, levels=3, m=3, corr_len=0.2, qoi="box", solver="gmg", rtol=1e-11,
                    precision=precision)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        for level in range(3):
            qf, qc, it = plan.sample_level(level, 0, 5)
            ref = [omlmc.coupled_sample(wl, level, i) for i in range(5)]
            for s in range(5):
                assert abs(qf[s] - ref[s][0]) <= RTOL_Q * abs(ref[s][0])
                if level > 0:
                    assert abs(qc[s] - ref[s][1]) <= RTOL_Q * abs(ref[s][1])
            n, mean, m2, _ = plan.level_stats(level)
            ys = np.array([a - b_ for a, b_ in ref])
            assert n == 5 and abs(mean - ys.mean()) <= 1e-9 * abs(ys.mean()) + 1e-15


@functools.lru_cache(maxsize=None)
def oracle3(level, i):
    return omlmc.coupled_sample(workload("3d-batched"), level, i)


@pytest.mark.parametrize("precision,level,checked", [("fp64", 3, (0, 63)), ("mixed", 3, (0,)),
                                                     ("fp64", 4, (0,))])
def test_3d_batched_full_size(m, precision, level, checked):
    """3D workload (8^3..128^3, M = 125, box QoI) at full size, 64 samples per call."""
    wl = workload("3d-batched", precision=precision)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        qf, qc, it = plan.sample_level(level, 0, 64)
        n, mean, m2, _ = plan.level_stats(level)
    assert n == 64 and np.all(it > 0)
    assert np.all(qf > 0) and np.all(qc > 0)
    assert np.max(np.abs(qf - qc)) < 0.2 * np.min(qf)
    for i in checked:
        rf, rc = oracle3(level, i)
        assert abs(qf[i] - rf) <= RTOL_Q * abs(rf)
        assert abs(qc[i] - rc) <= RTOL_Q * abs(rc)


@functools.lru_cache(maxsize=None)
def oracle4(level, i):
    return omlmc.coupled_sample(workload("3d-mixed"), level, i)


@pytest.mark.parametrize("level,count,checked", [(0, 32, (0, 31)), (1, 16, (0, 15)), (2, 8, (0, 7)),
                                                 (3, 4, (0,))])
def test_3d_mixed_workload_against_oracle(m, level, count, checked):
    """The 3D mixed-precision workload at its own field and sizes (16^3..256^3
    elements, corr_len 0.1, M = 343 tensor modes, box QoI, FP32 inner GMG-PCG
    with FP64 refinement to rtol 1e-10): coupled samples of levels 0..3
    (meshes up to 128^3) against the FP64 oracle, Q_f and Q_c each within
    1e-9 relative."""
    wl = workload("3d-mixed")
    cfg = m.config_from_workload(wl)
    assert cfg.precision == m.MIXED and cfg.modes_per_dim == 7
    with m.Plan(cfg, stream()) as plan:
        qf, qc, it = plan.sample_level(level, 0, count)
        n, mean, m2, _ = plan.level_stats(level)
    assert n == count and np.all(it > 0)
    for i in checked:
        rf, rc = oracle4(level, i)
        assert abs(qf[i] - rf) <= RTOL_Q * abs(rf), (level, i, qf[i], rf)
        if level > 0:
            assert abs(qc[i] - rc) <= RTOL_Q * abs(rc), (level, i, qc[i], rc)


def test_3d_mixed_workload_finest_level_against_fp64_form(m):
    """Level 4 of the 3D mixed workload (256^3 fine, 128^3 coarse meshes, 4
    coupled samples): the oracle cannot solve 16.6 M unknowns in test time, so
    the mixed form is checked sample by sample against the plain FP64 form of
    the library (Q_f and Q_c within 1e-9 relative), whose own parity with the
    oracle is tested on every smaller mesh."""
    wl = workload("3d-mixed")
    got = {}
    for precision in ("mixed", "fp64"):
        cfg = m.config_from_workload(wl, precision=precision)
        with m.Plan(cfg, stream()) as plan:
            qf, qc, it = plan.sample_level(4, 0, 4)
        assert np.all(it > 0)
        got[precision] = (qf, qc)
    for a, b in zip(got["mixed"], got["fp64"]):
        assert np.all(np.abs(a - b) <= RTOL_Q * np.abs(b)), (a, b)
