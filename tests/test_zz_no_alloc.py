"""mlmc_solve_noalloc: the batched solve for callers that may not allocate
device memory (code inside another framework's memory arena, latency-critical
loops that cannot take cudaMalloc's device synchronisation, hosts that forbid
device allocation). It keeps its scratch in a static device array of the
library instead of a plan workspace.

Checked through the C ABI against the plan-based mlmc_solve on the same
inputs, on two calls in a row (different meshes, solvers and batch sizes, so
the second call runs on scratch that still holds the first call's data).
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from synth import random_element_field

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


def _kappa_device(m, n, count, seed):
    es = m.elem_stride(2, n)
    k = np.zeros((count, es))
    k[:, :n * n] = random_element_field(2, n, count, seed=seed, spread=1.0)
    return torch.from_numpy(k.reshape(-1)).cuda()


def _plan_solve(m, cfg, mesh, kap, count):
    q = torch.zeros(count, dtype=torch.float64, device="cuda")
    it = torch.zeros(count, dtype=torch.int32, device="cuda")
    with m.Plan(cfg, torch.cuda.current_stream().cuda_stream) as plan:
        plan.solve(mesh, kap.data_ptr(), count, 0, q.data_ptr(), it.data_ptr())
    torch.cuda.synchronize()
    return q.cpu().numpy(), it.cpu().numpy()


def _noalloc_solve(m, cfg, mesh, kap, count):
    q = torch.full((count,), np.nan, dtype=torch.float64, device="cuda")
    it = torch.full((count,), -7, dtype=torch.int32, device="cuda")
    st = m.lib().mlmc_solve_noalloc(ctypes.byref(cfg), mesh, ctypes.c_void_p(kap.data_ptr()),
                                    count, ctypes.c_void_p(q.data_ptr()),
                                    ctypes.c_void_p(it.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, q.cpu().numpy(), it.cpu().numpy()


def test_noalloc_matches_plan_solve_on_two_calls(m):
    cases = [
        # (solver, n0, mesh, count, seed): GMG on 64^2, then Jacobi on 32^2
        ("gmg", 16, 2, 24, 1),
        ("jacobi", 8, 2, 10, 2),
    ]
    for solver, n0, mesh, count, seed in cases:
        cfg = m.config(dim=2, n_levels=mesh + 1, coarse_cells=n0, solver=solver, rtol=1e-11)
        n = n0 << mesh
        kap = _kappa_device(m, n, count, seed)
        q_ref, it_ref = _plan_solve(m, cfg, mesh, kap, count)
        st, q, it = _noalloc_solve(m, cfg, mesh, kap, count)
        assert st == m.MLMC_OK
        assert np.all(it_ref > 0)
        # mlmc_solve runs the FP64 2D stencils on precomputed operator
        # coefficients and a fused V-cycle bottom; this entry point runs the
        # kappa-form kernels and separate coarse levels. Same algorithm, so
        # the QoIs agree to rounding; the stopping test may then trip one
        # iteration apart.
        assert np.all(np.abs(it - it_ref) <= 1)
        assert np.all(np.abs(q - q_ref) <= RTOL_Q * np.abs(q_ref))


def test_noalloc_rejects_batches_beyond_the_scratch(m):
    """A batch one sample too large is rejected before any launch. The buffers
    passed are sized for the whole batch, so that a regression of the size
    check shows as a failed assertion and never as an access beyond them."""
    cfg = m.config(dim=2, n_levels=5, coarse_cells=16, solver="gmg")
    n = 16 << 4                                   # 256^2 cells
    ns = m.node_stride(2, n)
    # any PCG needs at least x, r, z, q and two directions on the finest mesh:
    # count samples of those alone already exceed the scratch
    count = m.NOALLOC_SCRATCH_BYTES // (6 * 8 * ns) + 1
    kap = torch.ones(count * m.elem_stride(2, n), dtype=torch.float64, device="cuda")
    q = torch.zeros(count, dtype=torch.float64, device="cuda")
    it = torch.zeros(count, dtype=torch.int32, device="cuda")
    st = m.lib().mlmc_solve_noalloc(ctypes.byref(cfg), 4, ctypes.c_void_p(kap.data_ptr()), count,
                                    ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(it.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == m.MLMC_ERR_INVALID
