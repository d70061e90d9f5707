"""The FP32 operator of the mixed form's inner solve (mlmc_apply32) against
the oracle's assembled Q1 matrix, on FP32 inputs, within the FP32 error
bound: |y - A x| <= 64 * 2^-24 * (|A| |x|) per node. In the mixed form the
FP64 outer residual corrects whatever the inner solve gets wrong, so a
fault in an FP32 stencil would only cost iterations there: this test
checks the FP32 kernels themselves. In 3D every stencil tile shape
(mlmc_config.stencil_tile: full-width TMA tiles with four or two rows per
thread, 32 x 16 cp.async tiles) is checked; on 128^3 (too large to assemble
here) against the FP64 operator of the same plan on the same inputs, which
the oracle pins on the smaller meshes."""
import numpy as np
import pytest

from oracle import fem
from synth import random_element_field, random_node_vectors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = 64 * 2.0 ** -24


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


def to_dev(arrs, stride, dtype):
    out = torch.zeros((arrs.shape[0], stride), dtype=dtype)
    out[:, :arrs.shape[1]] = torch.from_numpy(arrs).to(dtype)
    return out.reshape(-1).cuda()


def apply32(m, dim, n, x32, k32, tile=0):
    cfg = m.config(dim=dim, n_levels=1, coarse_cells=n, precision="mixed", stencil_tile=tile)
    ns, es = m.node_stride(dim, n), m.elem_stride(dim, n)
    count = x32.shape[0]
    with m.Plan(cfg, stream()) as plan:
        xd = to_dev(x32, ns, torch.float32)
        kd = to_dev(k32, es, torch.float32)
        yd = torch.full_like(xd, float("nan"))
        plan.apply32(0, kd.data_ptr(), xd.data_ptr(), yd.data_ptr(), count)
        y = yd.cpu().numpy().reshape(count, ns)[:, :(n + 1) ** dim].astype(np.float64)
        # the same inputs through the FP64 operator of the plan
        xd64 = to_dev(x32.astype(np.float64), ns, torch.float64)
        kd64 = to_dev(k32.astype(np.float64), es, torch.float64)
        yd64 = torch.full_like(xd64, float("nan"))
        plan.apply(0, kd64.data_ptr(), xd64.data_ptr(), yd64.data_ptr(), count)
        y64 = yd64.cpu().numpy().reshape(count, ns)[:, :(n + 1) ** dim]
    return y, y64


def inputs(dim, n, count, seed):
    x = random_node_vectors(dim, n, count, seed=seed).astype(np.float32)
    k = random_element_field(dim, n, count, seed=seed + 1).astype(np.float32)
    return x, k


def check_against_oracle(dim, n, x32, k32, y):
    for s in range(x32.shape[0]):
        A = fem.assemble_fast(dim, n, k32[s].astype(np.float64))
        xi_ = fem.from_node_grid(dim, n, x32[s].astype(np.float64))
        ref = A @ xi_
        scale = abs(A) @ np.abs(xi_)
        got = fem.from_node_grid(dim, n, y[s])
        assert np.all(np.abs(got - ref) <= BOUND * scale + 1e-30), (dim, n, s)
        full = y[s].reshape((n + 1,) * dim)
        assert np.all(full[0] == 0) and np.all(full[-1] == 0)
        assert np.all(np.take(full, 0, axis=-1) == 0) and np.all(np.take(full, -1, axis=-1) == 0)


@pytest.mark.parametrize("n", [2, 33, 64, 130])
def test_apply32_2d_against_oracle(m, n):
    x32, k32 = inputs(2, n, 3, seed=700 + n)
    y, _ = apply32(m, 2, n, x32, k32)
    check_against_oracle(2, n, x32, k32, y)


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("n", [8, 32, 64])
def test_apply32_3d_against_oracle(m, n, tile):
    x32, k32 = inputs(3, n, 2, seed=900 + n)
    y, _ = apply32(m, 3, n, x32, k32, tile)
    check_against_oracle(3, n, x32, k32, y)


@pytest.mark.parametrize("tile", [0, 1, 2])
def test_apply32_3d_128_against_fp64_operator(m, tile):
    n = 128
    x32, k32 = inputs(3, n, 2, seed=1234)
    y, y64 = apply32(m, 3, n, x32, k32, tile)
    # |A| |x| from the FP64 operator on |x| and the same kappa (A's
    # off-diagonal entries are <= 0, its diagonal > 0: |A| |x| = 2 D |x| - A |x|)
    cfg = m.config(dim=3, n_levels=1, coarse_cells=n)
    ns, es = m.node_stride(3, n), m.elem_stride(3, n)
    with m.Plan(cfg, stream()) as plan:
        xa = to_dev(np.abs(x32).astype(np.float64), ns, torch.float64)
        kd = to_dev(k32.astype(np.float64), es, torch.float64)
        ya = torch.zeros_like(xa)
        plan.apply(0, kd.data_ptr(), xa.data_ptr(), ya.data_ptr(), 2)
        a_abs = ya.cpu().numpy().reshape(2, ns)[:, :(n + 1) ** 3]
    h = 1.0 / n
    k = k32.astype(np.float64).reshape(2, n, n, n)
    ksum = np.zeros((2, n + 1, n + 1, n + 1))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                ksum[:, dz:dz + n, dy:dy + n, dx:dx + n] += k
    diag = (h / 3.0) * ksum.reshape(2, -1) * np.abs(x32.astype(np.float64))
    scale = 2 * diag - a_abs
    inner = np.zeros((n + 1,) * 3, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    inner = inner.reshape(-1)
    for s in range(2):
        err = np.abs(y[s] - y64[s])[inner]
        assert np.all(err <= BOUND * scale[s][inner] + 1e-30), (tile, s, float(err.max()))
        full = y[s].reshape((n + 1,) * 3)
        assert np.all(full[0] == 0) and np.all(full[-1] == 0)
        assert np.all(full[:, 0] == 0) and np.all(full[:, :, -1] == 0)
