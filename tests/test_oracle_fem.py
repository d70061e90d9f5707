"""Pins for the oracle's Q1 discretisation and solves (oracle/fem.py).

Pins: closed-form Q1 element entries; zero row sums and the textbook 2D
stencil for constant kappa; symmetry and positive definiteness; the loop and
vectorised assemblies agree; O(h^2) L2 convergence on manufactured
solutions in 2D and 3D; the domain-mean QoI converges at O(h^2) to the
Fourier-series value of int u for -Laplace u = 1; the box weights integrate
trilinear functions exactly; CG agrees with a dense Cholesky solve; the
CG QoI b^T x_k increases monotonically (b^T(u - x_k) = ||u - x_k||_A^2).
"""
import numpy as np
import pytest

from oracle import fem
from synth import random_element_field


def test_element_stiffness_closed_forms():
    for h in (1.0, 0.25):
        K2 = fem.element_stiffness(2, h)
        assert np.allclose(np.diag(K2), 2.0 / 3.0)
        assert np.isclose(K2[0, 1], -1.0 / 6.0) and np.isclose(K2[0, 2], -1.0 / 6.0)
        assert np.isclose(K2[0, 3], -1.0 / 3.0)
        K3 = fem.element_stiffness(3, h)
        assert np.allclose(np.diag(K3), h / 3.0)
        for b, ndiff in ((1, 1), (2, 1), (4, 1), (3, 2), (5, 2), (6, 2), (7, 3)):
            expect = {1: 0.0, 2: -h / 12.0, 3: -h / 12.0}[ndiff]
            assert np.isclose(K3[0, b], expect, atol=1e-15)
        assert np.allclose(K2.sum(axis=1), 0) and np.allclose(K3.sum(axis=1), 0)


def test_constant_kappa_stencil_and_row_sums():
    n, kap = 8, 2.5
    A = fem.assemble(2, n, np.full(n * n, kap)).toarray().reshape((n - 1,) * 4)
    # interior node (3,3): stencil kappa/3 [8 centre, -1 at the 8 neighbours]
    patch = A[3, 3, 2:5, 2:5]
    expect = kap / 3.0 * np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]])
    assert np.allclose(patch, expect)
    A3 = fem.assemble(3, 6, np.full(216, 1.0)).toarray()
    ids = np.arange(125).reshape(5, 5, 5)
    for node in ((2, 2, 2), (1, 2, 3), (3, 1, 2)):
        # rows whose stencil stays inside the interior: zero row sum
        assert abs(A3[ids[node]].sum()) < 1e-14


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_spd_and_fast_assembly(dim, n):
    kap = random_element_field(dim, n, 1, seed=11)[0]
    A = fem.assemble(dim, n, kap)
    B = fem.assemble_fast(dim, n, kap)
    assert abs(A - B).max() < 1e-15
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad).min() > 0


def _l2_error(dim, n, u_int, exact):
    """||u_h - u||_L2 with 3 Gauss points per axis per element."""
    full = fem.to_node_grid(dim, n, u_int).reshape((n + 1,) * dim)
    g, wg = np.polynomial.legendre.leggauss(3)
    g, wg = 0.5 * (g + 1), 0.5 * wg
    h = 1.0 / n
    err = 0.0
    if dim == 2:
        for a, wa in zip(g, wg):
            for b, wb in zip(g, wg):
                # [iy, ix] element arrays
                uh = ((1 - a) * (1 - b) * full[:-1, :-1] + a * (1 - b) * full[:-1, 1:]
                      + (1 - a) * b * full[1:, :-1] + a * b * full[1:, 1:])
                x = (np.arange(n)[None, :] + a) * h
                y = (np.arange(n)[:, None] + b) * h
                err += wa * wb * h * h * np.sum((uh - exact(x, y)) ** 2)
    else:
        for a, wa in zip(g, wg):
            for b, wb in zip(g, wg):
                for c, wc in zip(g, wg):
                    uh = 0.0
                    for v in range(8):
                        vx, vy, vz = v & 1, (v >> 1) & 1, (v >> 2) & 1
                        wgt = ((a if vx else 1 - a) * (b if vy else 1 - b) * (c if vz else 1 - c))
                        uh = uh + wgt * full[vz:n + vz, vy:n + vy, vx:n + vx]
                    x = (np.arange(n)[None, None, :] + a) * h
                    y = (np.arange(n)[None, :, None] + b) * h
                    z = (np.arange(n)[:, None, None] + c) * h
                    err += wa * wb * wc * h ** 3 * np.sum((uh - exact(x, y, z)) ** 2)
    return np.sqrt(err)


def test_manufactured_convergence_2d():
    exact = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    f = lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)
    errs = []
    for n in (16, 32, 64, 128):
        A = fem.assemble_fast(2, n, np.ones(n * n))
        u = fem.solve_direct(A, fem.load_vector(2, n, f))
        errs.append(_l2_error(2, n, u, exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 1.9) & (rates < 2.1)), rates


def test_manufactured_convergence_3d():
    exact = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = lambda x, y, z: 3 * np.pi ** 2 * exact(x, y, z)
    errs = []
    for n in (8, 16, 32):
        A = fem.assemble_fast(3, n, np.ones(n ** 3))
        u = fem.solve_direct(A, fem.load_vector(3, n, f))
        errs.append(_l2_error(3, n, u, exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 1.85) & (rates < 2.15)), rates


def _poisson_mean_series():
    """int_[0,1]^2 u for -Laplace u = 1, u = 0 on the boundary (Fourier sine series)."""
    j = np.arange(1, 4001, 2, dtype=np.float64)
    J, K = np.meshgrid(j, j)
    return float(np.sum(64.0 / (np.pi ** 6 * J ** 2 * K ** 2 * (J ** 2 + K ** 2))))


def test_domain_mean_qoi_converges_to_series_value():
    ref = _poisson_mean_series()
    assert abs(ref - 0.0351442537) < 1e-9
    errs = []
    for n in (8, 16, 32, 64):
        A = fem.assemble_fast(2, n, np.ones(n * n))
        b = fem.load_vector(2, n)
        assert np.allclose(b, 1.0 / n ** 2)
        u = fem.solve_direct(A, b)
        w = fem.qoi_weights(2, n, 'domain')
        assert np.allclose(w, b)
        errs.append(abs(w @ u - ref))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 1.9) & (rates < 2.1)), rates


def test_box_weights_exact_for_trilinear():
    for dim, n in ((2, 8), (3, 8)):
        w = fem.qoi_weights(dim, n, 'box', (0.25, 0.75))
        nodes = np.arange(1, n) / n
        grids = np.meshgrid(*([nodes] * dim), indexing='ij')[::-1]   # x fastest
        u = np.prod([g.reshape(-1) for g in grids], axis=0) if dim == 3 else \
            (grids[0] * grids[1]).reshape(-1)
        # mean of x y (z) over [1/4, 3/4]^d is 0.5^d
        assert abs(w @ u - 0.5 ** dim) < 1e-14
        assert abs(w.sum() - 1.0) < 1e-14
    with pytest.raises(ValueError):
        fem.qoi_weights(3, 6, 'box', (0.25, 0.75))


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_pcg_matches_dense_cholesky(dim, n):
    kap = random_element_field(dim, n, 1, seed=5, spread=1.0)[0]
    A = fem.assemble(dim, n, kap)
    b = fem.load_vector(dim, n)
    Lc = np.linalg.cholesky(A.toarray())
    ref = np.linalg.solve(Lc.T, np.linalg.solve(Lc, b))
    x, it = fem.pcg_jacobi(A, b, rtol=1e-15)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(fem.solve_direct(A, b) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_cg_qoi_is_monotone_energy_error():
    n = 16
    kap = random_element_field(2, n, 1, seed=9)[0]
    A = fem.assemble_fast(2, n, kap)
    b = fem.load_vector(2, n)
    u = fem.solve_direct(A, b)
    qs, gaps = [], []
    fem.pcg_jacobi(A, b, rtol=1e-12, callback=lambda x: (qs.append(b @ x),
                                                         gaps.append((u - x) @ (A @ (u - x)))))
    qs, gaps = np.array(qs), np.array(gaps)
    assert np.all(np.diff(qs) >= -4 * np.finfo(float).eps * qs[-1])   # up to rounding
    assert np.allclose(b @ u - qs, gaps, rtol=1e-6, atol=8 * np.finfo(float).eps * qs[-1])


def test_solve_dispatch_pcg_branch_matches_direct():
    """fem.solve switches to Jacobi-PCG (rtol 1e-13) on large 3D meshes; both branches agree."""
    n = 12
    kap = random_element_field(3, n, 1, seed=21)[0]
    A = fem.assemble_fast(3, n, kap)
    b = fem.load_vector(3, n)
    u_lu = fem.solve_direct(A, b)
    u_cg = fem.pcg_jacobi(A, b, rtol=1e-13)[0]
    assert np.abs(u_cg - u_lu).max() <= 1e-11 * np.abs(u_lu).max()
    assert np.array_equal(fem.solve(A, b, 3), u_lu)          # small: the LU branch
