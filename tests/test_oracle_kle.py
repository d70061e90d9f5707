"""Pins for the oracle's Karhunen-Loeve expansion (oracle/kle.py).

Sec. 5.2 fixes an exponential covariance with per-dimension eigenfunctions.
The pins: each root satisfies its transcendental equation (tan form); the
eigenfunctions are orthonormal and satisfy the integral eigen-equation by
quadrature; eigenvalues sum to the variance x length (trace of the kernel)
and the Mercer sum converges pointwise; a Nystrom discretisation of the
kernel gives the same leading eigenvalues; the tensor basis reproduces the
separable covariance and the sampled log-field has the truncated variance.
Total-order truncation (Sec. 5.2): the kept-mode count equals the closed form
C(K + d, d) when K < m and a brute-force count otherwise (680 modes for d =
3, m = 16 at K = 14); the truncated field equals the full-basis field with
the dropped coefficients set to zero; its pointwise variance is the Mercer
sum over the kept modes.
"""
import itertools
import math
import numpy as np
import pytest

from oracle import kle, philox

LAMBDAS = [0.1, 0.2, 0.3]


@pytest.mark.parametrize("lam", LAMBDAS)
def test_roots_satisfy_transcendental_equations(lam):
    om, th, even = kle.eigenpairs_1d(lam, 12)
    c, a = 1.0 / lam, 0.5
    for w, e in zip(om, even):
        if e:
            res = c - w * np.tan(w * a)
            scale = c + abs(w * np.tan(w * a))
        else:
            res = w + c * np.tan(w * a)
            scale = w + abs(c * np.tan(w * a))
        assert abs(res) <= 1e-13 * scale
    # one root per interval (n pi, (n+1) pi): strictly increasing, eigenvalues decreasing
    assert np.all(np.diff(om) > 0) and np.all(np.diff(th) < 0)
    assert np.all((om > np.arange(12) * np.pi) & (om < np.arange(1, 13) * np.pi))


@pytest.mark.parametrize("lam", LAMBDAS)
def test_orthonormal_and_integral_eigen_equation(lam):
    om, th, even = kle.eigenpairs_1d(lam, 8)
    xg, wg = np.polynomial.legendre.leggauss(200)
    x = 0.5 * (xg + 1.0)
    w = 0.5 * wg
    f = kle.eigfun_1d(om, even, x)
    gram = f.T @ (w[:, None] * f)
    assert np.abs(gram - np.eye(8)).max() < 1e-12
    # int_0^1 exp(-|s-t|/lam) f(t) dt = theta f(s): split the integral at the kink
    for s in (0.0, 0.13, 0.5, 0.77, 1.0):
        val = np.zeros(8)
        for lo, hi in ((0.0, s), (s, 1.0)):
            if hi <= lo:
                continue
            t = lo + (hi - lo) * x
            val += (hi - lo) * (w[:, None] * np.exp(-np.abs(s - t) / lam)[:, None]
                                * kle.eigfun_1d(om, even, t)).sum(axis=0)
        assert np.allclose(val, th * kle.eigfun_1d(om, even, [s])[0], rtol=0, atol=1e-12)


def test_eigenvalue_sum_and_mercer():
    """sum theta_n -> int_0^1 c(x, x) dx = 1 from below; sum theta f(x)^2 -> 1."""
    om, th, even = kle.eigenpairs_1d(0.3, 4000)
    partial = np.cumsum(th)
    assert np.all(partial < 1.0)
    assert abs(partial[-1] - 0.99983) < 2e-5
    x = np.array([0.1, 0.3, 0.5, 0.9])
    merc = (th[None, :] * kle.eigfun_1d(om, even, x) ** 2).sum(axis=1)
    assert np.all(np.abs(merc - 1.0) < 5e-4)


def test_nystrom_cross_check():
    """Leading eigenvalues of the midpoint-discretised kernel match theta."""
    n = 2000
    x = (np.arange(n) + 0.5) / n
    K = np.exp(-np.abs(x[:, None] - x[None, :]) / 0.3) / n
    ev = np.sort(np.linalg.eigvalsh(K))[::-1][:4]
    om, th, even = kle.eigenpairs_1d(0.3, 4)
    assert np.allclose(ev, th, rtol=0, atol=1e-6)   # midpoint rule error O(1/n^2)
    assert np.allclose(th, [0.436249, 0.216812, 0.106997, 0.059310], atol=2e-6)


def test_tensor_basis_convention_and_covariance():
    n, m = 8, 3
    phi = kle.phi_matrix(2, n, 0.3, 2.0, m)
    assert phi.shape == (n * n, m * m)
    grid = phi.reshape(n, n, m * m)                    # [iy, ix, k]
    # k = 1 is (k_x = 1, k_y = 0): its ratio to mode 0 is f_1(x)/f_0(x), free of y
    r1 = grid[:, :, 1] / grid[:, :, 0]
    assert np.allclose(r1, r1[:1, :]) and not np.allclose(r1, r1[:, :1])
    # k = m is (k_x = 0, k_y = 1): ratio f_1(y)/f_0(y), free of x
    rm = grid[:, :, m] / grid[:, :, 0]
    assert np.allclose(rm, rm[:, :1]) and not np.allclose(rm, rm[:1, :])
    # with many modes Phi Phi^T approaches sigma^2 exp(-|dx|/l - |dy|/l)
    big = kle.phi_matrix(2, 6, 0.3, 2.0, 400)   # diagonal truncation error ~ 1/m
    c = kle.centroids_1d(6)
    X, Y = np.meshgrid(c, c)
    X, Y = X.reshape(-1), Y.reshape(-1)
    cov = 2.0 * np.exp(-(np.abs(X[:, None] - X[None, :]) + np.abs(Y[:, None] - Y[None, :])) / 0.3)
    assert np.abs(big @ big.T - cov).max() < 1e-2


def test_log_field_sample_variance_matches_truncated_variance():
    dim, n, lam, s2, m = 2, 4, 0.3, 1.0, 4
    xi = philox.draw_xi(0, 0, 0, np.arange(40000), m * m)
    g = kle.log_field(dim, n, lam, s2, m, xi)
    om, th, even = kle.eigenpairs_1d(lam, m)
    f = kle.eigfun_1d(om, even, kle.centroids_1d(n))
    v1 = (th[None, :] * f ** 2).sum(axis=1)           # per-axis truncated variance
    expect = s2 * np.outer(v1, v1).reshape(-1)          # [iy, ix] flattened, x fastest
    assert np.allclose(g.var(axis=0), expect, rtol=3e-2)
    assert np.abs(g.mean(axis=0)).max() < 3e-2


def test_3d_tensor_index_order():
    phi = kle.phi_matrix(3, 4, 0.2, 1.0, 2).reshape(4, 4, 4, 8)   # [iz, iy, ix, k]
    r = phi / phi[..., :1]
    assert np.allclose(r[..., 1], r[:1, :1, :, 1])    # k = 1: k_x = 1, depends on x only
    assert np.allclose(r[..., 2], r[:1, :, :1, 2])    # k = 2: k_y = 1, y only
    assert np.allclose(r[..., 4], r[:, :1, :1, 4])    # k = 4: k_z = 1, z only


# ---------------------------------------------------- total-order truncation

@pytest.mark.parametrize("dim,m,K", [(2, 4, 0), (2, 4, 2), (2, 4, 3), (2, 6, 8), (3, 3, 1),
                                     (3, 5, 4), (3, 5, 7), (3, 7, 12)])
def test_total_order_count(dim, m, K):
    brute = sum(1 for k in itertools.product(range(m), repeat=dim) if sum(k) <= K)
    assert kle.n_modes(dim, m, K) == brute
    if K < m:
        assert brute == math.comb(K + dim, dim)
    assert kle.n_modes(dim, m, None) == m ** dim == kle.n_modes(dim, m, -1)


def test_total_order_680_modes():
    # 16 eigenfunctions per axis, 3D, sum of 0-based orders <= 14
    assert kle.n_modes(3, 16, 14) == 680


@pytest.mark.parametrize("dim,m,K,n", [(2, 5, 3, 12), (3, 4, 2, 5)])
def test_truncated_field_is_full_field_with_dropped_coefficients_zero(dim, m, K, n):
    rng = np.random.default_rng(4)
    full = kle.mode_indices(dim, m)
    kept = kle.mode_indices(dim, m, K)
    M = len(kept)
    xi = rng.standard_normal((3, M))
    # scatter into the full basis by matching per-axis indices
    pos = {tuple(k): i for i, k in enumerate(full)}
    xf = np.zeros((3, len(full)))
    for t, k in enumerate(kept):
        xf[:, pos[tuple(k)]] = xi[:, t]
    g_t = kle.log_field(dim, n, 0.2, 1.3, m, xi, K)
    g_f = kle.log_field(dim, n, 0.2, 1.3, m, xf)
    assert np.max(np.abs(g_t - g_f)) <= 1e-13 * np.max(np.abs(g_f))
    # kept modes in the full basis' flat order, sums within the bound
    assert all(sum(k) <= K for k in kept)
    flat = [pos[tuple(k)] for k in kept]
    assert flat == sorted(flat)


def test_truncated_pointwise_variance_is_kept_mercer_sum():
    dim, m, K, n, lam, s2 = 2, 8, 5, 10, 0.15, 1.7
    phi = kle.phi_matrix(dim, n, lam, s2, m, K)
    omega, theta, even = kle.eigenpairs_1d(lam, m)
    f = kle.eigfun_1d(omega, even, kle.centroids_1d(n))
    var = np.zeros((n, n))
    for kx, ky in kle.mode_indices(dim, m, K):
        var += s2 * theta[kx] * theta[ky] * np.outer(f[:, ky] ** 2, f[:, kx] ** 2)
    assert np.allclose((phi ** 2).sum(axis=1), var.reshape(-1), rtol=1e-12, atol=0)
