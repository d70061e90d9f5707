"""Oracle: Karhunen-Loeve expansion of the lognormal diffusion coefficient.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 5.2 describes the coefficient as kappa = exp(g) with g a zero-mean
Gaussian field of exponential covariance, expanded in eigenfunctions "in
each dimension" and combined by a tensor product. Readings fixed here:

* covariance C(x, y) = sigma^2 prod_a exp(-|x_a - y_a| / lambda) on [0, 1]^d
  (lambda = correlation length, no factor 2);
* 1D eigenpairs of c(s, t) = exp(-|s - t| / lambda) on [0, 1] in closed form
  (Ghanem & Spanos, ref. [ghanem1991], Sec. 2.3): with c = 1/lambda,
  a = 1/2 and t = x - 1/2,
    even mode:  c - w tan(w a) = 0,  f(t) = cos(w t) / sqrt(a + sin(2wa)/(2w))
    odd mode:   w + c tan(w a) = 0,  f(t) = sin(w t) / sqrt(a - sin(2wa)/(2w))
    eigenvalue  theta = 2c / (w^2 + c^2);
  modes ordered by increasing w (decreasing theta): mode n has its root in
  (n pi, (n + 1) pi) and is even for even n, odd for odd n;
* full tensor basis of m modes per axis, M = m^d, flat index
  k = (k_z m + k_y) m + k_x (k_x fastest), eigenvalue sigma^2 prod theta;
* g evaluated at element centroids, kappa = exp(g) constant per element.
"""
import numpy as np


def _bisect(fun, lo, hi, iters=200):
    """Plain bisection for a sign change of ``fun`` on [lo, hi]."""
    flo = fun(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        fm = fun(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def eigenpairs_1d(corr_len, m):
    """First m eigenpairs of exp(-|s-t|/corr_len) on [0, 1].

    Returns (omega[m], theta[m], is_even[m]). The transcendental equations
    are written without tan (multiplied through by cos(w a)) so each root is
    the unique sign change of a smooth function on (n pi, (n + 1) pi).
    """
    c = 1.0 / corr_len
    a = 0.5
    omega = np.empty(m)
    even = np.empty(m, dtype=bool)
    for n in range(m):
        lo, hi = n * np.pi, (n + 1) * np.pi
        if n % 2 == 0:
            fun = lambda w: c * np.cos(w * a) - w * np.sin(w * a)
        else:
            fun = lambda w: w * np.cos(w * a) + c * np.sin(w * a)
        omega[n] = _bisect(fun, lo, hi)
        even[n] = (n % 2 == 0)
    theta = 2.0 * c / (omega ** 2 + c ** 2)
    return omega, theta, even


def eigfun_1d(omega, even, x):
    """Normalised eigenfunctions f_n(x) on [0, 1]; shape (len(x), len(omega))."""
    a = 0.5
    t = np.asarray(x, dtype=np.float64)[:, None] - a
    w = omega[None, :]
    norm_even = np.sqrt(a + np.sin(2 * w * a) / (2 * w))
    norm_odd = np.sqrt(a - np.sin(2 * w * a) / (2 * w))
    return np.where(even[None, :], np.cos(w * t) / norm_even, np.sin(w * t) / norm_odd)


def centroids_1d(n):
    """Element centroids (i + 1/2) h, h = 1/n, of a uniform grid of n cells."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def mode_indices(dim, m, total_order=None):
    """Per-axis mode indices of flat mode k (k_x fastest); shape (M, dim).

    total_order K (Sec. 5.2, "total-order basis"): keep only the modes with
    k_x + k_y (+ k_z) <= K, in the same flat order; None or K < 0 keeps the
    full tensor basis (M = m^dim)."""
    grids = np.meshgrid(*([np.arange(m)] * dim), indexing='ij')
    # grids[0] varies slowest in C order -> reverse so axis 0 is x (fastest)
    flat = [g.reshape(-1) for g in grids]
    kidx = np.stack(flat[::-1], axis=1)
    if total_order is not None and total_order >= 0:
        kidx = kidx[kidx.sum(axis=1) <= total_order]
    return kidx


def phi_matrix(dim, n, corr_len, sigma2, m, total_order=None):
    """Dense Phi[e, k] = sqrt(sigma^2 prod_a theta_{k_a}) prod_a f_{k_a}(c_a(e)).

    Elements e are in lexicographic order, x fastest; c(e) is the centroid.
    Shape (n^dim, M) with M modes as chosen by ``mode_indices``.
    """
    omega, theta, even = eigenpairs_1d(corr_len, m)
    f = eigfun_1d(omega, even, centroids_1d(n))            # (n, m)
    kidx = mode_indices(dim, m, total_order)               # (M, dim)
    lam = sigma2 * np.prod(theta[kidx], axis=1)             # (M,)
    cells = np.stack([g.reshape(-1) for g in
                      np.meshgrid(*([np.arange(n)] * dim), indexing='ij')][::-1], axis=1)
    phi = np.ones((cells.shape[0], kidx.shape[0]))
    for ax in range(dim):
        phi *= f[cells[:, ax]][:, kidx[:, ax]]
    return phi * np.sqrt(lam)[None, :]


def log_field(dim, n, corr_len, sigma2, m, xi, total_order=None):
    """g = Phi xi at the element centroids; xi shape (M,) or (B, M) -> (B, n^dim)."""
    phi = phi_matrix(dim, n, corr_len, sigma2, m, total_order)
    xi = np.atleast_2d(xi)
    return xi @ phi.T


def kappa(dim, n, corr_len, sigma2, m, xi, total_order=None):
    """kappa = exp(Phi xi), one value per element (x fastest)."""
    return np.exp(log_field(dim, n, corr_len, sigma2, m, xi, total_order))


def n_modes(dim, m, total_order=None):
    """M: m^dim, or the number of modes of the total-order truncation."""
    return len(mode_indices(dim, m, total_order))
