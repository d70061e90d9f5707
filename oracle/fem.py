"""Oracle: Q1 finite elements for -div(kappa grad u) = f, u = 0 on the boundary.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (model) of Sec. 2.1 on the unit square (d = 2) or cube (d = 3) with
homogeneous Dirichlet data, discretised with a C0 Lagrangian (Q1) space on a
uniform grid of n cells per side (Sec. 2.2: h_l = h_0 s^-l, s = 2).
Readings fixed here:

* kappa is constant per element (its value at the centroid), so the element
  matrices are exact without quadrature: K_e = kappa_e K_ref with K_ref the
  tensor sum of the 1D stiffness k = (1/h)[[1,-1],[-1,1]] and mass
  m = (h/6)[[2,1],[1,2]] matrices;
* unknowns are the interior nodes, lexicographic, x fastest;
* load b_i = int f phi_i, exact for f = 1 (b_i = h^d) and by a 2-point Gauss
  rule per axis for a general f (manufactured-solution checks only);
* QoI (Sec. 2.1, "an integral of u on a sub-region") = the exact integral
  mean of the Q1 function u_h over the whole domain or over a node-aligned
  box, Q = w^T u with w_i = int_box phi_i / |box|;
* the solve is the plain definition u = A^{-1} b (sparse direct
  factorisation); ``pcg_jacobi`` is the Jacobi-preconditioned CG used for the
  CG-vs-direct pin and for timing.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _k1(h):
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


def _m1(h):
    return np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)


def element_stiffness(dim, h):
    """Reference Q1 stiffness (kappa = 1) on a cube of side h, 2^d x 2^d.

    Local vertex v has bits (v_x, v_y[, v_z]) = (v & 1, (v >> 1) & 1, ...):
    K[a, b] = sum_ax k[a_ax, b_ax] prod_{other} m[a_o, b_o].
    """
    k, m = _k1(h), _m1(h)
    nv = 2 ** dim
    K = np.zeros((nv, nv))
    for a in range(nv):
        for b in range(nv):
            tot = 0.0
            for ax in range(dim):
                term = 1.0
                for o in range(dim):
                    ao, bo = (a >> o) & 1, (b >> o) & 1
                    term *= k[ao, bo] if o == ax else m[ao, bo]
                tot += term
            K[a, b] = tot
    return K


def n_interior(dim, n):
    return (n - 1) ** dim


def _node_id(dim, n, node):
    """Interior index of grid node (tuple of ints 0..n) or -1 on the boundary."""
    idx = 0
    stride = 1
    for c in node:
        if c <= 0 or c >= n:
            return -1
        idx += (c - 1) * stride
        stride *= (n - 1)
    return idx


def _elements(dim, n):
    """All elements as integer corner tuples (lower-left-front), x fastest."""
    grids = np.meshgrid(*([np.arange(n)] * dim), indexing='ij')
    return np.stack([g.reshape(-1) for g in grids][::-1], axis=1)


def assemble(dim, n, kappa):
    """Global stiffness over interior nodes, element by element (CSR).

    kappa: per-element values, length n^dim, x fastest.
    """
    h = 1.0 / n
    K = element_stiffness(dim, h)
    kappa = np.asarray(kappa, dtype=np.float64).reshape(-1)
    assert kappa.size == n ** dim
    rows, cols, vals = [], [], []
    nv = 2 ** dim
    for e, corner in enumerate(_elements(dim, n)):
        ids = []
        for v in range(nv):
            node = tuple(int(corner[ax]) + ((v >> ax) & 1) for ax in range(dim))
            ids.append(_node_id(dim, n, node))
        for a in range(nv):
            if ids[a] < 0:
                continue
            for b in range(nv):
                if ids[b] < 0:
                    continue
                rows.append(ids[a])
                cols.append(ids[b])
                vals.append(kappa[e] * K[a, b])
    N = n_interior(dim, n)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def assemble_fast(dim, n, kappa):
    """Same matrix as ``assemble`` built with vectorised index arithmetic.

    Used for meshes where the element loop in Python is too slow; a test
    checks that both give identical matrices on small meshes.
    """
    h = 1.0 / n
    K = element_stiffness(dim, h)
    kappa = np.asarray(kappa, dtype=np.float64).reshape(-1)
    corners = _elements(dim, n)
    nv = 2 ** dim
    ids = _vertex_ids(dim, n, corners)
    rows = np.repeat(ids, nv, axis=1).reshape(-1)
    cols = np.tile(ids, (1, nv)).reshape(-1)
    vals = (kappa[:, None] * K.reshape(1, -1)).reshape(-1)
    keep = (rows >= 0) & (cols >= 0)
    N = n_interior(dim, n)
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(N, N))


def _vertex_ids(dim, n, corners):
    """Interior ids (or -1 on the boundary) of the 2^d vertices of each element."""
    nv = 2 ** dim
    ids = np.empty((corners.shape[0], nv), dtype=np.int64)
    for v in range(nv):
        node = corners + np.array([(v >> ax) & 1 for ax in range(dim)])[None, :]
        inside = np.all((node > 0) & (node < n), axis=1)
        idx = np.zeros(corners.shape[0], dtype=np.int64)
        stride = 1
        for ax in range(dim):
            idx += (node[:, ax] - 1) * stride
            stride *= (n - 1)
        ids[:, v] = np.where(inside, idx, -1)
    return ids


def load_vector(dim, n, f=None):
    """b_i = int f phi_i, assembled element by element.

    f = None means f = 1, integrated exactly: int_e phi_v = |e| / 2^d for
    each vertex v of element e. For a callable f the integral uses 2 Gauss
    points per axis per element.
    """
    h = 1.0 / n
    N = n_interior(dim, n)
    corners = _elements(dim, n)
    ids = _vertex_ids(dim, n, corners)
    nv = 2 ** dim
    b = np.zeros(N)
    if f is None:
        for v in range(nv):
            keep = ids[:, v] >= 0
            np.add.at(b, ids[keep, v], h ** dim / nv)
        return b
    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    for q in range(2 ** dim):
        ref = np.array([gp[(q >> ax) & 1] for ax in range(dim)])
        pts = (corners + ref[None, :]) * h
        fval = f(*[pts[:, ax] for ax in range(dim)]) * (h ** dim) / (2 ** dim)
        for v in range(nv):
            shape = np.prod([ref[ax] if (v >> ax) & 1 else 1.0 - ref[ax]
                             for ax in range(dim)])
            keep = ids[:, v] >= 0
            np.add.at(b, ids[keep, v], fval[keep] * shape)
    return b


def qoi_weights(dim, n, kind='domain', box=(0.25, 0.75)):
    """w with Q = w^T u = (1 / |R|) int_R u_h, R the domain or a box.

    For each element inside R add int_e phi_v = h^d / 2^d to each interior
    vertex; the box must be node-aligned (its faces on grid planes).
    """
    h = 1.0 / n
    N = n_interior(dim, n)
    if kind == 'domain':
        lo, hi = 0, n
        vol = 1.0
    elif kind == 'box':
        lo_f, hi_f = box[0] * n, box[1] * n
        if abs(lo_f - round(lo_f)) > 1e-12 or abs(hi_f - round(hi_f)) > 1e-12:
            raise ValueError("box QoI needs a node-aligned box")
        lo, hi = int(round(lo_f)), int(round(hi_f))
        vol = (box[1] - box[0]) ** dim
    else:
        raise ValueError(kind)
    corners = _elements(dim, n)
    inside_box = np.all((corners >= lo) & (corners < hi), axis=1)
    ids = _vertex_ids(dim, n, corners[inside_box])
    w = np.zeros(N)
    nv = 2 ** dim
    for v in range(nv):
        keep = ids[:, v] >= 0
        np.add.at(w, ids[keep, v], h ** dim / nv)
    return w / vol


def solve_direct(A, b, refine=2):
    """u = A^{-1} b by sparse LU (SuperLU); the plain definition of the solve.

    ``refine`` steps of fixed-precision iterative refinement
    (u += LU^{-1}(b - A u)) take the backward error of the pivoted LU down to
    the level the conditioning allows.
    """
    lu = spla.splu(A.tocsc())
    u = lu.solve(b)
    for _ in range(refine):
        u = u + lu.solve(b - A @ u)
    return u


def solve(A, b, dim):
    """u = A^{-1} b: sparse LU while its fill-in is affordable (2D up to
    3e5 unknowns, 3D up to 3e4), otherwise the Jacobi-PCG below to
    ||r|| <= 1e-13 ||b|| (far below any tolerance the device solves use)."""
    limit = 300000 if dim == 2 else 30000
    if A.shape[0] <= limit:
        return solve_direct(A, b)
    return pcg_jacobi(A, b, rtol=1e-13)[0]


def pcg_jacobi(A, b, rtol, max_iter=100000, callback=None):
    """Textbook Jacobi-preconditioned CG from x0 = 0.

    Stops when ||r_k||_2 <= rtol ||b||_2. Returns (x, iterations).
    ``callback(x)`` sees every iterate.
    """
    d = A.diagonal()
    x = np.zeros_like(b)
    r = b.copy()
    z = r / d
    p = z.copy()
    rz = r @ z
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    for it in range(1, max_iter + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if callback is not None:
            callback(x)
        if np.linalg.norm(r) <= rtol * bnorm:
            return x, it
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise RuntimeError("PCG did not converge")


def to_node_grid(dim, n, u_interior):
    """Interior vector -> full (n+1)^dim node array (boundary zeros), x fastest."""
    full = np.zeros((n + 1,) * dim)
    full[(slice(1, n),) * dim] = np.asarray(u_interior).reshape((n - 1,) * dim)
    return full.reshape(-1)


def from_node_grid(dim, n, full):
    """(n+1)^dim node array (x fastest) -> interior vector."""
    return np.asarray(full).reshape((n + 1,) * dim)[(slice(1, n),) * dim].reshape(-1)
