"""Oracle: coupled MLMC samples, level statistics, estimator, allocation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Eq. (mlmc_average): Q~_L = sum_l mean(Y_l), Y_0 = Q_0, Y_l = Q_l - Q_{l-1};
  both terms of Y_l^i use the same xi(l, i), each mesh evaluating the field
  at its own element centroids.
* Eq. (sample_variance): V(Y_l) = (1/N_l) sum (Y_l^i - mean)^2, kept as the
  Welford state (n, mean, M2) so that V = M2 / n; states of disjoint sample
  sets merge with Chan's pairwise formula (the partial sums of Algorithm 2,
  reduced at the end).
* Sec. 2.2: estimator variance V(Q~) = sum_l V(Y_l) / N_l, cost
  C_MLMC = sum N_l C_l with C_l the cost of the pair (l, l-1), and the
  allocation of Eq. (mlmc_num_samples)
  N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_i sqrt(V_i C_i)).
  Cost reading: C_l = interior DOFs of mesh l plus of mesh l-1 (a
  deterministic model; the paper measures CPU time).
* Sec. 2.3 / Algorithm 2 with L fixed: pilot samples, then repeat
  {update N_l from the current V_l, C_l; draw the missing samples} until no
  level needs more samples.
"""
import math

import numpy as np

from . import fem, kle, philox


def mesh_cells(cfg, mesh):
    """Cells per side n_mesh = n_0 2^mesh (Sec. 2.2, s = 2)."""
    return cfg['n0'] << mesh


def level_cost(cfg, level):
    """Deterministic cost model C_l = dofs(l) + dofs(l-1) (dofs(-1) = 0)."""
    d = cfg['dim']
    c = fem.n_interior(d, mesh_cells(cfg, level))
    if level > 0:
        c += fem.n_interior(d, mesh_cells(cfg, level - 1))
    return float(c)


def solve_qoi(cfg, mesh, xi):
    """Q(u_mesh) for one coefficient vector xi: kappa, assemble, solve, QoI."""
    d = cfg['dim']
    n = mesh_cells(cfg, mesh)
    kap = kle.kappa(d, n, cfg['corr_len'], cfg['sigma2'], cfg['m'], xi)[0]
    A = fem.assemble_fast(d, n, kap)
    b = fem.load_vector(d, n)
    u = fem.solve(A, b, d)
    w = fem.qoi_weights(d, n, cfg.get('qoi', 'domain'), tuple(cfg.get('box', (0.25, 0.75))))
    return float(w @ u)


def coupled_sample(cfg, level, i):
    """(Q_l, Q_{l-1}) of sample i on level l with shared xi(l, i); Q_{-1} = 0."""
    M = cfg['m'] ** cfg['dim']
    xi = philox.draw_xi(cfg['seed'], cfg.get('stream_id', 0), level, [i], M)[0]
    qf = solve_qoi(cfg, level, xi)
    qc = solve_qoi(cfg, level - 1, xi) if level > 0 else 0.0
    return qf, qc


class Welford:
    """Running (n, mean, M2) with V = M2 / n (Eq. (sample_variance))."""

    def __init__(self, n=0, mean=0.0, m2=0.0):
        self.n, self.mean, self.m2 = n, mean, m2

    def add(self, y):
        self.n += 1
        delta = y - self.mean
        self.mean += delta / self.n
        self.m2 += delta * (y - self.mean)

    def var(self):
        return self.m2 / self.n if self.n > 0 else 0.0


def chan_merge(a, b):
    """Merge two Welford states of disjoint sample sets (Chan et al. 1979)."""
    n = a.n + b.n
    if n == 0:
        return Welford()
    delta = b.mean - a.mean
    mean = a.mean + delta * b.n / n
    m2 = a.m2 + b.m2 + delta * delta * a.n * b.n / n
    return Welford(n, mean, m2)


def allocate(V, C, eps):
    """Eq. (mlmc_num_samples): N_l = ceil(2 eps^-2 sqrt(V_l/C_l) sum_i sqrt(V_i C_i))."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    s = float(np.sum(np.sqrt(V * C)))
    return [int(math.ceil(2.0 / eps ** 2 * math.sqrt(v / c) * s)) for v, c in zip(V, C)]


def estimate(states):
    """Q~ = sum_l mean_l (Eq. (mlmc_average)); V(Q~) = sum_l V_l / N_l (Sec. 2.2)."""
    q = sum(s.mean for s in states)
    v = sum(s.var() / s.n for s in states if s.n > 0)
    return q, v


def run(cfg, eps, pilot, max_rounds=20, sampler=None):
    """Adaptive MLMC with a fixed number of levels (Sec. 2.3, Algorithm 2).

    Returns (q_hat, stat_var, states, per-level lists of (Q_l, Q_{l-1})).
    ``sampler(level, i)`` defaults to ``coupled_sample``.
    """
    sampler = sampler or (lambda l, i: coupled_sample(cfg, l, i))
    L1 = cfg['levels']
    states = [Welford() for _ in range(L1)]
    qs = [[] for _ in range(L1)]
    target = [pilot] * L1
    for _ in range(max_rounds):
        for l in range(L1):
            while states[l].n < target[l]:
                qf, qc = sampler(l, states[l].n)
                qs[l].append((qf, qc))
                states[l].add(qf - qc)
        V = [s.var() for s in states]
        C = [level_cost(cfg, l) for l in range(L1)]
        need = allocate(V, C, eps)
        target = [max(t, nl) for t, nl in zip(target, need)]
        if all(s.n >= t for s, t in zip(states, target)):
            break
    q, v = estimate(states)
    return q, v, states, qs
