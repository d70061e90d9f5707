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
* Sec. 2.3 / Algorithm 2 with L adapted: the discretisation error is modelled
  as |E(Q_l - Q)| = c s^(-alpha l) (s = 2, c absorbing h_0^alpha), so
  |E(Y_l)| = c (s^alpha - 1) s^(-alpha l) for l >= 1; alpha and c are fitted
  from the level means |Ybar_l|, l = 1..L, and Eq. (mlmc_num_levels)
  L = ceil(log_s(sqrt(2) c / eps) / alpha) gives the level that brings the
  bias below eps / sqrt(2). Levels that appear get pilot samples first.
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
    kap = kle.kappa(d, n, cfg['corr_len'], cfg['sigma2'], cfg['m'], xi, cfg.get('total_order'))[0]
    A = fem.assemble_fast(d, n, kap)
    b = fem.load_vector(d, n)
    u = fem.solve(A, b, d)
    w = fem.qoi_weights(d, n, cfg.get('qoi', 'domain'), tuple(cfg.get('box', (0.25, 0.75))))
    return float(w @ u)


def coupled_sample(cfg, level, i):
    """(Q_l, Q_{l-1}) of sample i on level l with shared xi(l, i); Q_{-1} = 0."""
    M = kle.n_modes(cfg['dim'], cfg['m'], cfg.get('total_order'))
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


ALPHA_DEFAULT = 2.0          # the linear-FE rate quoted in Sec. 2.2, used with one difference level
ALPHA_RANGE = (0.5, 4.0)     # clamp of the fitted rate


def fit_bias(means):
    """(alpha, c) of |E(Q_l - Q)| = c 2^(-alpha l) from the level means.

    Least squares of y_l = log2|Ybar_l| = log2(c (2^alpha - 1)) - alpha l over
    the levels l >= 1 with a nonzero mean; alpha clamped to ALPHA_RANGE, then
    the intercept a = mean(y_l + alpha l) and c = 2^a / (2^alpha - 1).
    One usable level: alpha = ALPHA_DEFAULT. None: (None, None)."""
    pts = [(l, math.log2(abs(means[l]))) for l in range(1, len(means)) if means[l] != 0.0]
    if not pts:
        return None, None
    if len(pts) == 1:
        alpha = ALPHA_DEFAULT
    else:
        lbar = sum(l for l, _ in pts) / len(pts)
        ybar = sum(y for _, y in pts) / len(pts)
        sxy = sum((l - lbar) * (y - ybar) for l, y in pts)
        sxx = sum((l - lbar) * (l - lbar) for l, _ in pts)
        alpha = -sxy / sxx
    alpha = min(max(alpha, ALPHA_RANGE[0]), ALPHA_RANGE[1])
    a = sum(y + alpha * l for l, y in pts) / len(pts)
    c = 2.0 ** a / (2.0 ** alpha - 1.0)
    return alpha, c


def num_levels(alpha, c, eps):
    """Eq. (mlmc_num_levels) with s = 2: L = ceil(log2(sqrt(2) c / eps) / alpha)."""
    return int(math.ceil(math.log2(math.sqrt(2.0) * c / eps) / alpha))


def run_adaptive_levels(cfg, eps, pilot, L0, max_rounds=20, sampler=None):
    """Adaptive MLMC with L updated by Eq. (mlmc_num_levels) (Sec. 2.3, Algorithm 2).

    Starts on levels 0..L0; after every sampling phase the sample counts of
    the active levels follow Eq. (mlmc_num_samples) and L grows (never
    shrinks, never beyond the hierarchy) to the level the bias fit asks for;
    new levels get `pilot` samples. Stops when neither changes.
    Returns (q_hat, stat_var, states, L)."""
    sampler = sampler or (lambda l, i: coupled_sample(cfg, l, i))
    Lmax = cfg['levels'] - 1
    L = min(L0, Lmax)
    states = [Welford() for _ in range(Lmax + 1)]
    target = [pilot] * (L + 1) + [0] * (Lmax - L)
    for _ in range(max_rounds):
        for l in range(L + 1):
            while states[l].n < target[l]:
                qf, qc = sampler(l, states[l].n)
                states[l].add(qf - qc)
        V = [states[l].var() for l in range(L + 1)]
        C = [level_cost(cfg, l) for l in range(L + 1)]
        need = allocate(V, C, eps)
        alpha, c = fit_bias([states[l].mean for l in range(L + 1)])
        Lnew = L if alpha is None else min(max(num_levels(alpha, c, eps), L), Lmax)
        more = False
        for l in range(L + 1):
            if need[l] > target[l]:
                target[l] = need[l]
                more = True
        if Lnew > L:
            for l in range(L + 1, Lnew + 1):
                target[l] = pilot
            L = Lnew
            more = True
        if not more:
            break
    q, v = estimate(states[:L + 1])
    return q, v, states, L


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
