"""Pins for the oracle's MLMC layer (oracle/mlmc.py).

Pins: Welford equals the two-pass 1/N variance of Eq. (sample_variance);
Chan merges of any partition equal the whole; the allocation of Eq.
(mlmc_num_samples) on a hand-computed example and its defining property
sum V_l / N_l <= eps^2 / 2; Table 1 against Eq. (sample_scaling); the
coupling (both meshes of a pair see xi(l, i)); the telescoping identity of
Eq. (mlmc_average); level variances decay with the mesh (Sec. 2.2).
Adaptive L (Sec. 2.3, Eq. (mlmc_num_levels)): the bias fit recovers (alpha,
c) from level means built as differences of Q_l = Q + c 2^(-alpha l); the
level rule returns the smallest L with c 2^(-alpha L) <= eps / sqrt(2) (brute
force); the adaptive run on a synthetic sampler with a known bias ends with
both the bias and the statistical error within their eps^2 / 2 shares, and
reduces to the fixed-L run when it starts on every level.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fem, kle, mlmc, philox
from synth import small_case

GOLD = os.path.join(os.path.dirname(__file__), 'golden')


def test_welford_matches_two_pass():
    rng = np.random.default_rng(1)
    y = rng.standard_normal(1000) * 1e-3 + 0.04
    w = mlmc.Welford()
    for v in y:
        w.add(v)
    assert w.n == 1000
    assert abs(w.mean - y.mean()) <= 1e-15
    assert abs(w.var() - np.mean((y - y.mean()) ** 2)) <= 1e-13 * y.var()


def test_chan_merge_any_partition():
    rng = np.random.default_rng(2)
    y = rng.standard_normal(257)
    full = mlmc.Welford()
    for v in y:
        full.add(v)
    for cuts in ([0, 1, 257], [0, 100, 101, 257], [0, 64, 128, 192, 256, 257]):
        acc = mlmc.Welford()
        for a, b in zip(cuts[:-1], cuts[1:]):
            part = mlmc.Welford()
            for v in y[a:b]:
                part.add(v)
            acc = mlmc.chan_merge(acc, part)
        assert acc.n == full.n
        assert abs(acc.mean - full.mean) <= 1e-14
        assert abs(acc.m2 - full.m2) <= 1e-14 * full.m2


def test_allocation_hand_example_and_property():
    g = json.load(open(os.path.join(GOLD, 'allocation_hand_example.json')))
    assert mlmc.allocate(g['V'], g['C'], g['eps']) == g['N']
    rng = np.random.default_rng(3)
    for _ in range(50):
        V = rng.random(5) * 10.0 ** -rng.integers(1, 8, 5)
        C = rng.random(5) * 10.0 ** rng.integers(0, 6, 5)
        eps = 10.0 ** -rng.uniform(1, 4)
        N = mlmc.allocate(V, C, eps)
        assert sum(v / n for v, n in zip(V, N)) <= eps ** 2 / 2 * (1 + 1e-12)


def test_table1_matches_sample_scaling():
    g = json.load(open(os.path.join(GOLD, 'table1_sample_sizes.json')))
    N = g['N_star']
    ratio = math.exp(g['Gamma'] * math.log(g['s']))
    assert abs(ratio - 16.0) < 1e-12
    assert N[0] / N[1] == 16 and N[1] / N[2] == 16


def test_coupling_uses_same_xi_on_both_meshes():
    cfg = small_case(2)
    M = cfg['m'] ** 2
    qf, qc = mlmc.coupled_sample(cfg, 2, 5)
    xi = philox.draw_xi(cfg['seed'], 0, 2, [5], M)[0]
    assert qf == mlmc.solve_qoi(cfg, 2, xi)
    assert qc == mlmc.solve_qoi(cfg, 1, xi)
    # the fine solve of level 1, sample 5, has its own xi(1, 5)
    assert mlmc.coupled_sample(cfg, 1, 5)[0] != qc
    assert mlmc.coupled_sample(cfg, 0, 5)[1] == 0.0


def test_telescoping_identity():
    """With xi keyed by i only, sum_l Y_l^i = Q_L^i, so the MLMC mean = MC mean on level L."""
    cfg = small_case(2)
    M = cfg['m'] ** 2
    L1 = cfg['levels']
    N = 6

    def sampler(level, i):
        xi = philox.draw_xi(cfg['seed'], 0, 0, [i], M)[0]     # level-free key (test only)
        qf = mlmc.solve_qoi(cfg, level, xi)
        qc = mlmc.solve_qoi(cfg, level - 1, xi) if level > 0 else 0.0
        return qf, qc

    states = [mlmc.Welford() for _ in range(L1)]
    fine = []
    for i in range(N):
        ys = []
        for l in range(L1):
            qf, qc = sampler(l, i)
            states[l].add(qf - qc)
            ys.append(qf - qc)
        fine.append(mlmc.solve_qoi(cfg, L1 - 1, philox.draw_xi(cfg['seed'], 0, 0, [i], M)[0]))
        assert abs(sum(ys) - fine[-1]) <= 1e-15
    q, _ = mlmc.estimate(states)
    assert abs(q - np.mean(fine)) <= 1e-13 * abs(q)


def test_level_variance_decays():
    """V(Y_l) shrinks with h (O(h^4) for this functional, Sec. 2.2)."""
    cfg = small_case(2, n0=4, levels=4, corr_len=0.3)
    V = []
    for l in range(1, 4):
        s = mlmc.Welford()
        for i in range(24):
            qf, qc = mlmc.coupled_sample(cfg, l, i)
            s.add(qf - qc)
        V.append(s.var())
    assert V[0] > 4 * V[1] > 16 * V[2] > 0


def test_run_reaches_statistical_tolerance():
    cfg = small_case(2, n0=4, levels=3)
    q, v, states, qs = mlmc.run(cfg, eps=2e-3, pilot=10)
    assert v <= (2e-3) ** 2 / 2 * (1 + 1e-12)
    assert all(s.n >= 10 for s in states)
    assert abs(q - sum(np.mean([a - b for a, b in lvl]) for lvl in qs)) < 1e-15


def test_cost_model():
    cfg = small_case(3, n0=2, levels=3)
    assert mlmc.level_cost(cfg, 0) == 1
    assert mlmc.level_cost(cfg, 1) == 27 + 1
    assert mlmc.level_cost(cfg, 2) == 343 + 27


# ---------------------------------------------------------- adaptive L

def model_means(q_inf, c, alpha, L):
    """Level means of Y_0 = Q_0, Y_l = Q_l - Q_{l-1} for Q_l = q_inf + c 2^(-alpha l)."""
    Q = [q_inf + c * 2.0 ** (-alpha * l) for l in range(L + 1)]
    return [Q[0]] + [Q[l] - Q[l - 1] for l in range(1, L + 1)]


@pytest.mark.parametrize("alpha,c,q_inf", [(2.0, 0.3, 0.7), (1.0, 5e-3, 0.7), (1.37, 2.0, 0.7),
                                           (3.5, 1e-4, 0.0)])
def test_bias_fit_recovers_rate_and_constant(alpha, c, q_inf):
    # (q_inf = 0 where the differences would lose digits to cancellation)
    a, cc = mlmc.fit_bias(model_means(q_inf, c, alpha, 5))
    assert abs(a - alpha) < 1e-10 and abs(cc - c) < 1e-10 * c


def test_bias_fit_single_level_uses_default_rate_and_clamps():
    # one difference level: the default rate, c from that level
    a, c = mlmc.fit_bias(model_means(1.0, 0.2, 2.0, 1))
    assert a == mlmc.ALPHA_DEFAULT and abs(c - 0.2) < 1e-12
    # a mean that grows with l (noise) is clamped to the smallest rate
    a, _ = mlmc.fit_bias([1.0, 1e-3, 4e-3, 1.6e-2])
    assert a == mlmc.ALPHA_RANGE[0]
    assert mlmc.fit_bias([1.0]) == (None, None)


def test_level_rule_is_smallest_level_meeting_bias_share():
    rng = np.random.default_rng(3)
    for _ in range(500):
        alpha = rng.uniform(0.5, 4.0)
        c = 10 ** rng.uniform(-4, 1)
        eps = 10 ** rng.uniform(-5, -1)
        L = mlmc.num_levels(alpha, c, eps)
        ok = [l for l in range(-60, 200) if c * 2.0 ** (-alpha * l) <= eps / math.sqrt(2.0)]
        brute = min(ok)
        # equal unless the bias sits on the boundary to rounding
        if L != brute:
            edge = c * 2.0 ** (-alpha * brute) / (eps / math.sqrt(2.0))
            assert abs(edge - 1.0) < 1e-12
        assert c * 2.0 ** (-alpha * L) <= eps / math.sqrt(2.0) * (1 + 1e-12)


def synthetic_sampler(q_inf, c, alpha, noise, seed=0):
    """Coupled pairs with a known bias c 2^(-alpha l) and noise shrinking with l."""
    def sample(level, i):
        r = np.random.default_rng([seed, level, i]).standard_normal(2)
        qf = q_inf + c * 2.0 ** (-alpha * level) + noise * r[0] + noise * 2.0 ** (-level) * r[1]
        if level == 0:
            return qf, 0.0
        qc = q_inf + c * 2.0 ** (-alpha * (level - 1)) + noise * r[0]
        return qf, qc
    return sample


@pytest.mark.parametrize("eps", [3e-3, 1e-3, 3e-4])
def test_adaptive_levels_meet_both_error_shares(eps):
    cfg = dict(dim=2, n0=4, levels=9)
    q_inf, c, alpha = 0.5, 0.2, 2.0
    q, v, states, L = mlmc.run_adaptive_levels(
        cfg, eps, pilot=20, L0=2, sampler=synthetic_sampler(q_inf, c, alpha, 0.01))
    # the bias at the final level is within its share (up to the fit's noise)
    assert c * 2.0 ** (-alpha * L) <= eps / math.sqrt(2.0) * 1.5
    assert L < 8 and L >= 2
    assert v <= eps ** 2 / 2 * (1 + 1e-12)
    assert all(s.n == 0 for s in states[L + 1:])
    assert abs(q - q_inf) < 4 * math.sqrt(v) + c * 2.0 ** (-alpha * L)


def test_adaptive_levels_reduce_to_fixed_run_when_starting_on_every_level():
    cfg = small_case(2, n0=4, levels=3)
    smp = synthetic_sampler(0.3, 0.05, 2.0, 0.02, seed=4)
    q1, v1, s1, _ = mlmc.run(cfg, 1e-3, 10, sampler=smp)
    q2, v2, s2, L = mlmc.run_adaptive_levels(cfg, 1e-3, 10, L0=2, sampler=smp)
    assert L == 2 and (q1, v1) == (q2, v2)
    assert [s.n for s in s1] == [s.n for s in s2]
