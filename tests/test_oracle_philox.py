"""Pins for the oracle's counter-based normals (oracle/philox.py).

The paper names no generator, so nothing here comes from it. The pins are:
an independent Philox4x32-10 implementation (Triton's, run in its CPU
interpreter), the mathematical functions against arbitrary-precision values,
and the distribution of the normals against N(0, 1).
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import philox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_philox_matches_triton_library():
    """Oracle Philox4x32-10 == triton.language.random.philox (CPU interpreter).

    This is the generator's only pin by an independent implementation, so a
    missing Triton or interpreter fails the test instead of skipping it."""
    code = textwrap.dedent("""
        import numpy as np, torch, triton, triton.language as tl, sys
        from triton.language.random import philox as tphilox
        @triton.jit
        def k(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
            o = tl.arange(0, N)
            a, b, c, d = tphilox(seed, tl.load(c0p + o), tl.load(c1p + o),
                                 tl.load(c2p + o), tl.load(c3p + o))
            tl.store(out + 4 * o, a); tl.store(out + 4 * o + 1, b)
            tl.store(out + 4 * o + 2, c); tl.store(out + 4 * o + 3, d)
        sys.path.insert(0, %r)
        from oracle.philox import philox4x32_10
        N = 64
        rng = np.random.default_rng(7)
        ok = True
        for seed in (0, 1, 0x0123456789ABCDEF, 2**64 - 1):
            cs = [rng.integers(0, 2**32, N, dtype=np.uint64) for _ in range(4)]
            cs[0][:4] = [0, 1, 2**32 - 1, 5]
            ts = [torch.from_numpy(c.astype(np.uint32).view(np.int32).copy()) for c in cs]
            out = torch.zeros(4 * N, dtype=torch.int32)
            k[(1,)](out, *ts, seed, N=N)
            got = out.numpy().view(np.uint32).reshape(N, 4).astype(np.uint64)
            ref = philox4x32_10(*cs, seed & 0xFFFFFFFF, seed >> 32)
            ok &= all(bool((got[:, i] == ref[i]).all()) for i in range(4))
        print("MATCH" if ok else "MISMATCH")
    """ % ROOT)
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                         text=True, timeout=600)
    assert res.returncode == 0, "triton interpreter run failed: " + res.stderr[-600:]
    assert "MATCH" in res.stdout and "MISMATCH" not in res.stdout


def test_uniform52_range_and_exactness():
    w = np.array([0, 0xFFFFFFFF, 0x80000000, 12345], dtype=np.uint64)
    u = philox.uniform52(w, w[::-1])
    assert np.all(u > 0) and np.all(u < 1)
    assert philox.uniform52(0, 0) == 2.0 ** -53
    assert philox.uniform52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53


def test_ln_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(3)
    u = np.concatenate([rng.random(3000), [2.0 ** -53, 1 - 2.0 ** -53, 0.5,
                                            np.sqrt(0.5), np.nextafter(np.sqrt(0.5), 1)]])
    u = u[u > 0]
    got = philox.ln(u)
    exact = np.array([float(mp.log(mp.mpf(float(x)))) for x in u])
    err_ulp = np.abs(got - exact) / np.spacing(np.abs(exact) + 1e-300)
    err_ulp[exact == 0] = np.abs(got[exact == 0]) / 2.0 ** -1074
    assert err_ulp.max() <= 4.0


def test_sincos_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(4)
    u = np.concatenate([rng.random(3000), [0.125, 0.25, 0.375, 0.5, 0.625, 0.75,
                                            0.875, 2.0 ** -53, 1 - 2.0 ** -53]])
    c, s = philox.sincos_2pi(u)
    ce = np.array([float(mp.cos(2 * mp.pi * mp.mpf(float(x)))) for x in u])
    se = np.array([float(mp.sin(2 * mp.pi * mp.mpf(float(x)))) for x in u])
    # absolute error in units of 2^-53 (the angle reduction is exact, so the
    # error is that of a few rounded products on values of magnitude <= 1)
    assert np.abs(c - ce).max() <= 3 * 2.0 ** -53
    assert np.abs(s - se).max() <= 3 * 2.0 ** -53
    # quadrant points are exact
    c0, s0 = philox.sincos_2pi(np.array([0.25, 0.5, 0.75]))
    assert np.array_equal(c0, [0.0, -1.0, 0.0]) and np.array_equal(s0, [1.0, 0.0, -1.0])


def test_normals_distribution():
    """xi ~ N(0,1): moments and a Kolmogorov-Smirnov test over 10^6 draws."""
    stats = pytest.importorskip("scipy.stats")
    xi = philox.draw_xi(seed=0, stream_id=0, level=2, samples=np.arange(31250),
                        n_modes=32).reshape(-1)
    assert xi.size == 10 ** 6
    assert abs(xi.mean()) < 5e-3
    assert abs(xi.var() - 1.0) < 5e-3
    assert abs(np.mean(xi ** 4) - 3.0) < 3e-2
    assert stats.kstest(xi, 'norm').pvalue > 1e-3


def test_normals_independence_across_modes_samples_levels():
    xi = philox.draw_xi(0, 0, 0, np.arange(20000), 8)
    c = np.corrcoef(xi.T)
    assert np.abs(c - np.eye(8)).max() < 0.04
    a = philox.draw_xi(0, 0, 0, np.arange(20000), 2)[:, 0]
    b = philox.draw_xi(0, 0, 1, np.arange(20000), 2)[:, 0]
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.04
    lag = philox.draw_xi(0, 0, 0, np.arange(20001), 1)[:, 0]
    assert abs(np.corrcoef(lag[:-1], lag[1:])[0, 1]) < 0.04


def test_addressing_is_counter_based():
    """xi(l, i) depends only on (seed, stream, l, i), not on the batch it is drawn in."""
    all_ = philox.draw_xi(5, 3, 4, np.arange(100), 17)
    part = philox.draw_xi(5, 3, 4, np.arange(40, 60), 17)
    assert np.array_equal(all_[40:60], part)
    # odd M drops the last sine branch: prefix property across M
    assert np.array_equal(philox.draw_xi(5, 3, 4, [7], 16)[0],
                          philox.draw_xi(5, 3, 4, [7], 17)[0][:16])
    assert not np.array_equal(philox.draw_xi(5, 3, 4, [7], 4), philox.draw_xi(5, 3, 3, [7], 4))
    assert not np.array_equal(philox.draw_xi(5, 3, 4, [7], 4), philox.draw_xi(6, 3, 4, [7], 4))
    assert not np.array_equal(philox.draw_xi(5, 3, 4, [7], 4), philox.draw_xi(5, 2, 4, [7], 4))
