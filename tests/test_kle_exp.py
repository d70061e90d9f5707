"""The FP64 exp of the KLE kernels (field.cu, Tang's table-driven method,
ACM TOMS 15(2), 1989): the reduction constants written in the CUDA source
and the method as the kernel evaluates it, simulated here in exact rational
arithmetic (every fma rounded once, every product and sum rounded once), stay
within 1 ulp of the correctly rounded exp over the range the log-field of
the KLE reaches and beyond. The GPU side is checked against the oracle's exp
in the kappa parity tests."""
import math
import random
import re
from fractions import Fraction
from pathlib import Path

import pytest

SRC = Path(__file__).resolve().parents[1] / "paper_2111_11788_gb300" / "csrc" / "field.cu"


def _const(text, name):
    m = re.search(r"constexpr double %s = ([^;]+);" % name, text)
    assert m, name
    tok = m.group(1).strip()
    return float.fromhex(tok) if tok.startswith("0x") else float(tok)


@pytest.fixture(scope="module")
def consts():
    text = SRC.read_text()
    return _const(text, "kInvLn2x64"), _const(text, "kLn2d64Hi"), _const(text, "kLn2d64Lo")


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _rint(x):
    # round half to even, as rint in the default rounding mode
    return float(round(x))


def kle_exp_sim(x, inv, hi, lo, tab):
    nf = _rint(x * inv)
    N = int(nf)
    r = _fma(-nf, lo, _fma(-nf, hi, x))
    j = N & 63
    k = (N - j) >> 6
    q = _fma(r, _fma(r, _fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5)
    p = _fma(r * r, q, r)
    T = tab[j]
    return _fma(T, p, T) * math.ldexp(1.0, k)


def _exact_exp(x):
    # exp to ~30 digits with the decimal module (correctly rounded reference)
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    return float(Decimal(x).exp())


def _ulp_err(a, ref):
    return abs(a - ref) / math.ulp(ref)


def test_split_of_ln2_over_64(consts):
    inv, hi, lo = consts
    ln2_64 = Fraction(6931471805599453094172321214581765680755, 10 ** 40) / 64
    # hi carries at most 32 significant bits, so N * hi is exact for |N| < 2^21
    m, e = math.frexp(hi)
    assert (Fraction(m) * 2 ** 32).denominator == 1
    # hi + lo is ln2 / 64 to within half an ulp of lo (about 2^-92)
    assert abs(Fraction(hi) + Fraction(lo) - ln2_64) <= Fraction(math.ulp(lo)) / 2
    assert abs(inv - 64 / math.log(2)) <= math.ulp(inv)


def test_within_one_ulp(consts):
    inv, hi, lo = consts
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    tab = [float((Decimal(j) / 64 * Decimal(2).ln()).exp()) for j in range(64)]
    rng = random.Random(7)
    xs = [rng.uniform(-12.0, 12.0) for _ in range(3000)] + [rng.uniform(-700.0, 700.0) for _ in range(500)]
    xs += [0.0, 1e-300, -1e-300, math.log(2) / 128, -math.log(2) / 128, 1.0, -1.0]
    worst = 0.0
    for x in xs:
        worst = max(worst, _ulp_err(kle_exp_sim(x, inv, hi, lo, tab), _exact_exp(x)))
    assert worst <= 1.0, worst
