"""Oracle: counter-based standard normals xi_k(l, i).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper does not name a random number generator; it only needs the
coefficients xi of a sample to be reproducible and independent between
samples, and the MLMC coupling of Eq. (mlmc_average) needs the *same* xi on
both meshes of a level pair. This module fixes the reading used throughout:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 10-round bijection of a 128-bit counter under a
  64-bit key. Round: two 32x32->64 multiplies by 0xD2511F53 (word 0) and
  0xCD9E8D57 (word 2); the new words are (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1,
  lo0). Between rounds the key is bumped by (0x9E3779B9, 0xBB67AE85).
* counter = (j, i, l, stream_id) for the j-th normal pair of sample i on
  level l; key = (seed mod 2^32, seed >> 32).
* uniforms: 52 bits from two output words, u = (x + 1/2) 2^-52, so u lies in
  [2^-53, 1 - 2^-53]: never 0 or 1, and every step is exact in binary64.
* Box-Muller: xi_{2j} = r cos(2 pi u2), xi_{2j+1} = r sin(2 pi u2),
  r = sqrt(-2 ln u1). ``ln``, ``cos`` and ``sin`` are built here from +, -,
  *, /, sqrt, floor and frexp only (no fused multiply-add, no libm), so that
  an independent implementation on another processor that performs the same
  correctly-rounded operations in the same order produces the same bits.
  For odd M the last second normal is discarded.

Parity of xi against the device generator is bit-exact.
"""
import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 of Salmon et al. (SC'11) on arrays of 32-bit words.

    All arguments are broadcastable integer arrays holding values < 2^32.
    Returns the four output words as uint64 arrays (values < 2^32).
    """
    c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & MASK32
                              for v in (c0, c1, c2, c3, k0, k1))
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3, k0, k1 = (v.copy() for v in (c0, c1, c2, c3, k0, k1))
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0          # < 2^64, exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform52(w_hi, w_lo):
    """u = (x + 1/2) 2^-52 with x = (w_hi << 20) | (w_lo >> 12), a 52-bit int.

    x + 1/2 needs 53 significant bits and the scaling is a power of two, so u
    is exact; it lies in [2^-53, 1 - 2^-53].
    """
    x = ((np.asarray(w_hi, np.uint64) << np.uint64(20))
         | (np.asarray(w_lo, np.uint64) >> np.uint64(12)))
    return (x.astype(np.float64) + 0.5) * (2.0 ** -52)


# ln 2 split so that e * LN2_HI is exact for |e| < 2^10 (LN2_HI has 42
# significant bits); LN2_LO is ln 2 - LN2_HI rounded to binary64. Both were
# derived from ln 2 = 0.6931471805599453094172321214581765680755...
LN2_HI = float.fromhex('0x1.62e42fefa3800p-1')
LN2_LO = float.fromhex('0x1.ef35793c76730p-45')
SQRT_HALF = float.fromhex('0x1.6a09e667f3bcdp-1')   # sqrt(1/2) rounded
PIO2 = float.fromhex('0x1.921fb54442d18p+0')        # pi/2 rounded

# ln m = 2 atanh(s) = 2 s sum_k s^(2k) / (2k+1); |s| <= 0.1716 so s^2 <= 0.0295
# and 12 terms (k = 0..11) leave a truncation error below 2^-59 relative.
LOG_COEF = [1.0 / (2 * k + 1) for k in range(12)]
# Taylor coefficients (-1)^k / (2k+1)! and (-1)^k / (2k)! for |x| <= pi/4;
# 11 terms each leave a truncation error below 2^-70.
SIN_COEF = [(-1.0) ** k / float(np.prod(np.arange(1, 2 * k + 2, dtype=np.float64)))
            for k in range(11)]
COS_COEF = [(-1.0) ** k / float(np.prod(np.arange(1, 2 * k + 1, dtype=np.float64)))
            for k in range(11)]


def ln(u):
    """Natural log of u > 0 from exact exponent split + atanh series.

    u = m' 2^e' (frexp, m' in [1/2, 1)); if m' < sqrt(1/2) take m = 2 m',
    e = e' - 1, else m = m', e = e'; so m in [sqrt(1/2), sqrt(2)).
    ln u = e ln 2 + 2 atanh((m - 1) / (m + 1)).
    """
    u = np.asarray(u, dtype=np.float64)
    m, e = np.frexp(u)
    small = m < SQRT_HALF
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    t = s * s
    p = np.full_like(t, LOG_COEF[-1])
    for c in LOG_COEF[-2::-1]:
        p = p * t + c
    lnm = (s * p) * 2.0
    return e * LN2_HI + (e * LN2_LO + lnm)


def sincos_2pi(u):
    """(cos(2 pi u), sin(2 pi u)) for u in (0, 1).

    Exact quadrant reduction: t = 4u, q = floor(t), f = t - q (all exact);
    if f > 1/2 then f -= 1, q += 1, so 2 pi u = q pi/2 + x with x = f pi/2,
    |x| <= pi/4. sin x and cos x by Horner on their Taylor series; the
    quadrant q mod 4 picks and signs the pair.
    """
    u = np.asarray(u, dtype=np.float64)
    t = u * 4.0
    q = np.floor(t)
    f = t - q
    hi = f > 0.5
    f = np.where(hi, f - 1.0, f)
    q = np.where(hi, q + 1.0, q)
    x = f * PIO2
    z = x * x
    ps = np.full_like(z, SIN_COEF[-1])
    for c in SIN_COEF[-2::-1]:
        ps = ps * z + c
    s = x * ps
    pc = np.full_like(z, COS_COEF[-1])
    for c in COS_COEF[-2::-1]:
        pc = pc * z + c
    c = pc
    qi = q.astype(np.int64) & 3
    cos_a = np.select([qi == 0, qi == 1, qi == 2], [c, -s, -c], s)
    sin_a = np.select([qi == 0, qi == 1, qi == 2], [s, c, -s], -c)
    return cos_a, sin_a


def box_muller(u1, u2):
    """Normal pair from two uniforms: r (cos 2 pi u2, sin 2 pi u2), r = sqrt(-2 ln u1)."""
    r = np.sqrt(ln(u1) * -2.0)
    c, s = sincos_2pi(u2)
    return r * c, r * s


def draw_xi(seed, stream_id, level, samples, n_modes):
    """xi[s, k] for sample indices ``samples`` on ``level``; shape (len, n_modes).

    Pair j of sample i comes from Philox counter (j, i, level, stream_id) and
    key (seed mod 2^32, seed >> 32); xi_{2j} from the cosine and xi_{2j+1}
    from the sine branch.
    """
    samples = np.atleast_1d(np.asarray(samples, dtype=np.int64))
    if np.any(samples < 0) or np.any(samples >= 2 ** 32):
        raise ValueError("sample index must lie in [0, 2^32)")
    n_pairs = (n_modes + 1) // 2
    j = np.arange(n_pairs, dtype=np.uint64)[None, :]
    i = samples.astype(np.uint64)[:, None]
    seed = int(seed)
    w0, w1, w2, w3 = philox4x32_10(j, i, np.uint64(level), np.uint64(stream_id),
                                   np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32))
    u1 = uniform52(w0, w1)
    u2 = uniform52(w2, w3)
    a, b = box_muller(u1, u2)
    xi = np.empty((samples.size, 2 * n_pairs), dtype=np.float64)
    xi[:, 0::2] = a
    xi[:, 1::2] = b
    return xi[:, :n_modes]
