"""The streamed bilinear prolongation of the FP32 2D post-smoother
(k_mgpost2f), checked on the CPU against the textbook form.

The kernel forms the field e + P e_c of a warp strip on paired node rows
(2J + 1, 2J + 2), strips starting at rows that are multiples of 32:

  x(i, 2J + 1) = e + (H(J) + H(J + 1)) / 4,   x(i, 2J + 2) = e + H(J + 1) / 2,

H(J) = e_c(J, i // 2) + e_c(J, (i + 1) // 2), with the coarse row sum of
the previous pair carried. The first test replays that schedule (the same
fetch and form order, lanes i = -1 .. n + 1, the pair before the first
output row and the pairs past the last) in float32 and asks for the
textbook value 0.5 (0.5 (a + b) + 0.5 (c + d)) bit for bit at every
interior node and 0 elsewhere, and that every output row reads b and W
(fetched with the field pair one step ahead) of its own row. The second pins the textbook form itself to
bilinear interpolation of the coarse grid (scipy's regular-grid
interpolator) in float64."""
import numpy as np
import pytest

SROWS = 32   # output rows of a strip (the kernel's strip height)

f32 = np.float32


def textbook(e, ec, i, j):
    """e + (P e_c)(i, j) in the arrays' precision, each operation rounded as
    written."""
    T = ec.dtype.type
    a = ec[j >> 1, i >> 1]
    ox, oy = i & 1, j & 1
    v0 = a
    if ox:
        v0 = T(0.5) * T(v0 + ec[j >> 1, (i >> 1) + 1])
    if not oy:
        return T(e[j, i] + v0)
    v1 = ec[(j >> 1) + 1, i >> 1]
    if ox:
        v1 = T(0.5) * T(v1 + ec[(j >> 1) + 1, (i >> 1) + 1])
    return T(e[j, i] + T(0.5) * T(v0 + v1))


def interior(n, i, j):
    return 0 < i < n and 0 < j < n


def strip_fields(n, e, ec, y0):
    """The fields the kernel forms for one strip: {(i, j): x} for every lane
    i = -1 .. n + 1 and every row the strip's window sees."""
    nc, y1 = n // 2, min(y0 + SROWS, n + 1)
    formed = {}
    outputs = strip_fields.outputs = {}
    for c in range(-1, n + 2):
        cin = 1 <= c < n

        def hrow(J):
            if cin and 0 <= J <= nc:
                return f32(ec[J, c >> 1] + ec[J, (c >> 1) + (c & 1)])
            return f32(0.0)

        def fetch(j):
            e0 = e[j, c] if interior(n, c, j) else f32(0.0)
            e1 = e[j + 1, c] if interior(n, c, j + 1) else f32(0.0)
            # the rows whose b and W come with this pair
            return e0, e1, hrow((j + 1) >> 1), (j - 1, j)

        hprev = hrow(y0 // 2 - 1)
        bw = None

        def form(raw, j):
            nonlocal hprev, bw
            e0, e1, h, bw = raw
            x0 = f32(e0 + f32(0.25) * f32(hprev + h)) if interior(n, c, j) else f32(0.0)
            x1 = f32(e1 + f32(0.5) * h) if interior(n, c, j + 1) else f32(0.0)
            hprev = h
            formed[(c, j)] = x0
            formed[(c, j + 1)] = x1

        def out(j):
            # the even output row of a step takes the first of the pair's b, W rows
            outputs[(c, j)] = bw[0] if j % 2 == 0 else bw[1]

        # the order of stream_strip_pair: the pair (y0 - 1, y0), then one
        # pair fetched ahead of each pair formed, and the step's outputs
        form(fetch(y0 - 1), y0 - 1)
        nxt = fetch(y0 + 1)
        for j in range(y0, y1, 2):
            cur = nxt
            if j + 2 < y1:
                nxt = fetch(j + 3)
            form(cur, j + 1)
            out(j)
            if j + 1 < y1:
                out(j + 1)
    return formed


@pytest.mark.parametrize("n", [2, 4, 8, 32, 64, 128])
def test_streamed_prolongation_is_the_textbook_form_bitwise(n):
    rng = np.random.default_rng(n)
    nc = n // 2
    ec = np.zeros((nc + 1, nc + 1), f32)
    ec[1:nc, 1:nc] = rng.standard_normal((nc - 1, nc - 1)).astype(f32)
    e = np.zeros((n + 1, n + 1), f32)
    e[1:n, 1:n] = rng.standard_normal((n - 1, n - 1)).astype(f32)
    seen = set()
    for y0 in range(0, n + 1, SROWS):
        y1 = min(y0 + SROWS, n + 1)
        for (i, j), x in strip_fields(n, e, ec, y0).items():
            # every row of the window: y0 - 1 .. y1 (the stencil's rows)
            if y0 - 1 <= j <= y1 and -1 <= i <= n + 1:
                want = textbook(e, ec, i, j) if interior(n, i, j) else f32(0.0)
                assert x.view(np.uint32) == want.view(np.uint32), (n, y0, i, j, x, want)
                seen.add((i, j))
        # each output row reads b and W of its own row
        for (i, j), row in strip_fields.outputs.items():
            assert row == j and y0 <= j < y1, (n, y0, i, j, row)
        assert {j for (_, j) in strip_fields.outputs} == set(range(y0, y1))
    # every node of the grid was formed by some strip
    assert all((i, j) in seen for i in range(n + 1) for j in range(n + 1))


@pytest.mark.parametrize("n", [4, 16])
def test_textbook_form_is_bilinear_interpolation(n):
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(100 + n)
    nc = n // 2
    ec = np.zeros((nc + 1, nc + 1))
    ec[1:nc, 1:nc] = rng.standard_normal((nc - 1, nc - 1))
    e = np.zeros((n + 1, n + 1))
    xs = np.linspace(0.0, 1.0, nc + 1)
    f = interp.RegularGridInterpolator((xs, xs), ec, method="linear")
    for j in range(n + 1):
        for i in range(n + 1):
            want = f([[j / n, i / n]])[0]
            got = textbook(e.astype(np.float64), ec, i, j)
            assert abs(got - want) <= 1e-15 * (1 + abs(want)), (i, j, got, want)
