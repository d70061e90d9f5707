"""The warp-strip full weighting of the 2D multigrid (k_restrict2s), replayed
on the CPU: its grid, lanes, paired loads, shuffles and carried row sums.

bc = P^T r1 on the interior coarse nodes, with P the bilinear prolongation
(the Kronecker product of the 1D interpolation matrices, fine node 2I <-
coarse I with weight 1, fine nodes 2I +- 1 with weight 1/2), and 0 on the
coarse boundary. The replay also checks what the kernel may touch: every
load stays inside its fine row (columns 0..2n_c, rows 0..2n_c), paired
loads start at even offsets (aligned vectors), and every coarse node is
written exactly once."""
import numpy as np
import pytest

SWARPS = 4          # warps per CTA (the stencil kernels' CTA)
RSTRIP_ROWS = 16    # coarse rows per CTA


def prolongation_1d(nc):
    P = np.zeros((2 * nc + 1, nc + 1))
    for I in range(nc + 1):
        P[2 * I, I] = 1.0
        if I > 0:
            P[2 * I - 1, I] = 0.5
        if I < nc:
            P[2 * I + 1, I] = 0.5
    return P


def replay(nc, r1):
    """The kernel's launch on one sample: {(I, J): value} and the set of
    fine (row, col) read."""
    N1c, N1 = nc + 1, 2 * nc + 1
    flat = r1.reshape(-1)
    out, reads = {}, []

    def load(off):
        fr, col = divmod(off, N1)
        assert 0 <= fr < N1 and 0 <= col < N1, (nc, off)
        reads.append((fr, col))
        return flat[off]

    gx = (N1c + 32 * SWARPS - 1) // (32 * SWARPS)
    gy = (N1c + RSTRIP_ROWS - 1) // RSTRIP_ROWS
    for bx in range(gx):
        for w in range(SWARPS):
            I0 = (bx * SWARPS + w) * 32
            if I0 > nc:
                continue
            lanes = range(32)
            for by in range(gy):
                J0, J1 = by * RSTRIP_ROWS, min(by * RSTRIP_ROWS + RSTRIP_ROWS, N1c)

                def even_sum(fr):
                    p = []
                    for l in lanes:
                        I = I0 + l
                        if I < nc:
                            off = fr * N1 + 2 * I
                            assert off % 2 == 0
                            p.append((load(off), load(off + 1)))
                        else:
                            p.append((0.0, 0.0))
                    s = []
                    for l in lanes:
                        I = I0 + l
                        left = p[l - 1][1] if l > 0 else (load(fr * N1 + 2 * I - 1) if I >= 1 else 0.0)
                        s.append(0.5 * left + p[l][0] + 0.5 * p[l][1])
                    return s

                def odd_sum(fr):
                    p = []
                    for l in lanes:
                        I = I0 + l
                        if 1 <= I <= nc:
                            off = fr * N1 + 2 * I - 1
                            assert off % 2 == 0
                            p.append((load(off), load(off + 1)))
                        else:
                            p.append((0.0, 0.0))
                    s = []
                    for l in lanes:
                        I = I0 + l
                        right = p[l + 1][0] if l < 31 else (load(fr * N1 + 2 * I + 1) if I < nc else 0.0)
                        s.append(0.5 * p[l][0] + p[l][1] + 0.5 * right)
                    return s

                oprev = odd_sum(2 * J0 - 1) if J0 >= 1 else [0.0] * 32
                for J in range(J0, J1):
                    jin = 1 <= J < nc
                    o = odd_sum(2 * J + 1) if J < nc else [0.0] * 32
                    ev = even_sum(2 * J) if jin else [0.0] * 32
                    for l in lanes:
                        I = I0 + l
                        v = 0.5 * (oprev[l] + o[l]) + ev[l] if (jin and 1 <= I < nc) else 0.0
                        if I <= nc:
                            assert (I, J) not in out, (nc, I, J)
                            out[(I, J)] = v
                    oprev = o
    return out, reads


@pytest.mark.parametrize("nc", [1, 2, 8, 31, 32, 33, 64, 128])
def test_strip_restriction_is_the_transpose_of_bilinear_prolongation(nc):
    rng = np.random.default_rng(7 + nc)
    n = 2 * nc
    r1 = np.zeros((n + 1, n + 1))
    r1[1:n, 1:n] = rng.standard_normal((n - 1, n - 1))
    P1 = prolongation_1d(nc)
    want = P1.T @ r1 @ P1          # [J, I]: rows are y, columns x
    out, reads = replay(nc, r1)
    assert len(out) == (nc + 1) ** 2
    for (I, J), v in out.items():
        if 1 <= I < nc and 1 <= J < nc:
            assert abs(v - want[J, I]) <= 1e-13 * (1 + abs(want[J, I])), (nc, I, J, v, want[J, I])
        else:
            assert v == 0.0
    # the interior fine nodes that feed interior coarse nodes are all read
    need = {(fr, fc) for fr in range(1, n) for fc in range(1, n)}
    if nc >= 2:
        assert need <= set(reads)
