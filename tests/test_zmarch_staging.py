"""The plane staging of the FP32 3D z-march on full-width tiles (k_zm3w),
replayed on the CPU for every mesh it serves (32^3..256^3), both row
counts per thread (2 and 4) and one or two staged arrays.

Each plane pp of a node array is one bulk copy of the tile's node rows
ylo..yhi (rows ty0 - 1 .. ty0 + R, clipped), widened to 16-byte
boundaries [Ga, Gb) and landed at a slot offset that keeps the destination
16-byte aligned; each kappa layer is one bulk copy of element rows
kylo..ty0 + R - 1. The replay checks what the copy engine and the threads
may touch:
  - sources lie inside the sample's node / element array, start 16-byte
    aligned and move a multiple of 16 bytes;
  - destinations start 16-byte aligned and stay inside their array's part of
    the slot; the ring and its barriers fit the CTA's shared memory;
  - every staged value a thread reads lies inside its slot, and every value
    that feeds an interior output (interior field node, element inside the
    mesh) was copied and is the right one: slot index -> global index equals
    the node (plane, row jr0 - 1 + r, column i - 1 + dx) or element the
    stencil wants;
  - the CTA grid covers every tile and z-chunk once and the per-CTA partials
    land inside the sample's partial block.
The formulas below restate the kernel's index arithmetic; they are the
subject of the check, the bounds and the wanted global indices its
yardstick."""
import numpy as np
import pytest

ZTHREADS = 256
ZW_S = 4


def rnd(x, m):
    return (x + m - 1) // m * m


def zw_rows(n, rt):
    return 256 * rt // n


def zw_vslot(n, rt):
    return (12 + (zw_rows(n, rt) + 2) * (n + 1) + 3) // 4 * 4


def zw_kslot(n, rt):
    return (8 + (zw_rows(n, rt) + 1) * n + 3) // 4 * 4


@pytest.mark.parametrize("rt", [2, 4])
@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_zmarch_staging_stays_in_bounds_and_reads_the_right_values(n, rt):
    N1, P, KPn = n + 1, (n + 1) ** 2, n * n
    ns, es = rnd(N1 ** 3, 32), rnd(n ** 3, 32)
    R, VS, KS = zw_rows(n, rt), zw_vslot(n, rt), zw_kslot(n, rt)
    tx, tyc = n, ZTHREADS // n            # block (n, 256 / n)
    assert tx * tyc == ZTHREADS and R == rt * tyc
    for NA in (1, 2):
        SS = NA * VS + KS
        assert VS % 4 == 0 and KS % 4 == 0 and SS % 4 == 0
        smem = 4 * ZW_S * SS + 8 * ZW_S
        assert smem <= (96 if rt == 4 else 48) * 1024, (n, rt, NA, smem)
    i = np.arange(tx)
    tyn = n // R
    for t in range(tyn):
        ty0 = t * R
        ylo, yhi = max(ty0 - 1, 0), min(ty0 + R, n)
        r0 = ylo - ty0 + 1
        kylo = max(ty0 - 1, 0)
        kr0 = kylo - ty0 + 1
        kcount = (ty0 + R - kylo) * n
        for pp in range(-1, n + 2):       # every plane a chunk may visit
            pv, pk = 1 <= pp < n, 0 <= pp < n
            sh = (pp * P + ylo * N1) & 3
            voff = (sh - r0 * N1) & 3
            G0, G1 = pp * P + ylo * N1, pp * P + (yhi + 1) * N1
            Ga, Gb = G0 & ~3, (G1 + 3) & ~3
            dst = 4 + voff + r0 * N1 - (G0 - Ga)
            if pv:
                assert 0 <= Ga and Gb <= ns and Ga % 4 == 0 and (Gb - Ga) % 4 == 0
                assert dst >= 0 and dst % 4 == 0 and dst + (Gb - Ga) <= VS, (n, rt, ty0, pp)
            ksrc, kdst = pp * KPn + kylo * n, 4 + kr0 * n
            if pk:
                assert 0 <= ksrc and ksrc + kcount <= es and ksrc % 4 == 0 and kcount % 4 == 0
                assert kdst % 4 == 0 and kdst + kcount <= KS
            for ty in range(tyc):
                jr0 = ty0 + rt * ty
                vrow = 4 + rt * ty * N1 + i - 1
                krow = 4 + rt * ty * n + i - 1
                for r in range(rt + 2):
                    for dx in range(3):
                        idx = voff + vrow + r * N1 + dx
                        assert idx.min() >= 0 and idx.max() < VS
                        row, col = jr0 - 1 + r, i - 1 + dx
                        need = pv & (row >= 1) & (row <= n - 1) & (col >= 1) & (col <= n - 1) & \
                            (i >= 1) & (i <= n - 1)
                        if need.any():
                            k = idx[need]
                            assert np.all((k >= dst) & (k < dst + (Gb - Ga))), (n, rt, ty0, pp, r, dx)
                            assert np.all(Ga + (k - dst) == pp * P + row * N1 + col[need])
                for r in range(rt + 1):
                    for a in range(2):
                        idx = krow + r * n + a
                        assert idx.min() >= 0 and idx.max() < KS
                        erow, ecol = jr0 - 1 + r, i - 1 + a
                        need = pk & (erow >= 0) & (erow <= n - 1) & (ecol >= 0) & (ecol <= n - 1) & \
                            (i >= 1) & (i <= n - 1)
                        if need.any():
                            k = idx[need]
                            assert np.all((k >= kdst) & (k < kdst + kcount)), (n, rt, ty0, pp, r, a)
                            assert np.all(ksrc + (k - kdst) == pp * KPn + erow * n + ecol[need])


@pytest.mark.parametrize("n", [32, 64, 128, 256])
@pytest.mark.parametrize("zc", [16, 24, 32, 64, 257])
def test_zmarch_grid_covers_tiles_and_chunks_once(n, zc):
    zc = min(zc, n + 1)
    nzq = (n + 1 + zc - 1) // zc
    zx = ((n + 31) // 32) * ((n + 15) // 16) * nzq   # CTAs of the 32 x 16 tiling (and partials)
    R2 = zw_rows(n, 2)
    assert zx == (n // R2) * nzq                       # the launch's precondition
    for rt in (2, 4):
        R, np_ = zw_rows(n, rt), rt // 2
        tyn = n // R
        grid = zx if rt == 2 else zx // 2
        seen, parts = set(), set()
        for t in range(grid):
            zq, ty0 = t // tyn, (t % tyn) * R
            z0, z1 = zq * zc, min(zq * zc + zc, n + 1)
            assert z0 < z1
            for z in range(z0, z1):
                for row in range(ty0, ty0 + R):
                    assert (z, row) not in seen
                    seen.add((z, row))
            base = zq * (n // R2) + ty0 // R2
            for k in range(np_):
                assert 0 <= base + k < zx and base + k not in parts
                parts.add(base + k)
        assert len(seen) == (n + 1) * n                # planes 0..n, rows 0..n-1 (row n: zeroed by row n-1)
        assert parts == set(range(zx))
