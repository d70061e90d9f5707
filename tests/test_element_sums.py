"""The element-sum form of the trilinear Q1 operator that the FP64 3D
z-march (k_zm3q) evaluates, checked on the CPU against the oracle's
assembled matrix:

  (A u)_n = h/12 [5 u_n K_n - sum_{e ni n} kappa_e S_e + sum_{6 d} u_{n+d} K_{n,n+d}],

K_n the sum of the 8 kappa around node n, K_{n,n+d} the sum of the 4
elements sharing the edge (n, n + d), S_e the sum of u over the 8 nodes of
element e (from the element stiffness h/12 (4, 0, -1, -1) by the number of
coordinates in which two vertices differ). The second test follows the
kernel's schedule step by step: 32 x 16 node tiles with a one-node halo,
z-chunks, per plane the element sums of the plane and Q = kappa S of the
layer below formed once per element position, and the carried values (the
sums of the layer below, the centre and K_z of the plane below)."""
import numpy as np
import pytest

from oracle import fem


def kappa_sums(kap):
    n = kap.shape[0]
    N1 = n + 1
    kp = np.zeros((n + 2, n + 2, n + 2))
    kp[1:-1, 1:-1, 1:-1] = kap
    Kn = sum(kp[dz:dz + N1, dy:dy + N1, dx:dx + N1] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1))
    Kx = sum(kp[dz:dz + N1, dy:dy + N1, 1:N1 + 1] for dz in (0, 1) for dy in (0, 1))
    Ky = sum(kp[dz:dz + N1, 1:N1 + 1, dx:dx + N1] for dz in (0, 1) for dx in (0, 1))
    Kz = sum(kp[1:N1 + 1, dy:dy + N1, dx:dx + N1] for dy in (0, 1) for dx in (0, 1))
    return Kn, Kx, Ky, Kz


def random_problem(n, seed):
    rng = np.random.default_rng(seed)
    N1 = n + 1
    kap = np.exp(rng.standard_normal((n, n, n)))   # [z, y, x]
    u = rng.standard_normal((N1, N1, N1))
    u[0] = u[-1] = 0
    u[:, 0] = u[:, -1] = 0
    u[:, :, 0] = u[:, :, -1] = 0
    return kap, u


def oracle_apply(n, kap, u):
    A = fem.assemble(3, n, kap.reshape(-1)) if n <= 5 else fem.assemble_fast(3, n, kap.reshape(-1))
    return A @ fem.from_node_grid(3, n, u.reshape(-1))


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8])
def test_element_sum_identity(n):
    kap, u = random_problem(n, n)
    N1, h = n + 1, 1.0 / n
    Kn, Kx, Ky, Kz = kappa_sums(kap)
    S = sum(u[dz:dz + n, dy:dy + n, dx:dx + n] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1))
    Q = np.zeros((n + 2, n + 2, n + 2))
    Q[1:-1, 1:-1, 1:-1] = kap * S
    A_el = sum(Q[dz:dz + N1, dy:dy + N1, dx:dx + N1] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1))
    up = np.zeros((N1 + 2,) * 3)
    up[1:-1, 1:-1, 1:-1] = u

    def U(dz, dy, dx):
        return up[1 + dz:1 + dz + N1, 1 + dy:1 + dy + N1, 1 + dx:1 + dx + N1]

    Kxm = np.zeros((N1, N1, N1 + 1))
    Kxm[:, :, 1:] = Kx
    Kym = np.zeros((N1, N1 + 1, N1))
    Kym[:, 1:, :] = Ky
    Kzm = np.zeros((N1 + 1, N1, N1))
    Kzm[1:] = Kz
    six = (U(0, 0, 1) * Kx + U(0, 0, -1) * Kxm[:, :, :N1] + U(0, 1, 0) * Ky + U(0, -1, 0) * Kym[:, :N1, :]
           + U(1, 0, 0) * Kz + U(-1, 0, 0) * Kzm[:N1])
    y = (h / 12.0) * (5 * u * Kn - A_el + six)
    ref = oracle_apply(n, kap, u)
    got = fem.from_node_grid(3, n, y.reshape(-1))
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


ZTX, ZTY = 32, 16


def zm3q_schedule(n, zc, kap, u):
    """k_zm3q's per-tile, per-plane schedule (all output nodes of the mesh)."""
    N1, h = n + 1, 1.0 / n
    Kn, Kx, Ky, Kz = kappa_sums(kap)
    ZSX, ZSY, ZKX, ZKY = ZTX + 2, ZTY + 2, ZTX + 1, ZTY + 1

    def node(z, y, x):
        inside = 1 <= z <= n - 1 and 1 <= y <= n - 1 and 1 <= x <= n - 1
        return u[z, y, x] if inside else 0.0

    def element(z, y, x):
        return kap[z, y, x] if (0 <= z < n and 0 <= y < n and 0 <= x < n) else 0.0

    Y = np.zeros((N1, N1, N1))
    for zq in range((n + zc) // zc):
        z0, z1 = zq * zc, min(zq * zc + zc, n + 1)
        if z0 > n:
            continue
        for ty0 in range(0, n, ZTY):
            for tx0 in range(0, n, ZTX):
                sv = [np.zeros((ZSY, ZSX)) for _ in range(3)]
                sk = [np.zeros((ZKY, ZKX)) for _ in range(2)]
                sp = [np.zeros((ZKY, ZKX)) for _ in range(2)]
                Bprev, ucar = {}, {}
                buf, cur, prv = 0, 0, 2
                for p in range(z0 - 1, z1 + 1):
                    for ey in range(ZSY):
                        for ex in range(ZSX):
                            sv[cur][ey, ex] = node(p, ty0 - 1 + ey, tx0 - 1 + ex)
                    for ey in range(ZKY):
                        for ex in range(ZKX):
                            sk[buf][ey, ex] = element(p, ty0 - 1 + ey, tx0 - 1 + ex)
                    sq = np.zeros((ZKY, ZKX))
                    for ey in range(ZKY):
                        for ex in range(ZKX):
                            v = sv[cur]
                            pxy = (v[ey, ex] + v[ey, ex + 1]) + (v[ey + 1, ex] + v[ey + 1, ex + 1])
                            sq[ey, ex] = sk[buf ^ 1][ey, ex] * (pxy + sp[buf ^ 1][ey, ex])
                            sp[buf][ey, ex] = pxy
                    m = p - 1
                    for j in range(ty0, ty0 + ZTY):
                        for i in range(tx0, tx0 + ZTX):
                            key = (i, j)
                            ey, ex = j - ty0, i - tx0   # element (i - 1, j - 1)
                            qx0 = sq[ey, ex] + sq[ey, ex + 1]
                            qx1 = sq[ey + 1, ex] + sq[ey + 1, ex + 1]
                            bcur = qx0 + qx1
                            vo = sv[prv]
                            cy, cx = j - ty0 + 1, i - tx0 + 1
                            uc = vo[cy, cx]
                            inside = 1 <= i <= n - 1 and 1 <= j <= n - 1 and 1 <= m <= n - 1
                            if z0 <= m < z1 and inside:
                                sx = (Kx[m, j, i] * vo[cy, cx + 1] + Kx[m, j, i - 1] * vo[cy, cx - 1]
                                      + Ky[m, j, i] * vo[cy + 1, cx] + Ky[m, j - 1, i] * vo[cy - 1, cx]
                                      + Kz[m, j, i] * sv[cur][cy, cx] + Kz[m - 1, j, i] * ucar[key])
                                Y[m, j, i] = (h / 12.0) * (5 * uc * Kn[m, j, i] + sx - (Bprev[key] + bcur))
                            Bprev[key] = bcur
                            ucar[key] = uc
                    buf ^= 1
                    prv, cur = cur, (cur + 1) % 3
    return Y


@pytest.mark.parametrize("n,zc", [(4, 5), (8, 3), (33, 8)])
def test_zm3q_schedule_matches_the_oracle(n, zc):
    kap, u = random_problem(n, 100 + n)
    Y = zm3q_schedule(n, zc, kap, u)
    ref = oracle_apply(n, kap, u)
    got = fem.from_node_grid(3, n, Y.reshape(-1))
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
