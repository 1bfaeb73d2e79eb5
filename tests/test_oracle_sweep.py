"""Pins for the oracle sweep (Sec. 3: Eqs. upwind and dgsn_transport, lumped
with the 2-point Gauss-Lobatto rule of Sec. 6).

* 1D pure absorber: the exact discrete attenuation (2/((1+tau)^2+1))^N and
  second-order convergence to exp(-sigma x / mu);
* constants are reproduced exactly;
* per-cell particle balance (test function u = 1) to round-off;
* tiny 2D meshes: the global system assembled independently from the
  symmetric average/jump form of Eq. dgsn_transport and solved densely;
* group splitting, x<->y mirror symmetry, boundary-side bookkeeping.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W


def _one_group_sweep(dim, nx, ny, ext, omx, omy, sig, inv_cdt, q, Iprev, infl):
    return O.sweep(dim, nx, ny, ext, omx, omy, sig, inv_cdt, q, Iprev, infl)


@pytest.mark.parametrize("mu,sigma,nx", [(0.3, 2.0, 20), (0.9, 0.1, 7), (0.05, 40.0, 13)])
def test_1d_pure_absorber_exact_discrete(mu, sigma, nx):
    h = 1.0 / nx
    omx = np.array([mu])
    sig = np.full((1, nx), sigma)
    q = np.zeros((1, nx, 2))
    infl = np.zeros((4, 1))
    infl[0, 0] = 1.0
    I = _one_group_sweep(1, nx, 1, (0, 1, 0, 1), omx, np.zeros(1), sig, 0.0, q, None, infl)[0, 0]
    tau = sigma * h / mu
    r = 2.0 / ((1 + tau) ** 2 + 1)
    k = np.arange(nx)
    assert np.allclose(I[:, 1], r ** (k + 1), rtol=1e-13, atol=0)
    assert np.allclose(I[:, 0], r ** (k + 1) * (1 + tau), rtol=1e-13, atol=0)


def test_1d_pure_absorber_negative_mu_enters_right():
    nx, mu, sigma = 10, -0.4, 3.0
    sig = np.full((1, nx), sigma)
    infl = np.zeros((4, 1))
    infl[1, 0] = 2.0
    I = _one_group_sweep(1, nx, 1, (0, 1, 0, 1), np.array([mu]), np.zeros(1), sig, 0.0,
                         np.zeros((1, nx, 2)), None, infl)[0, 0]
    tau = sigma / nx / abs(mu)
    r = 2.0 / ((1 + tau) ** 2 + 1)
    # cell nx-1 is first downwind of the right boundary; its node 0 is downwind
    k = np.arange(nx)[::-1]
    assert np.allclose(I[:, 0], 2.0 * r ** (k + 1), rtol=1e-13)


def test_1d_pure_absorber_second_order_to_exponential():
    mu, sigma = 0.5, 1.5
    errs = []
    for nx in (40, 80, 160):
        sig = np.full((1, nx), sigma)
        infl = np.zeros((4, 1))
        infl[0, 0] = 1.0
        I = _one_group_sweep(1, nx, 1, (0, 1, 0, 1), np.array([mu]), np.zeros(1), sig, 0.0,
                             np.zeros((1, nx, 2)), None, infl)[0, 0]
        errs.append(abs(I[-1, 1] - math.exp(-sigma / mu)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4


@pytest.mark.parametrize("dim", [1, 2])
def test_constants_reproduced(dim):
    nx, ny = 5, (4 if dim == 2 else 1)
    ncell = nx * ny
    nn = 2 if dim == 1 else 4
    omx, omy, w = O.quadrature(dim, 4, 2) if dim == 2 else O.quadrature(1, 4)
    nd = len(w)
    rng = np.random.default_rng(5)
    G = 2
    sig = rng.uniform(0.1, 50.0, size=(G, ncell))
    C = np.array([0.7, 3.1])
    inv_cdt = 5.0
    q = sig[:, :, None] * C[:, None, None] * np.ones((G, ncell, nn))
    Iprev = np.broadcast_to(C[None, :, None, None], (nd, G, ncell, nn)).copy()
    infl = np.tile(C[None, :], (4, 1))
    I = O.sweep(dim, nx, ny, (0, 1, 0, 2), omx, omy, sig, inv_cdt, q, Iprev, infl)
    assert np.allclose(I, Iprev, rtol=1e-14, atol=0)


def _cell_balance_residual(nx, ny, ext, Ox, Oy, sig_t, S, infl, I):
    """sum_faces (len/2) sum_pts (Omega.n) I_hat + sigma~ sum m I - sum m S, per cell."""
    x0, x1, y0, y1 = ext
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    Ic = I.reshape(ny, nx, 2, 2)  # [iy][ix][b][a]
    Sc = S.reshape(ny, nx, 2, 2)
    res = np.zeros((ny, nx))
    for iy in range(ny):
        for ix in range(nx):
            tot = 0.0
            # x faces: left (a=0, n=-x), right (a=1, n=+x)
            for a, nrm, nb in ((0, -1.0, ix - 1), (1, 1.0, ix + 1)):
                On = Ox * nrm
                for b in range(2):
                    if On > 0:
                        Ih = Ic[iy, ix, b, a]
                    elif 0 <= nb < nx:
                        Ih = Ic[iy, nb, b, 1 - a]
                    else:
                        Ih = infl[0 if a == 0 else 1]
                    tot += 0.5 * hy * On * Ih
            for b, nrm, nb in ((0, -1.0, iy - 1), (1, 1.0, iy + 1)):
                On = Oy * nrm
                for a in range(2):
                    if On > 0:
                        Ih = Ic[iy, ix, b, a]
                    elif 0 <= nb < ny:
                        Ih = Ic[nb, ix, 1 - b, a]
                    else:
                        Ih = infl[2 if b == 0 else 3]
                    tot += 0.5 * hx * On * Ih
            m = 0.25 * hx * hy
            tot += sig_t[iy * nx + ix] * m * Ic[iy, ix].sum() - m * Sc[iy, ix].sum()
            res[iy, ix] = tot
    return res


def test_2d_particle_balance_per_cell():
    nx, ny, ext = 6, 5, (0.0, 1.2, -0.5, 0.5)
    ox, oy, w = O.quadrature(2, 2, 2)
    rng = np.random.default_rng(11)
    G, ncell = 1, nx * ny
    sig = np.exp(rng.uniform(-3, 6, size=(G, ncell)))
    inv_cdt = 3.0
    q = rng.uniform(0, 2, size=(G, ncell, 4))
    Ip = rng.uniform(0, 1, size=(len(w), G, ncell, 4))
    infl = rng.uniform(0, 1, size=(4, G))
    I = O.sweep(2, nx, ny, ext, ox, oy, sig, inv_cdt, q, Ip, infl)
    for d in range(len(w)):
        S = q[0] + inv_cdt * Ip[d, 0]
        res = _cell_balance_residual(nx, ny, ext, ox[d], oy[d], sig[0] + inv_cdt, S, infl[:, 0],
                                     I[d, 0])
        scale = (sig[0] + inv_cdt).max() * np.abs(I[d, 0]).max() * 0.25 * (1.2 / nx) * (1.0 / ny)
        assert np.max(np.abs(res)) < 1e-13 * scale


def _dense_global_2d(nx, ny, ext, Ox, Oy, sig_t, S, infl):
    """Global lumped system from the symmetric average/jump form of
    Eq. dgsn_transport over unique interior faces, solved densely."""
    x0, x1, y0, y1 = ext
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    N = nx * ny * 4

    def gid(ix, iy, a, b):
        return (iy * nx + ix) * 4 + a + 2 * b

    A = np.zeros((N, N))
    rhs = np.zeros(N)
    m = 0.25 * hx * hy
    for iy in range(ny):
        for ix in range(nx):
            k = iy * nx + ix
            for b in range(2):
                for a in range(2):
                    i = gid(ix, iy, a, b)
                    rhs[i] += m * S[k, a + 2 * b]
                    A[i, i] += m * sig_t[k]
                    # -int Omega.grad(u_i) I at the four corners
                    for bb in range(2):
                        for aa in range(2):
                            j = gid(ix, iy, aa, bb)
                            g = 0.0
                            if bb == b:
                                g += Ox * (2 * a - 1) / hx
                            if aa == a:
                                g += Oy * (2 * b - 1) / hy
                            A[i, j] -= m * g
    # interior faces: Omega.n [u]{I} + 1/2 |Omega.n| [u][I], n from K1 to K2
    def face(K1nodes, K2nodes, On, wgt):
        for p in range(2):
            i1, i2 = K1nodes[p], K2nodes[p]
            for (iu, su) in ((i1, 1.0), (i2, -1.0)):
                A[iu, i1] += wgt * su * (On * 0.5 + 0.5 * abs(On))
                A[iu, i2] += wgt * su * (On * 0.5 - 0.5 * abs(On))

    for iy in range(ny):
        for ix in range(nx - 1):
            face([gid(ix, iy, 1, b) for b in range(2)], [gid(ix + 1, iy, 0, b) for b in range(2)],
                 Ox, 0.5 * hy)
    for iy in range(ny - 1):
        for ix in range(nx):
            face([gid(ix, iy, a, 1) for a in range(2)], [gid(ix, iy + 1, a, 0) for a in range(2)],
                 Oy, 0.5 * hx)
    # boundary faces: outflow on the left side of the equation, inflow on the right
    def bface(nodes, On, wgt, val):
        for i in nodes:
            if On > 0:
                A[i, i] += wgt * On
            else:
                rhs[i] -= wgt * On * val

    for iy in range(ny):
        bface([gid(0, iy, 0, b) for b in range(2)], -Ox, 0.5 * hy, infl[0])
        bface([gid(nx - 1, iy, 1, b) for b in range(2)], Ox, 0.5 * hy, infl[1])
    for ix in range(nx):
        bface([gid(ix, 0, a, 0) for a in range(2)], -Oy, 0.5 * hx, infl[2])
        bface([gid(ix, ny - 1, a, 1) for a in range(2)], Oy, 0.5 * hx, infl[3])
    return np.linalg.solve(A, rhs).reshape(nx * ny, 4)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (4, 4)])
def test_2d_matches_dense_global_system(nx, ny):
    ext = (0.0, 2.0, 0.0, 1.0)
    ox, oy, w = O.quadrature(2, 2, 2)
    rng = np.random.default_rng(nx * 10 + ny)
    ncell = nx * ny
    sig = np.exp(rng.uniform(-2, 5, size=(1, ncell)))
    inv_cdt = 0.7
    q = rng.uniform(0, 1, size=(1, ncell, 4))
    Ip = rng.uniform(0, 1, size=(len(w), 1, ncell, 4))
    infl = rng.uniform(0, 1, size=(4, 1))
    I = O.sweep(2, nx, ny, ext, ox, oy, sig, inv_cdt, q, Ip, infl)
    for d in range(len(w)):
        S = q[0] + inv_cdt * Ip[d, 0]
        ref = _dense_global_2d(nx, ny, ext, ox[d], oy[d], sig[0] + inv_cdt, S, infl[:, 0])
        assert np.allclose(I[d, 0], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_group_splitting_equals_gray():
    nx, ny = 5, 4
    ox, oy, w = O.quadrature(2, 2, 2)
    rng = np.random.default_rng(2)
    ncell = nx * ny
    sig1 = rng.uniform(0.5, 20, size=(1, ncell))
    q1 = rng.uniform(0, 1, size=(1, ncell, 4))
    Ip1 = rng.uniform(0, 1, size=(len(w), 1, ncell, 4))
    inf1 = rng.uniform(0, 1, size=(4, 1))
    f = np.array([0.2, 0.5, 0.3])
    G = 3
    sigG = np.repeat(sig1, G, axis=0)
    qG = f[:, None, None] * q1
    IpG = f[None, :, None, None] * Ip1
    infG = inf1 * f[None, :]
    Ig = O.sweep(2, nx, ny, (0, 1, 0, 1), ox, oy, sig1, 2.0, q1, Ip1, inf1)
    IG = O.sweep(2, nx, ny, (0, 1, 0, 1), ox, oy, sigG, 2.0, qG, IpG, infG)
    assert np.allclose(IG.sum(axis=1), Ig[:, 0], rtol=1e-13)
    assert np.allclose(IG[:, 1], 0.5 * Ig[:, 0], rtol=1e-13)


def test_xy_mirror_symmetry():
    n = 5
    ox, oy, w = O.quadrature(2, 2, 3)
    rng = np.random.default_rng(9)
    s = rng.uniform(0.5, 30, size=(n, n))
    s = s + s.T
    q = rng.uniform(0, 1, size=(n, n, 2, 2))  # [iy][ix][b][a]
    q = q + q.transpose(1, 0, 3, 2)
    sig = s.reshape(1, n * n)
    qq = q.reshape(1, n * n, 4)
    infl = np.array([[0.8], [0.1], [0.8], [0.1]])  # left == bottom, right == top
    I = O.sweep(2, n, n, (0, 1, 0, 1), ox, oy, sig, 0.0, qq, None, infl)
    for d in range(len(w)):
        dp = int(np.argmin((ox - oy[d]) ** 2 + (oy - ox[d]) ** 2))
        assert abs(ox[dp] - oy[d]) < 1e-14 and abs(oy[dp] - ox[d]) < 1e-14
        A = I[d, 0].reshape(n, n, 2, 2)
        B = I[dp, 0].reshape(n, n, 2, 2).transpose(1, 0, 3, 2)
        assert np.allclose(A, B, rtol=1e-13)


def test_boundary_sides_select_directions():
    nx = ny = 3
    ox, oy, w = O.quadrature(2, 2, 2)
    sig = np.full((1, 9), 1.0)
    for side, pred in ((0, ox > 0), (1, ox < 0), (2, oy > 0), (3, oy < 0)):
        infl = np.zeros((4, 1))
        infl[side] = 1.0
        I = O.sweep(2, nx, ny, (0, 1, 0, 1), ox, oy, sig, 0.0, np.zeros((1, 9, 4)), None, infl)
        # lumped DG carries no positivity fix-up, so only the support is pinned
        assert np.all(np.abs(I[pred]).reshape(pred.sum(), -1).max(axis=1) > 0)
        assert np.all(I[~pred] == 0)


def test_sweep_pairs_subset_matches_full():
    nx, ny = 4, 3
    ox, oy, w = O.quadrature(2, 2, 2)
    rng = np.random.default_rng(4)
    G = 3
    sig = rng.uniform(0.5, 5, size=(G, 12))
    q = rng.uniform(0, 1, size=(G, 12, 4))
    Ip = rng.uniform(0, 1, size=(len(w), G, 12, 4))
    infl = rng.uniform(0, 1, size=(4, G))
    full = O.sweep(2, nx, ny, (0, 1, 0, 1), ox, oy, sig, 1.0, q, Ip, infl)
    pairs = [(5, 2), (0, 0), (15, 1)]
    sub = O.sweep_pairs(2, nx, ny, (0, 1, 0, 1), ox, oy, sig, 1.0, q, Ip, infl, pairs)
    for i, (d, g) in enumerate(pairs):
        assert np.array_equal(sub[i], full[d, g])
