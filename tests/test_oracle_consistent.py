"""Pins for the oracle's consistent SM low-order sources (Sec. 4, consistent
method; derived in oracle/consistent.py by the discrete residual approach):

* consistency identity: for ANY high-order intensity that solves the lumped
  upwind DG transport equations, the low-order linear system (emission frozen
  as the same source) with the consistent sources reproduces that intensity's
  energy density and flux to round-off;
* at convergence the consistent SM step equals the converged high-order step
  (the unaccelerated iteration of oracle/adjoint.py), while the independent
  step differs by its discretization inconsistency (Sec. 6 observations);
* half-range sums reproduce the full-range moments.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from oracle import adjoint as OA
from oracle import consistent as C
from oracle import lo as L
from paper_2504_21784_gb300 import workloads as W


def _cfg(nx, ny, G, npol=2, naz=2, T_bdr=(1.0, 0.3, 0.5, 0.0)):
    return W.Config("c", 2, nx, ny, (0.0, 1.0, 0.0, 0.7), W.log_edges(G), npol, naz, 1, 10.0,
                    T_bdr, dt=0.01)


@pytest.mark.parametrize("nx,ny,G,seed", [(4, 3, 3, 4), (1, 1, 2, 1), (5, 2, 4, 9)])
def test_consistency_identity(nx, ny, G, seed):
    cfg = _cfg(nx, ny, G)
    m = L.make_mesh(2, nx, ny, cfg.extent)
    rng = np.random.default_rng(seed)
    T = 0.1 + 0.8 * rng.random((m.ncell, 4))
    sigma = O.opacity(1, 10.0, cfg.edges, T, np.exp(0.5 * rng.standard_normal(m.ncell)))
    omx, omy, w = O.quadrature(2, cfg.n_polar, cfg.n_azim)
    alpha = O.alpha(omx, w)
    Ik = W.intensity_random(len(w), G, m.ncell, 4, seed=seed + 1, scale=0.05)
    q = O.emission(cfg.edges, 1.0, 1.0, T, sigma)
    infl = O.inflow(cfg.edges, 1.0, 1.0, cfg.T_bdr)
    inv_cdt = 1.0 / (cfg.c * cfg.dt)
    I = O.sweep(2, nx, ny, cfg.extent, omx, omy, sigma, inv_cdt, q, Ik, infl)
    mom = O.moments(2, omx, omy, w, sigma, I)
    clo = O.closures(2, cfg.edges, 1.0, sigma, T, mom)
    R1, R0 = C.consistent_sources(m, 1.0, alpha, clo, omx, omy, w, I, infl.sum(axis=1))
    AEF, AFE, P = L.lo_operators(m, 1.0, alpha)
    N, mass = m.nnode, m.mass()
    flat = clo.reshape(N, -1)
    momk = O.moments(2, omx, omy, w, sigma, Ik)
    emis = 4.0 * np.pi * q.sum(axis=0).reshape(-1)   # sum_g sigma_g B_g(T)
    K = sp.bmat([[sp.diags(np.repeat(mass * (flat[:, 7] + inv_cdt), 2)), AFE],
                 [AEF, P + sp.diags(mass * (flat[:, 6] + inv_cdt))]], format="csc")
    b = np.concatenate([mass * inv_cdt * momk[..., 1:3].reshape(-1) + R1,
                        mass * (emis + momk[..., 0].reshape(-1) / cfg.dt) + R0])
    sol = spla.spsolve(K, b)
    El, Fl = sol[2 * N:], sol[:2 * N]
    Eh, Fh = mom[..., 0].reshape(-1), mom[..., 1:3].reshape(-1)
    assert np.abs(El - Eh).max() < 1e-13 * np.abs(Eh).max()
    assert np.abs(Fl - Fh).max() < 1e-13 * np.abs(Eh).max()


@pytest.mark.parametrize("nx,G,npol,seed", [(7, 3, 4, 2), (1, 2, 2, 5), (12, 1, 8, 7)])
def test_consistency_identity_1d(nx, G, npol, seed):
    """The same identity on the 1D slab (point faces, half ranges by the sign
    of mu), including one cell and the gray case."""
    edges = W.log_edges(G) if G > 1 else W.GRAY_EDGES.copy()
    cfg = W.Config("c1", 1, nx, 1, (0.0, 1.0, 0.0, 1.0), edges, npol, 0, 1, 10.0,
                   (1.0, 0.4, 0.0, 0.0), dt=0.01)
    m = L.make_mesh(1, nx, 1, cfg.extent)
    rng = np.random.default_rng(seed)
    T = 0.1 + 0.8 * rng.random((m.ncell, 2))
    sigma = O.opacity(1, 10.0, cfg.edges, T, np.exp(0.5 * rng.standard_normal(m.ncell)))
    mu, omy, w = O.quadrature(1, npol)
    alpha = O.alpha(mu, w)
    Ik = W.intensity_random(len(w), G, m.ncell, 2, seed=seed + 1, scale=0.05)
    q = O.emission(cfg.edges, 1.0, 1.0, T, sigma)
    infl = O.inflow(cfg.edges, 1.0, 1.0, cfg.T_bdr)
    inv_cdt = 1.0 / (cfg.c * cfg.dt)
    I = O.sweep(1, nx, 1, cfg.extent, mu, omy, sigma, inv_cdt, q, Ik, infl)
    mom = O.moments(1, mu, omy, w, sigma, I)
    clo = O.closures(1, cfg.edges, 1.0, sigma, T, mom)
    R1, R0 = C.consistent_sources(m, 1.0, alpha, clo, mu, omy, w, I, infl.sum(axis=1))
    AEF, AFE, P = L.lo_operators(m, 1.0, alpha)
    N, mass = m.nnode, m.mass()
    flat = clo.reshape(N, -1)
    momk = O.moments(1, mu, omy, w, sigma, Ik)
    emis = 4.0 * np.pi * q.sum(axis=0).reshape(-1)
    K = sp.bmat([[sp.diags(mass * (flat[:, 4] + inv_cdt)), AFE],
                 [AEF, P + sp.diags(mass * (flat[:, 3] + inv_cdt))]], format="csc")
    b = np.concatenate([mass * inv_cdt * momk[..., 1].reshape(-1) + R1,
                        mass * (emis + momk[..., 0].reshape(-1) / cfg.dt) + R0])
    sol = spla.spsolve(K, b)
    El, Fl = sol[N:], sol[:N]
    Eh, Fh = mom[..., 0].reshape(-1), mom[..., 1].reshape(-1)
    assert np.abs(El - Eh).max() < 1e-13 * np.abs(Eh).max()
    assert np.abs(Fl - Fh).max() < 1e-13 * np.abs(Eh).max()


def test_half_moments_1d_sum_to_full_range():
    mu, omy, w = O.quadrature(1, 6)
    I = W.intensity_random(len(w), 3, 5, 2, seed=4, scale=1.0)
    qm = C.half_moments_1d(mu, w, I).reshape(10, 4, 6)
    sig = np.ones((3, 5))
    mom = O.moments(1, mu, omy, w, sig, I).reshape(10, 5)
    tot = qm.sum(axis=1)
    assert np.allclose(tot[:, 0], mom[:, 0], rtol=1e-14, atol=0)
    assert np.allclose(tot[:, 1], mom[:, 1], rtol=1e-13, atol=1e-15)
    assert np.allclose(tot[:, 3] - tot[:, 0] / 3.0, mom[:, 2], rtol=1e-12, atol=1e-14)
    assert np.all(qm[:, 0, 1] >= 0) and np.all(qm[:, 1, 1] <= 0)
    assert np.all(qm[:, 2:] == 0) and np.all(qm[:, :, [2, 4, 5]] == 0)


def test_half_ranges_sum_to_full_range():
    cfg = _cfg(3, 2, 2)
    omx, omy, w = O.quadrature(2, 2, 4)
    I = W.intensity_random(len(w), 2, 6, 4, seed=3, scale=1.0)
    qm = C.quadrant_moments(omx, omy, w, I).reshape(24, 4, 6)
    full = qm.sum(axis=1)
    for n in ((1.0, 0.0), (0.0, -1.0)):
        Fp, Fm, Pp, Pm = C.half_range(qm, n)
        assert np.allclose(Fp + Fm, full[:, 1] * n[0] + full[:, 2] * n[1], rtol=1e-14, atol=0)
        assert np.all(Fp >= 0) and np.all(Fm <= 0)
        Pn = np.stack([full[:, 3] * n[0] + full[:, 4] * n[1], full[:, 4] * n[0] + full[:, 5] * n[1]], 1)
        assert np.allclose(Pp + Pm, Pn, rtol=1e-13, atol=1e-15)
    del cfg


def test_consistent_step_equals_converged_high_order_step():
    nx, ny, G = 4, 3, 3
    cfg = _cfg(nx, ny, G)
    ncell = nx * ny
    rng = np.random.default_rng(4)
    T0 = 0.1 + 0.8 * rng.random((ncell, 4))
    scale = np.exp(0.5 * rng.standard_normal(ncell))
    cv = np.full((ncell, 4), 0.3)
    omx, omy, w = O.quadrature(2, 2, 2)
    pb = OA.Problem(nx, ny, cfg.extent, cfg.edges, 2, 2, 1, 10.0, cfg.T_bdr, dt=cfg.dt)
    B4, _ = OA.planck_parts(pb, T0)
    I0 = np.broadcast_to(B4[None], (len(w),) + B4.shape).copy()
    _, Ts, Is, _ = OA.forward(pb, scale, cv, T0, I0, 1, tol=1e-14)
    mom0 = O.moments(2, omx, omy, w, O.opacity(1, 10.0, cfg.edges, T0, scale), I0)
    res = {}
    for method in ("consistent", "independent"):
        prm = L.StepParams(eps_outer=1e-14, max_outer=300, method=method,
                           lo=L.LOParams(eps_inner=1e-14, max_inner=40, elim_rtol=1e-15,
                                         max_elim=80))
        T, E, F, I, mom, st = L.sm_step(cfg, scale, cv, T0, I0, mom0, prm)
        res[method] = (np.abs(T - Ts[1]).max() / Ts[1].max(),
                       np.abs(E - mom[..., 0]).max() / np.abs(mom[..., 0]).max())
    assert res["consistent"][0] < 1e-11 and res["consistent"][1] < 1e-11
    assert res["independent"][0] > 1e-4   # the independent method is not consistent


def test_consistent_step_equals_converged_high_order_step_1d():
    """1D slab: the converged consistent SM step equals the converged
    high-order step (source iteration on the sweep with the nodal energy
    balance), the independent step does not."""
    import types
    nx, G = 6, 3
    cfg = W.Config("c1s", 1, nx, 1, (0.0, 1.0, 0.0, 1.0), W.log_edges(G), 4, 0, 1, 10.0,
                   (1.0, 0.2, 0.0, 0.0), dt=0.01)
    rng = np.random.default_rng(11)
    T0 = 0.1 + 0.6 * rng.random((nx, 2))
    scale = np.exp(0.5 * rng.standard_normal(nx))
    cv = np.full((nx, 2), 0.3)
    mu, omy, w = O.quadrature(1, 4)
    I0 = L.equilibrium_intensity(cfg, T0, mu)
    sigma = O.opacity(1, 10.0, cfg.edges, T0, scale)
    mom0 = O.moments(1, mu, omy, w, sigma, I0)
    # high-order step: sweep <-> nodal energy balance until T stops changing
    pb = types.SimpleNamespace(edges=cfg.edges, a=cfg.a, c=cfg.c, dt=cfg.dt)
    infl = O.inflow(cfg.edges, cfg.a, cfg.c, cfg.T_bdr)
    T = T0.copy()
    for _ in range(2000):
        q = O.emission(cfg.edges, cfg.a, cfg.c, T, sigma)
        I = O.sweep(1, nx, 1, cfg.extent, mu, omy, sigma, 1.0 / (cfg.c * cfg.dt), q, I0, infl)
        SE = O.moments(1, mu, omy, w, sigma, I)[..., 3]
        Tn = OA._solve_energy(pb, cv, T0, T, sigma, SE)
        done = np.abs(Tn - T).max() <= 1e-15 * np.abs(Tn).max()
        T = Tn
        if done:
            break
    res = {}
    for method in ("consistent", "independent"):
        prm = L.StepParams(eps_outer=1e-14, max_outer=400, method=method,
                           lo=L.LOParams(eps_inner=1e-14, max_inner=40, elim_rtol=1e-15,
                                         max_elim=80))
        Ts, E, F, Is, mom, st = L.sm_step(cfg, scale, cv, T0, I0, mom0, prm)
        res[method] = np.abs(Ts - T).max() / T.max()
    assert res["consistent"] < 1e-11
    assert res["independent"] > 1e-5
