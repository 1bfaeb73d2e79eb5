"""Pins for the oracle's gray low-order solve and step (Sec. 4 independent LDG,
Sec. 5 Newton with nonlinear temperature elimination, Algorithm 1).

* LDG duality: the first-moment E coupling equals -(c/3) times the transpose
  of the zeroth-moment F coupling (what makes the Schur complement symmetric);
* the Schur complement of Eq. schur is symmetric positive definite on tiny
  meshes for lumped forms (Sec. 5);
* discrete energy conservation of one converged Newton solve:
  sum m [(E - E*) + C_v (T - T*)] / dt + boundary net outflow = 0;
* Newton converges quadratically;
* infinite-medium closed system: with uniform data and the boundary inflow at
  the answer's radiation temperature, a full SM step reproduces the scalar
  backward-Euler pair (E - E*)/dt + c sigma E = sigma a c T^4,
  C_v (T - T*)/dt = c sigma E - sigma a c T^4, solved by scalar Newton.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import lo as L
from paper_2504_21784_gb300 import workloads as W


@pytest.mark.parametrize("dim,nx,ny", [(1, 5, 1), (2, 3, 2), (2, 4, 4)])
def test_ldg_duality(dim, nx, ny):
    m = L.make_mesh(dim, nx, ny, (0.0, 1.3, 0.0, 0.7))
    AEF, AFE, P = L.lo_operators(m, c=2.5, alpha=0.47)
    diff = AFE.toarray() + (2.5 / 3.0) * AEF.toarray().T
    assert np.max(np.abs(diff)) < 1e-14
    Pd = P.toarray()
    assert np.max(np.abs(Pd - Pd.T)) < 1e-15


@pytest.mark.parametrize("dim,nx,ny", [(1, 6, 1), (2, 3, 3), (2, 5, 2)])
def test_schur_spd(dim, nx, ny):
    m = L.make_mesh(dim, nx, ny, (0.0, 1.0, 0.0, 1.0))
    ops = L.lo_operators(m, c=1.0, alpha=0.5)
    rng = np.random.default_rng(dim * 10 + nx)
    sEt = np.exp(rng.uniform(-3, 5, m.nnode))
    nu = rng.uniform(0, 0.99, m.nnode)
    sE = sEt * rng.uniform(0.0, 1.0, m.nnode)
    coefE = 1.0 * (sEt - nu * sE)             # c (sigma~_E - nu sigma_E) > 0
    sFt = np.exp(rng.uniform(-3, 5, m.nnode))
    S = L.schur(m, ops, coefE, sFt)
    assert np.max(np.abs(S - S.T)) < 1e-12 * np.abs(S).max()
    np.linalg.cholesky(0.5 * (S + S.T))        # raises unless positive definite


def _lo_case(dim, nx, ny, seed):
    cfg = W.Config("lo", dim, nx, ny if dim == 2 else 1, (0.0, 1.0, 0.0, 1.0), W.log_edges(3),
                   4 if dim == 1 else 2, 0 if dim == 1 else 3, W.OPACITY_LARSEN, 10.0,
                   (1.0, 0.0, 0.3, 0.0), a=1.0, c=1.0, dt=0.01)
    m = L.make_mesh(dim, nx, ny, cfg.extent)
    rng = np.random.default_rng(seed)
    nn = m.nn
    T = W.temperature_random(m.ncell, nn, seed=seed, lo=0.05, hi=1.0)
    sigma = O.opacity(1, 10.0, cfg.edges, T, np.ones(m.ncell))
    omx, omy, w = O.quadrature(dim, cfg.n_polar, cfg.n_azim)
    Ik = W.intensity_random(len(w), 3, m.ncell, nn, seed=seed + 1, scale=0.01)
    mom_k = O.moments(dim, omx, omy, w, sigma, Ik)
    q = O.emission(cfg.edges, 1.0, 1.0, T, sigma)
    infl = O.inflow(cfg.edges, 1.0, 1.0, cfg.T_bdr)
    I = O.sweep(dim, nx, ny, cfg.extent, omx, omy, sigma, 100.0, q, Ik, infl)
    mom = O.moments(dim, omx, omy, w, sigma, I)
    clo = O.closures(dim, cfg.edges, 1.0, sigma, T, mom)
    cv = np.full(T.shape, 0.3)
    alpha = O.alpha(omx, w)
    jin2 = L.boundary_partial_currents(dim, omx, omy, w, infl.sum(axis=1))
    return cfg, m, clo, T, cv, mom_k, alpha, jin2


@pytest.mark.parametrize("dim,nx,ny", [(1, 12, 1), (2, 5, 4)])
def test_lo_energy_conservation(dim, nx, ny):
    cfg, m, clo, T, cv, mom_k, alpha, jin2 = _lo_case(dim, nx, ny, seed=3)
    ops = L.lo_operators(m, 1.0, alpha)
    Estar = mom_k[..., 0]
    Fstar = mom_k[..., 1:1 + dim]
    prm = L.LOParams(eps_inner=1e-14, max_inner=30, elim_rtol=1e-15, max_elim=60)
    Tn, En, Fn, st = L.lo_newton(m, ops, 1.0, 1.0, cfg.dt, alpha, clo, T, cv, Estar, Fstar, jin2,
                                 T, Estar, prm)
    mass = m.mass()
    vol = mass * np.sum((En - Estar) / cfg.dt + cv * (Tn - T) / cfg.dt)
    out = 0.0
    for kind, n, wf, pairs in L.faces(m):
        if kind == "bdr":
            for nb, _ in pairs:
                out += wf * (alpha * En.reshape(-1)[nb] - jin2[n[2]])
    scale = mass * np.sum(np.abs(En - Estar) / cfg.dt) + abs(out)
    assert abs(vol + out) < 1e-11 * scale
    assert st["newton"] >= 2


def test_newton_converges_quadratically():
    cfg, m, clo, T, cv, mom_k, alpha, jin2 = _lo_case(2, 4, 4, seed=5)
    ops = L.lo_operators(m, 1.0, alpha)
    Estar = mom_k[..., 0]
    Fstar = mom_k[..., 1:3]
    ref, _, _, _ = L.lo_newton(m, ops, 1.0, 1.0, cfg.dt, alpha, clo, T, cv, Estar, Fstar, jin2,
                               T, Estar, L.LOParams(eps_inner=1e-15, max_inner=40,
                                                    elim_rtol=1e-15, max_elim=80))
    errs = []
    for k in range(1, 5):
        Tk, _, _, _ = L.lo_newton(m, ops, 1.0, 1.0, cfg.dt, alpha, clo, T, cv, Estar, Fstar,
                                  jin2, T, Estar, L.LOParams(eps_inner=0.0, max_inner=k,
                                                             elim_rtol=1e-15, max_elim=80))
        errs.append(np.max(np.abs(Tk - ref)))
    # the error contracts faster than linearly once it is small
    assert errs[1] < errs[0] and errs[2] < 1e-3 * errs[0] + 1e-14


def _zero_d_answer(sig, cv, dt, a, c, T0):
    Estar = a * T0 ** 4
    T = T0
    for _ in range(200):
        # eliminate E: E = (sig a c T^4 + E*/dt) / (1/dt + c sig)
        E = (sig * a * c * T ** 4 + Estar / dt) / (1.0 / dt + c * sig)
        dEdT = sig * a * c * 4 * T ** 3 / (1.0 / dt + c * sig)
        f = cv * (T - T0) / dt - (c * sig * E - sig * a * c * T ** 4)
        df = cv / dt - (c * sig * dEdT - 4 * sig * a * c * T ** 3)
        T -= f / df
    E = (sig * a * c * T ** 4 + Estar / dt) / (1.0 / dt + c * sig)
    return T, E


@pytest.mark.parametrize("dim", [1, 2])
def test_step_reproduces_infinite_medium(dim):
    T0, s, cv0, dt, a, c = 0.2, 0.5, 0.3, 0.01, 1.0, 1.0
    sig = s / T0 ** 3
    # a cold start heated by an external radiation field: start T0, radiation at T_r
    Tans, Eans = _zero_d_answer(sig, cv0, dt, a, c, T0)
    Tb = (Eans / a) ** 0.25
    nx, ny = (6, 1) if dim == 1 else (3, 3)
    cfg = W.Config("zd", dim, nx, ny, (0.0, 1.0, 0.0, 1.0), W.GRAY_EDGES.copy(),
                   4 if dim == 1 else 2, 0 if dim == 1 else 2, W.OPACITY_POWER, 0.0,
                   (Tb, Tb, Tb if dim == 2 else 0.0, Tb if dim == 2 else 0.0), a=a, c=c, dt=dt)
    ncell = nx * (ny if dim == 2 else 1)
    nn = 2 if dim == 1 else 4
    Tk = np.full((ncell, nn), T0)
    omx, omy, w = O.quadrature(dim, cfg.n_polar, cfg.n_azim)
    Ik = L.equilibrium_intensity(cfg, Tk, omx)
    sigma = O.opacity(0, 0.0, cfg.edges, Tk, np.full(ncell, s))
    mom_k = O.moments(dim, omx, omy, w, sigma, Ik)
    prm = L.StepParams(eps_outer=1e-14, max_outer=200,
                       lo=L.LOParams(eps_inner=1e-14, max_inner=40, elim_rtol=1e-15, max_elim=80))
    T, E, F, I, mom, st = L.sm_step(cfg, np.full(ncell, s), np.full((ncell, nn), cv0), Tk, Ik,
                                    mom_k, prm)
    assert np.max(np.abs(T - Tans)) < 1e-12 * Tans
    assert np.max(np.abs(E - Eans)) < 1e-12 * Eans
    assert np.max(np.abs(mom[..., 0] / c - Eans)) < 1e-11 * Eans
    assert np.max(np.abs(F)) < 1e-11 * c * Eans


@pytest.mark.parametrize("dim,nx,ny", [(1, 12, 1), (2, 5, 4)])
def test_schur_solve_equals_block_solve(dim, nx, ny):
    """Eliminating the diagonal A_FF exactly and solving the Schur complement
    (Eq. schur) gives the solution of the whole linearised block system."""
    cfg, m, clo, T, cv, mom_k, alpha, jin2 = _lo_case(dim, nx, ny, seed=11)
    ops = L.lo_operators(m, 1.0, alpha)
    Estar = mom_k[..., 0]
    Fstar = mom_k[..., 1:1 + dim]
    out = {}
    for linear in ("schur", "block"):
        prm = L.LOParams(eps_inner=1e-14, max_inner=30, elim_rtol=1e-15, max_elim=60,
                         linear=linear)
        out[linear] = L.lo_newton(m, ops, 1.0, 1.0, cfg.dt, alpha, clo, T, cv, Estar, Fstar,
                                  jin2, T, Estar, prm)
    (Ts, Es, Fs, _), (Tb, Eb, Fb, _) = out["schur"], out["block"]
    assert np.max(np.abs(Ts - Tb)) < 1e-13 * np.abs(Tb).max()
    assert np.max(np.abs(Es - Eb)) < 1e-13 * np.abs(Eb).max()
    assert np.max(np.abs(Fs - Fb)) < 1e-12 * np.abs(Eb).max()


@pytest.mark.parametrize("dim,nx,ny", [(1, 12, 1), (2, 5, 4)])
def test_factored_newton_source_equals_printed_form(dim, nx, ny):
    """The Newton linearisation written with 1 - nu = (C_v/dt)/(C_v/dt + sigma_P dB)
    (sigma_E (1 - nu) + 1/(c dt), sigma_P B (1 - nu) + nu C_v/dt (T* - T))
    is the printed pseudo-fission form (sigma~_E - nu sigma_E,
    sigma_P B + nu q_T0, Sec. 5): on a case without stiff cancellation the two
    give the same solve."""
    cfg, m, clo, T, cv, mom_k, alpha, jin2 = _lo_case(dim, nx, ny, seed=13)
    ops = L.lo_operators(m, 1.0, alpha)
    Estar = mom_k[..., 0]
    Fstar = mom_k[..., 1:1 + dim]
    out = {}
    for form in ("factored", "pseudo_fission"):
        prm = L.LOParams(eps_inner=1e-14, max_inner=30, elim_rtol=1e-15, max_elim=60,
                         source_form=form)
        out[form] = L.lo_newton(m, ops, 1.0, 1.0, cfg.dt, alpha, clo, T, cv, Estar, Fstar,
                                jin2, T, Estar, prm)
    (Ta, Ea, _, _), (Tb, Eb, _, _) = out["factored"], out["pseudo_fission"]
    assert np.max(np.abs(Ta - Tb)) < 1e-13 * np.abs(Tb).max()
    assert np.max(np.abs(Ea - Eb)) < 1e-13 * np.abs(Eb).max()
