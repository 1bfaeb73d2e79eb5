"""FP64 oracle of the gray low-order solve and the full SM step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy / scipy.sparse,
assembled term by term from the weak forms; slow and small-mesh only.

Follows:
* the independent LDG low-order system (Sec. 4) with the LDG fluxes
  F^.n = {F.n} + s/2 [F.n] + c kappa [E],  P^n = n/3 ({E} - s/2 [E]),
  kappa = alpha/2, s = sign(w.n) with w = (1, 1) (w = 1 in 1D), the Marshak-type
  boundary F.n = c alpha E + 2 F_in, and the independent closure source
  R1_ind(v) = int v . sum_g (sigma_F - sigma_g) F_g + int grad_h v : T
              - int_Gamma0 [v] . {T n};
* the semi-implicit backward Euler system (Eq. smm_be) with the HO time-edge
  sources E*, F* (Sec. 6.1, time-edge choice);
* the Newton iteration with frozen gray opacities and nonlinear temperature
  elimination (Sec. 5, Eqs. absem, nonlinear_T_update), each linearised block
  system solved by a sparse direct method (no Krylov method): A_FF is
  diagonal under lumping, so F is eliminated exactly and the Schur complement
  of Eq. schur is factorised by sparse LU; the whole block system can be
  solved directly instead (``LOParams.linear = "block"``), which a pin checks
  gives the same solution;
* Algorithm 1 with the stopping rule Eq. relative_tol.
All forms are lumped with the 2-point Gauss-Lobatto rule (Sec. 6).

Stopping: Eq. relative_tol with epsilon = 1e-3 and the caps of Sec. 6, plus a
round-off guard (stop when the update is below 1e-14 of the iterate).

Readings (where the paper is silent): F_in is the signed incoming partial
current of the boundary source, F_in = -sum_{Omega.n<0} w |Omega.n| I_in, so
that an isotropic inflow in equilibrium satisfies the boundary condition
exactly; gray opacities are nodal (Rem. opacity); T is floored at T_floor.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import (closures, emission, group_spectra, inflow, moments, opacity, quadrature, sweep,
               sweep_pairs, alpha as quad_alpha)


# --------------------------------------------------------------------------- mesh helpers
@dataclasses.dataclass
class Mesh:
    dim: int
    nx: int
    ny: int
    hx: float
    hy: float

    @property
    def ncell(self):
        return self.nx * self.ny

    @property
    def nn(self):
        return 2 if self.dim == 1 else 4

    @property
    def nnode(self):
        return self.ncell * self.nn

    def node(self, ix, iy, a, b=0):
        """global node index of node (a, b) of cell (ix, iy)"""
        return (iy * self.nx + ix) * self.nn + (a if self.dim == 1 else a + 2 * b)

    def mass(self):
        """lumped nodal mass m_n = |K| / 2^dim"""
        return self.hx / 2 if self.dim == 1 else self.hx * self.hy / 4


def make_mesh(dim, nx, ny, extent) -> Mesh:
    x0, x1, y0, y1 = extent
    return Mesh(dim, nx, ny if dim == 2 else 1, (x1 - x0) / nx,
                (y1 - y0) / ny if dim == 2 else 1.0)


def faces(m: Mesh):
    """Yields (kind, n, wf, pairs) for every face.  kind 'int': pairs of
    (node in K1, node in K2) at the face's quadrature points, n the unit normal
    from K1 to K2 (+x or +y); kind 'bdr': pairs (node, None) with n the outward
    normal and side index 0..3 (left, right, bottom, top) attached as n[2]."""
    if m.dim == 1:
        for ix in range(m.nx - 1):
            yield "int", (1.0, 0.0), 1.0, [(m.node(ix, 0, 1), m.node(ix + 1, 0, 0))]
        yield "bdr", (-1.0, 0.0, 0), 1.0, [(m.node(0, 0, 0), None)]
        yield "bdr", (1.0, 0.0, 1), 1.0, [(m.node(m.nx - 1, 0, 1), None)]
        return
    for iy in range(m.ny):
        for ix in range(m.nx - 1):
            yield "int", (1.0, 0.0), 0.5 * m.hy, [(m.node(ix, iy, 1, b), m.node(ix + 1, iy, 0, b))
                                                 for b in range(2)]
    for iy in range(m.ny - 1):
        for ix in range(m.nx):
            yield "int", (0.0, 1.0), 0.5 * m.hx, [(m.node(ix, iy, a, 1), m.node(ix, iy + 1, a, 0))
                                                 for a in range(2)]
    for iy in range(m.ny):
        yield "bdr", (-1.0, 0.0, 0), 0.5 * m.hy, [(m.node(0, iy, 0, b), None) for b in range(2)]
        yield "bdr", (1.0, 0.0, 1), 0.5 * m.hy, [(m.node(m.nx - 1, iy, 1, b), None)
                                                 for b in range(2)]
    for ix in range(m.nx):
        yield "bdr", (0.0, -1.0, 2), 0.5 * m.hx, [(m.node(ix, 0, a, 0), None) for a in range(2)]
        yield "bdr", (0.0, 1.0, 3), 0.5 * m.hx, [(m.node(ix, m.ny - 1, a, 1), None)
                                                 for a in range(2)]


def grad_at_corner(m: Mesh, i_loc, q_loc):
    """gradient of the nodal basis function i at Lobatto point q (cell-local)"""
    if m.dim == 1:
        return ((2 * i_loc - 1) / m.hx,)
    ai, bi = i_loc & 1, i_loc >> 1
    aq, bq = q_loc & 1, q_loc >> 1
    gx = (2 * ai - 1) / m.hx if bq == bi else 0.0
    gy = (2 * bi - 1) / m.hy if aq == ai else 0.0
    return (gx, gy)


# --------------------------------------------------------------------------- operators
def lo_operators(m: Mesh, c: float, alpha: float):
    """Geometry-only pieces of the lumped LDG system (Sec. 4, independent):
    A_EF (zeroth-moment rows, F columns), A_FE (first-moment rows, E
    columns), P (penalty (c alpha/2)[u][E] on interior faces + c alpha u E on
    the boundary).  F unknowns are ordered [node][component]."""
    N, D = m.nnode, m.dim
    mass = m.mass()
    AEF = sp.lil_matrix((N, N * D))
    AFE = sp.lil_matrix((N * D, N))
    P = sp.lil_matrix((N, N))
    # volume terms: -int grad u . F and -(c/3) int div v E, at the Lobatto points
    for k in range(m.ncell):
        base = k * m.nn
        for i in range(m.nn):
            for q in range(m.nn):
                g = grad_at_corner(m, i, q)
                for d in range(D):
                    if g[d] != 0.0:
                        AEF[base + i, (base + q) * D + d] += -mass * g[d]
                        AFE[(base + i) * D + d, base + q] += -(c / 3.0) * mass * g[d]
    for kind, n, wf, pairs in faces(m):
        if kind == "int":
            # s = sign(w . n) = +1 for the +x / +y oriented faces: F^ = F1, E^ = E2
            for n1, n2 in pairs:
                for d in range(D):
                    if n[d] == 0.0:
                        continue
                    # zeroth: int [u] F1.n  ([u] = u1 - u2)
                    AEF[n1, n1 * D + d] += wf * n[d]
                    AEF[n2, n1 * D + d] -= wf * n[d]
                    # first: (c/3) int [v.n] E2
                    AFE[n1 * D + d, n2] += (c / 3.0) * wf * n[d]
                    AFE[n2 * D + d, n2] -= (c / 3.0) * wf * n[d]
                # penalty (c alpha / 2) int [u][E]
                for (iu, su) in ((n1, 1.0), (n2, -1.0)):
                    P[iu, n1] += su * 0.5 * c * alpha * wf
                    P[iu, n2] -= su * 0.5 * c * alpha * wf
        else:
            for nb, _ in pairs:
                P[nb, nb] += c * alpha * wf  # int_Gamma_b c alpha u E
                for d in range(D):
                    if n[d] != 0.0:
                        AFE[nb * D + d, nb] += (c / 3.0) * wf * n[d]  # (c/3) int v.n E
    return AEF.tocsr(), AFE.tocsr(), P.tocsr()


def closure_sources(m: Mesh, clo: np.ndarray, face_term: bool = True):
    """R1_ind(v) for every first-moment test function (Sec. 4, independent),
    from nodal closures (2D: [E,Fx,Fy,Txx,Txy,Tyy,sigE,sigF,sigP,Cx,Cy];
    1D: [E,F,T,sigE,sigF,sigP,C])."""
    N, D = m.nnode, m.dim
    mass = m.mass()
    flat = clo.reshape(N, -1)
    if D == 1:
        Ccorr = flat[:, 6:7]
        Tten = flat[:, 2].reshape(N, 1, 1)
    else:
        Ccorr = flat[:, 9:11]
        Tten = np.zeros((N, 2, 2))
        Tten[:, 0, 0] = flat[:, 3]
        Tten[:, 0, 1] = Tten[:, 1, 0] = flat[:, 4]
        Tten[:, 1, 1] = flat[:, 5]
    r = np.zeros(N * D)
    # int v . sum_g (sigma_F - sigma_g) F_g   (lumped)
    r += (mass * Ccorr).reshape(-1)
    # int grad_h v : T  = sum_q m (grad u_i)_l T_{d l}, for every cell at once
    rc = r.reshape(m.ncell, m.nn, D)
    Tc = Tten.reshape(m.ncell, m.nn, D, D)
    for i in range(m.nn):
        for q in range(m.nn):
            g = grad_at_corner(m, i, q)
            for d in range(D):
                for l in range(D):
                    if g[l] != 0.0:
                        rc[:, i, d] += mass * g[l] * Tc[:, q, d, l]
    # - int_Gamma0 [v] . {T n}
    for kind, n, wf, pairs in faces(m):
        if kind != "int" or not face_term:
            continue
        for n1, n2 in pairs:
            Tn = 0.5 * (Tten[n1] + Tten[n2]) @ np.array(n[:D])
            for d in range(D):
                r[n1 * D + d] -= wf * Tn[d]
                r[n2 * D + d] += wf * Tn[d]
    return r


def boundary_partial_currents(dim, omx, omy, w, I_in_side):
    """2 |F_in| per side: 2 sum_{Omega.n<0} w |Omega.n| I_in (gray I_in)."""
    nrm = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    out = np.zeros(4)
    for s, (nx_, ny_) in enumerate(nrm):
        on = omx * nx_ + (omy * ny_ if dim == 2 else 0.0)
        out[s] = 2.0 * np.sum(w[on < 0] * np.abs(on[on < 0])) * I_in_side[s]
    return out


def boundary_source(m: Mesh, jin2):
    """-2 int_Gamma_b u F_in per node (positive where radiation enters)."""
    b = np.zeros(m.nnode)
    for kind, n, wf, pairs in faces(m):
        if kind == "bdr":
            for nb, _ in pairs:
                b[nb] += wf * jin2[n[2]]
    return b


# --------------------------------------------------------------------------- Newton
@dataclasses.dataclass
class LOParams:
    eps_inner: float = 1e-3
    max_inner: int = 30
    elim_rtol: float = 1e-10
    max_elim: int = 40
    T_floor: float = 1e-8
    linear: str = "schur"      # "schur" (F eliminated, Eq. schur) or "block"
    source_form: str = "factored"  # or "pseudo_fission" (the printed form; see lo_newton)


def eliminate_T(T0, a, c, cv_dt, sigP, sigE, E, Tstar, rtol, maxit, T_floor):
    """Pointwise Newton on (C_v/dt) T + sigma_P a c T^4 = c sigma_E E + (C_v/dt) T*
    (Eq. nonlinear_T_update, lumped).  Returns (T, iterations)."""
    rhs = c * sigE * E + cv_dt * Tstar
    T = T0.copy()
    it_max = 0
    done = np.zeros(T.shape, bool)
    for it in range(1, maxit + 1):
        f = cv_dt * T + sigP * a * c * T ** 4 - rhs
        df = cv_dt + 4.0 * sigP * a * c * T ** 3
        dT = -f / df
        Tn = np.maximum(T + dT, T_floor)
        conv = np.abs(Tn - T) <= rtol * np.abs(Tn)
        T = np.where(done, T, Tn)
        newly = conv & ~done
        done |= conv
        if newly.any():
            it_max = it
        if done.all():
            break
    return T, it_max


def lo_newton(m: Mesh, ops, c, a, dt, alpha, clo, T_k, cv, Estar, Fstar, jin2, T0, E0,
              prm: LOParams, R1=None, bnd=None):
    """Solve the gray LO system with the energy balance (Eq. absem) by the
    Newton-type iteration of Sec. 5 with nonlinear temperature elimination.
    clo: nodal closures; T_k: previous-step temperature T*; cv: nodal C_v;
    Estar, Fstar: time-edge sources; T0, E0: initial guesses.  R1 and bnd
    replace the first-moment closure source and the zeroth-moment boundary
    source of the independent method (the consistent method supplies its own).
    Returns (T, E, F, stats)."""
    AEF, AFE, P = ops
    N, D = m.nnode, m.dim
    mass = m.mass()
    flat = clo.reshape(N, -1)
    sE, sF, sP = (flat[:, 3], flat[:, 4], flat[:, 5]) if D == 1 else (flat[:, 6], flat[:, 7], flat[:, 8])
    inv_cdt = 1.0 / (c * dt)
    sEt, sFt = sE + inv_cdt, sF + inv_cdt
    cv_dt = cv.reshape(-1) / dt
    Tk = T_k.reshape(-1)
    if R1 is None:
        R1 = closure_sources(m, clo)
    bF = mass * inv_cdt * Fstar.reshape(-1) + R1
    AFF = sp.diags(np.repeat(mass * sFt, D))
    if bnd is None:
        bnd = boundary_source(m, jin2)
    T, E = T0.reshape(-1).copy(), E0.reshape(-1).copy()
    u0 = np.concatenate([T, E])
    d1 = None
    stats = {"newton": 0, "elim_max": 0}
    F = np.zeros(N * D)
    for it in range(1, prm.max_inner + 1):
        B0 = a * c * T ** 4
        dB = 4.0 * a * c * T ** 3
        den = cv_dt + sP * dB
        nu = sP * dB / den                     # pseudo-fission coefficient (Eq. pseudo_fission)
        if prm.source_form == "pseudo_fission":
            # as printed: sigma~_E - nu sigma_E and sigma_P B + nu q_T0 with
            # q_T0 = C_v/dt (T* - T) - sigma_P B
            qT0 = cv_dt * (Tk - T) - sP * B0
            coefE = sEt - nu * sE
            src = sP * B0 + nu * qT0
        else:
            # the same two terms with 1 - nu = (C_v/dt) / den written out, so that
            # nu sigma_E is never subtracted from sigma_E, nor nu sigma_P B from
            # sigma_P B: where sigma_P dB >> C_v/dt (optically thick, nu -> 1)
            # those differences cancel catastrophically and the Newton iterates
            # inherit their rounding
            omnu = cv_dt / den
            coefE = sE * omnu + inv_cdt
            src = sP * B0 * omnu + nu * cv_dt * (Tk - T)
        AEE = P + sp.diags(mass * c * coefE)
        bE = mass * (src + Estar.reshape(-1) / dt) + bnd
        if prm.linear == "block":
            K = sp.bmat([[AFF, AFE], [AEF, AEE]], format="csc")
            sol = spla.spsolve(K, np.concatenate([bF, bE]))
            F, E = sol[:N * D], sol[N * D:]
        else:
            # A_FF F + A_FE E = b_F with A_FF diagonal: F = A_FF^{-1}(b_F - A_FE E);
            # then S E = b_E - A_EF A_FF^{-1} b_F with S = A_EE - A_EF A_FF^{-1} A_FE
            # (Eq. schur).  S is symmetric positive definite (Sec. 5), so it is
            # factorised by sparse LU with diagonal pivots (stable for SPD
            # matrices, the LU form of Cholesky) in a symmetric fill-reducing order
            affi = 1.0 / AFF.diagonal()
            S = (AEE - AEF @ sp.diags(affi) @ AFE).tocsc()
            lu = spla.splu(S, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                           options=dict(SymmetricMode=True))
            E = lu.solve(bE - AEF @ (affi * bF))
            F = affi * (bF - AFE @ E)
        T, ite = eliminate_T(T, a, c, cv_dt, sP, sE, E, Tk, prm.elim_rtol, prm.max_elim,
                             prm.T_floor)
        stats["elim_max"] = max(stats["elim_max"], ite)
        stats["newton"] = it
        u1 = np.concatenate([T, E])
        d = np.linalg.norm(u1 - u0)
        if d1 is None:
            d1 = d
        u0 = u1
        # Eq. relative_tol, plus a round-off guard (the first update itself can
        # be at round-off level once the outer iteration has converged)
        if d == 0.0 or d < prm.eps_inner * d1 or d <= 1e-14 * np.linalg.norm(u1):
            break
    return T.reshape(T_k.shape), E.reshape(T_k.shape), F.reshape(N // m.nn, m.nn, D), stats


def schur(m: Mesh, ops, mass_coef_E, sFt):
    """S = A_EE - A_EF A_FF^{-1} A_FE for given nodal coefficients (Eq. schur)."""
    AEF, AFE, P = ops
    D = m.dim
    AFFi = sp.diags(1.0 / np.repeat(m.mass() * sFt, D))
    AEE = P + sp.diags(m.mass() * mass_coef_E)
    return (AEE - AEF @ AFFi @ AFE).toarray()


# --------------------------------------------------------------------------- step
@dataclasses.dataclass
class StepParams:
    eps_outer: float = 1e-3
    max_outer: int = 100
    lo: LOParams = dataclasses.field(default_factory=LOParams)
    method: str = "independent"   # or "consistent" (Sec. 4)


def equilibrium_intensity(cfg, T0, omx):
    """I^0 = B_g(T0)/4pi isotropic at every node ([d][g][cell][node])."""
    G = cfg.n_groups
    ncell, nn = T0.shape
    I = np.zeros((len(omx), G, ncell, nn))
    for k in range(ncell):
        for n in range(nn):
            b, _ = group_spectra(cfg.edges, T0[k, n])
            I[:, :, k, n] = cfg.a * cfg.c * T0[k, n] ** 4 * b[None, :] / (4 * math.pi)
    return I


_OPS_CACHE: dict = {}


def cached_operators(m: Mesh, c: float, alpha: float):
    """lo_operators of a mesh, assembled once and kept for the next steps (they
    depend on the geometry, c and alpha only)."""
    key = (m.dim, m.nx, m.ny, m.hx, m.hy, float(c), float(alpha))
    if key not in _OPS_CACHE:
        if len(_OPS_CACHE) >= 2:
            _OPS_CACHE.clear()
        _OPS_CACHE[key] = lo_operators(m, c, alpha)
    return _OPS_CACHE[key]


def sm_step(cfg, scale, cv, T_k, I_k, mom_k, prm: StepParams):
    """One time step of Algorithm 1 (semi-implicit backward Euler, Eq. smm_be).
    T_k [cell][node], mom_k = HO moments of I_k.  I_k is [d][g][cell][node], or
    a function of d returning direction d's [g][cell][node] intensity: then each
    sweep runs one direction (all its groups) at a time and sums the moments
    direction by direction (they are linear in I), so that the whole intensity
    is never held; the returned I is then None (independent method only).
    Returns (T, E, F, I, mom, stats)."""
    m = make_mesh(cfg.dim, cfg.nx, cfg.ny, cfg.extent)
    omx, omy, w = quadrature(cfg.dim, cfg.n_polar, cfg.n_azim)
    alpha = quad_alpha(omx, w)
    c, a, dt = cfg.c, cfg.a, cfg.dt
    inv_cdt = 1.0 / (c * dt)
    ops = cached_operators(m, c, alpha)
    infl = inflow(cfg.edges, a, c, cfg.T_bdr)
    I_in_side = infl.sum(axis=1)
    jin2 = boundary_partial_currents(cfg.dim, omx, omy, w, I_in_side)
    sigma = opacity(cfg.opacity_kind, cfg.opacity_alpha, cfg.edges, T_k, scale)  # sigma_g(T^k)
    D = cfg.dim
    G = sigma.shape[0]
    streamed = callable(I_k)
    if streamed and prm.method != "independent":
        raise ValueError("the direction-streamed step supports the independent method only")

    def high_order(T):
        q = emission(cfg.edges, a, c, T, sigma)
        if not streamed:
            I = sweep(cfg.dim, cfg.nx, cfg.ny, cfg.extent, omx, omy, sigma, inv_cdt, q, I_k, infl)
            return I, moments(cfg.dim, omx, omy, w, sigma, I)
        mom = np.zeros_like(mom_k)
        for d in range(len(omx)):
            I_d = sweep_pairs(cfg.dim, cfg.nx, cfg.ny, cfg.extent, omx, omy, sigma, inv_cdt, q,
                              I_k(d), infl, [(d, g) for g in range(G)])
            mom += moments(cfg.dim, omx[d:d + 1], omy[d:d + 1], w[d:d + 1], sigma, I_d[None])
        return None, mom

    Estar = mom_k[..., 0] / c                      # HO time-edge sources (Sec. 6.1)
    Fstar = mom_k[..., 1:1 + D]
    T, E = T_k.copy(), Estar.copy()
    u0 = np.concatenate([T.ravel(), E.ravel()])
    d1 = None
    stats = {"outer": 0, "newton": [], "elim_max": 0}
    for it in range(1, prm.max_outer + 1):
        I, mom = high_order(T)
        clo = closures(cfg.dim, cfg.edges, c, sigma, T, mom)
        R1 = bnd = None
        if prm.method == "consistent":
            from .consistent import consistent_sources
            R1, bnd = consistent_sources(m, c, alpha, clo, omx, omy, w, I, I_in_side)
        T, E, F, st = lo_newton(m, ops, c, a, dt, alpha, clo, T_k, cv, Estar, Fstar, jin2, T, E,
                                prm.lo, R1=R1, bnd=bnd)
        stats["newton"].append(st["newton"])
        stats["elim_max"] = max(stats["elim_max"], st["elim_max"])
        stats["outer"] = it
        u1 = np.concatenate([T.ravel(), E.ravel()])
        d = np.linalg.norm(u1 - u0)
        if d1 is None:
            d1 = d
        u0 = u1
        if d == 0.0 or d < prm.eps_outer * d1 or d <= 1e-14 * np.linalg.norm(u1):
            break
    return T, E, F, I, mom, stats
