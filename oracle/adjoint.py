"""FP64 oracle of the time-dependent high-order problem, its right-edge
leakage objective, and the discrete adjoint that gives the objective's
gradient with respect to per-cell opacity scales.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy on top of the
oracle's own sweep; small meshes only.

Forward: the multigroup S_N system of Eq. transport and Eq. energy_balance,
backward Euler in time with the opacities frozen at the start of each step,
sigma^n_{g,K} = s_K f_g(Tbar^n_K) (Sec. 3, Rem. opacity; Sec. 6.2 form), the
lumped upwind DG transport of Eq. dgsn_transport and the lumped (nodal)
energy balance:
    A_{d,g}(sigma~^n) I^{n+1} = sigma^n_g B_g(T^{n+1})/4pi + I^n/(c dt) + inflow
    C_v (T^{n+1} - T^n)/dt = sum_g sigma^n_g (phi^{n+1}_g - B_g(T^{n+1})),
phi_g = sum_d w_d I_{d,g} (= c E_g).  Each step is converged by the
unaccelerated iteration: a sweep with the current T, then the pointwise energy
balance solved for T by Newton with phi fixed, until the relative change of T
is below tol; a final sweep makes I consistent with the final T.

Objective: J = sum_n dt Lambda(I^{n+1}), Lambda the outgoing partial current
through the right edge, lumped at the face's Gauss-Lobatto points:
    Lambda(I) = sum_{d: Omega_x > 0} w_d Omega_x sum_g sum_{right-edge nodes} (h_y/2) I_{d,g}.

Adjoint: the transposed linearisation of the converged discrete system,
stepped backwards in time.  With psi_{d,g} = lambda_{d,g}/w_d (lambda the
multiplier of the transport residual) and theta the multiplier of the energy
balance, step n reads
    A_{d,g}(sigma~^n)^T psi^n = sigma^n_g theta^n + psi^{n+1}/(c dt)
                                + (inflow dt m on the right edge),
    (C_v/dt + sum_g sigma^n_g B'_g) theta^n = sum_g sigma^n_g B'_g phipsi_g/4pi + X^{n+1},
with A(Omega)^T = A(-Omega) (the transposed upwind operator is the upwind
operator of the reversed direction: reversed directions, reversed wavefront),
phipsi_g = sum_d w_d psi_{d,g}, B'_g = dB_g/dT = 4acT^3 r_g (Sec. 2), m the
lumped nodal mass, and X^{n+1} = theta^{n+1} C_v/dt + sum_g G^{n+1}_g
dsigma^{n+1}_g/dT^{n+1} the later step's dependence on T^{n+1}.  The opacity
sensitivity of step n is
    G^n_{g,K} = -sum_{nodes of K} [ sum_d w_d psi I^{n+1} - B_g phipsi_g/4pi
                                    - theta (phi^{n+1}_g - B_g) ],
and dJ/ds_K = sum_n sum_g G^n_{g,K} f_g(Tbar^n_K).  The coupled adjoint step
is converged by the same source iteration as the forward.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

from . import emission, group_spectra, inflow, moments, opacity, quadrature, sweep


@dataclasses.dataclass
class Problem:
    """A 2D time-dependent problem (uniform mesh, Marshak-type isotropic
    inflow B_g(T_bdr)/4pi per side)."""
    nx: int
    ny: int
    extent: tuple
    edges: np.ndarray
    n_polar: int
    n_azim: int
    opacity_kind: int
    opacity_alpha: float
    T_bdr: tuple
    a: float = 1.0
    c: float = 1.0
    dt: float = 0.01

    @property
    def hx(self):
        return (self.extent[1] - self.extent[0]) / self.nx

    @property
    def hy(self):
        return (self.extent[3] - self.extent[2]) / self.ny

    @property
    def G(self):
        return len(self.edges) - 1


def opacity_shape(pb: Problem, Tbar):
    """f_g(Tbar) and df_g/dTbar per [g][cell] (sigma = s f): POWER f = Tbar^-3,
    LARSEN f = alpha (1 - e^{-E_g/Tbar})/E_g^3, E_g the geometric mean of the
    group's edges (Sec. 6.2 form, reading 6)."""
    Tb = np.asarray(Tbar)[None, :]
    if pb.opacity_kind == 0:
        f = np.broadcast_to(Tb ** -3.0, (pb.G, Tb.shape[1])).copy()
        df = np.broadcast_to(-3.0 * Tb ** -4.0, (pb.G, Tb.shape[1])).copy()
        return f, df
    E = np.sqrt(pb.edges[:-1] * pb.edges[1:])[:, None]
    ex = np.exp(-E / Tb)
    f = pb.opacity_alpha * (-np.expm1(-E / Tb)) / E ** 3
    df = -pb.opacity_alpha * ex / (E ** 2 * Tb ** 2)
    return f, df


def planck_parts(pb: Problem, T):
    """B_g(T)/4pi and dB_g/dT per [g][cell][node]: B_g = a c T^4 b_g,
    dB_g/dT = 4 a c T^3 r_g (Sec. 2)."""
    ncell, nn = T.shape
    B = np.zeros((pb.G, ncell, nn))
    dB = np.zeros((pb.G, ncell, nn))
    for k in range(ncell):
        for n in range(nn):
            b, r = group_spectra(pb.edges, T[k, n])
            B[:, k, n] = pb.a * pb.c * T[k, n] ** 4 * b
            dB[:, k, n] = 4.0 * pb.a * pb.c * T[k, n] ** 3 * r
    return B / (4.0 * math.pi), dB


def leakage(pb: Problem, omx, w, I):
    """Lambda(I): outgoing partial current through the right edge (lumped)."""
    nx, ny = pb.nx, pb.ny
    right = [(iy * nx + nx - 1, a_b) for iy in range(ny) for a_b in (1, 3)]  # nodes (a=1, b)
    tot = 0.0
    for d in range(len(omx)):
        if omx[d] <= 0.0:
            continue
        s = sum(I[d, :, k, n].sum() for k, n in right)
        tot += w[d] * omx[d] * 0.5 * pb.hy * s
    return tot


def _solve_energy(pb: Problem, cv, T_old, T_guess, sigma, SE, tol=1e-15, maxit=100):
    """Per node: C_v (T - T_old)/dt + sum_g sigma_g B_g(T) = SE, by Newton."""
    T = T_guess.copy()
    ncell, nn = T.shape
    for k in range(ncell):
        for n in range(nn):
            x = T[k, n]
            for _ in range(maxit):
                b, r = group_spectra(pb.edges, x)
                sB = pb.a * pb.c * x ** 4 * np.dot(sigma[:, k], b)
                dsB = 4.0 * pb.a * pb.c * x ** 3 * np.dot(sigma[:, k], r)
                f = cv[k, n] * (x - T_old[k, n]) / pb.dt + sB - SE[k, n]
                xn = x - f / (cv[k, n] / pb.dt + dsB)
                done = abs(xn - x) <= tol * abs(xn)
                x = xn
                if done:
                    break
            T[k, n] = x
    return T


@dataclasses.dataclass
class StepRecord:
    T_new: np.ndarray
    I_new: np.ndarray
    sweeps: int


def forward(pb: Problem, scale, cv, T0, I0, nsteps: int, tol: float = 1e-13,
            max_iter: int = 500):
    """Returns (J, Ts, Is, records): Ts[n], Is[n] for n = 0..nsteps."""
    omx, omy, w = quadrature(2, pb.n_polar, pb.n_azim)
    infl = inflow(pb.edges, pb.a, pb.c, pb.T_bdr)
    inv_cdt = 1.0 / (pb.c * pb.dt)
    Ts, Is, recs = [T0.copy()], [I0.copy()], []
    J = 0.0
    for n in range(nsteps):
        Tn, In = Ts[-1], Is[-1]
        sigma = opacity(pb.opacity_kind, pb.opacity_alpha, pb.edges, Tn, scale)
        T = Tn.copy()
        it = 0
        for it in range(1, max_iter + 1):
            q = emission(pb.edges, pb.a, pb.c, T, sigma)
            I = sweep(2, pb.nx, pb.ny, pb.extent, omx, omy, sigma, inv_cdt, q, In, infl)
            SE = moments(2, omx, omy, w, sigma, I)[..., 6]
            T_next = _solve_energy(pb, cv, Tn, T, sigma, SE)
            change = np.linalg.norm(T_next - T) / np.linalg.norm(T_next)
            T = T_next
            if change <= tol:
                break
        q = emission(pb.edges, pb.a, pb.c, T, sigma)
        I = sweep(2, pb.nx, pb.ny, pb.extent, omx, omy, sigma, inv_cdt, q, In, infl)
        Ts.append(T)
        Is.append(I)
        recs.append(StepRecord(T, I, it + 1))
        J += pb.dt * leakage(pb, omx, w, I)
    return J, Ts, Is, recs


def adjoint(pb: Problem, scale, cv, Ts: List[np.ndarray], Is: List[np.ndarray],
            tol: float = 1e-13, max_iter: int = 500):
    """Gradient dJ/ds (per cell) from the converged forward states Ts, Is."""
    omx, omy, w = quadrature(2, pb.n_polar, pb.n_azim)
    nsteps = len(Ts) - 1
    ncell, nn = Ts[0].shape
    G = pb.G
    inv_cdt = 1.0 / (pb.c * pb.dt)
    m = 0.25 * pb.hx * pb.hy
    infl_adj = np.zeros((4, G))
    infl_adj[1, :] = pb.dt * m        # the leakage objective enters through the right edge
    grad = np.zeros(ncell)
    psi_next: Optional[np.ndarray] = None
    X_next = np.zeros((ncell, nn))
    for n in range(nsteps - 1, -1, -1):
        Tn, Tn1, I1 = Ts[n], Ts[n + 1], Is[n + 1]
        Tbar = Tn.mean(axis=1)
        f, df = opacity_shape(pb, Tbar)
        sigma = scale[None, :] * f
        B4, dB = planck_parts(pb, Tn1)
        sdB = np.einsum("gk,gkn->kn", sigma, dB)
        theta = np.zeros((ncell, nn))
        psi = None
        for _ in range(max_iter):
            q = sigma[:, :, None] * theta[None, :, :]
            psi = sweep(2, pb.nx, pb.ny, pb.extent, -omx, -omy, sigma, inv_cdt, q,
                        psi_next if psi_next is not None else np.zeros_like(I1), infl_adj)
            phipsi = np.einsum("d,dgkn->gkn", w, psi)
            th_new = (np.einsum("gk,gkn,gkn->kn", sigma, dB, phipsi) / (4.0 * math.pi)
                      + X_next) / (cv / pb.dt + sdB)
            change = np.linalg.norm(th_new - theta) / max(np.linalg.norm(th_new), 1e-300)
            theta = th_new
            if change <= tol:
                break
        q = sigma[:, :, None] * theta[None, :, :]
        psi = sweep(2, pb.nx, pb.ny, pb.extent, -omx, -omy, sigma, inv_cdt, q,
                    psi_next if psi_next is not None else np.zeros_like(I1), infl_adj)
        phipsi = np.einsum("d,dgkn->gkn", w, psi)
        phi = np.einsum("d,dgkn->gkn", w, I1)
        cross = np.einsum("d,dgkn,dgkn->gkn", w, psi, I1)
        Bg = 4.0 * math.pi * B4
        Gn = -(cross - B4 * phipsi - theta[None] * (phi - Bg)).sum(axis=2)  # [g][cell]
        grad += (Gn * f).sum(axis=0)
        X_next = theta * cv / pb.dt + ((Gn * scale[None, :] * df).sum(axis=0) / nn)[:, None]
        psi_next = psi
    return grad
