"""Consistent SM low-order sources (Sec. 4, consistent method) for the lumped
upwind DG transport discretization, 1D slab and 2D.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The consistent method keeps the independent LDG left-hand side and corrects
its right-hand side so that, upon iterative convergence, the low-order
solution equals the moments of the high-order solution.  The corrections are
derived here by the discrete residual approach Sec. 4 describes: take the
zeroth and first angular moments of the lumped upwind DG equations of
Eq. dgsn_transport (test function u_i of node i, Gauss-Lobatto lumping) and
subtract the LDG low-order operator applied to the high-order moments.  Only
the face terms differ; with F^pm_n = sum_{Omega.n >< 0} w (Omega.n) I and
Pi^pm_n = sum_{Omega.n >< 0} w Omega (Omega.n) I (all groups), for node i of
cell K on a face with outward normal n and face weight w_f:

  zeroth moment, interior face (K1 the low side, s = +1):
      R0_i = w_f [ (F.n)(K1) + (c alpha/2)(E_K1 - E_K2) - F^+_n(K1) - F^-_n(K2) ]
    for the node of K1, and its negative for the matching node of K2 (the
    jump form -1/2 [u][beta] + 1/2 [u][F.n] of Sec. 4, beta the closure of
    Eq. smm_bc_analytic);
  zeroth moment, boundary face:
      R0_i = w_f [ J_in + alpha phi_K - F^+_n(K) ]     (J_in = sum_{Omega.n<0} w |Omega.n| I_in)
    which replaces the independent method's 2 w_f J_in;
  first moment, interior face:
      R1_i = w_f [ (c/3) n E_K2 - Pi^+_n(K1) - Pi^-_n(K2) ]   for the node of K1,
      and its negative for the node of K2 (the -[v].{T n} -
      1/2 [v].[Pi^+ - Pi^- + (n/3) phi] terms of Sec. 4);
  first moment, boundary face:
      R1_i = w_f [ (c/3) n E_K - Pi^+_n(K) - Pi_in ]      (Pi_in = sum_{Omega.n<0} w Omega (Omega.n) I_in)
plus the volume terms of the independent method (int v.sum_g (sigma_F -
sigma_g) F_g and int grad v : T).  Reading: the paper's garbled half-range
macros are these quantities, and its phi_HO in the boundary and P terms is the
energy density E_HO (dimensional consistency with c alpha and c/3).

In 1D the faces are points (w_f = 1), n = +-1, and the two half ranges are
the directions with mu > 0 and mu < 0; they are stored in the layout of the 2D
quadrant moments (mu > 0 as quadrant (+,+), mu < 0 as (-,+), the other two
zero; components phi, F, 0, Pi, 0, 0) so that the same half-range sums apply.
"""
from __future__ import annotations

import numpy as np

from . import lo as L

# canonical quadrant order (signs of Omega_x, Omega_y)
QUAD_SIGNS = ((1, 1), (-1, 1), (-1, -1), (1, -1))


def half_moments_1d(mu, w, I):
    """1D: qm[cell][node][q][k] in the 2D quadrant layout: q = 0 sums the
    directions with mu > 0, q = 1 those with mu < 0 (q = 2, 3 zero); k: phi,
    F = sum w mu I, 0, Pi = sum w mu^2 I, 0, 0.  I canonical [d][g][cell][node]."""
    Ig = I.sum(axis=1)
    ncell, nn = Ig.shape[1:]
    qm = np.zeros((ncell, nn, 4, 6))
    for q, sel in ((0, mu > 0), (1, mu < 0)):
        m_, ww, X = mu[sel], w[sel], Ig[sel]
        for k, f in ((0, ww), (1, ww * m_), (3, ww * m_ * m_)):
            qm[:, :, q, k] = np.einsum("d,dkn->kn", f, X)
    return qm


def quadrant_moments(omx, omy, w, I):
    """qm[cell][node][q][k] over all groups, k: phi, F_x, F_y, Pi_xx, Pi_xy,
    Pi_yy with Pi = sum w Omega Omega I; I canonical [d][g][cell][node]."""
    nd = len(w)
    nq = nd // 4
    Ig = I.sum(axis=1)
    ncell, nn = Ig.shape[1:]
    qm = np.zeros((ncell, nn, 4, 6))
    for q in range(4):
        sl = slice(q * nq, (q + 1) * nq)
        ox, oy, ww, X = omx[sl], omy[sl], w[sl], Ig[sl]
        for k, f in enumerate((ww, ww * ox, ww * oy, ww * ox * ox, ww * ox * oy, ww * oy * oy)):
            qm[:, :, q, k] = np.einsum("d,dkn->kn", f, X)
    return qm


def half_range(qm_flat, n):
    """(F^+_n, F^-_n, Pi^+_n, Pi^-_n) per node for an axis-aligned unit normal n."""
    nx, ny = n
    pos = [q for q, (sx, sy) in enumerate(QUAD_SIGNS) if sx * nx + sy * ny > 0]
    neg = [q for q in range(4) if q not in pos]

    def part(qs):
        S = qm_flat[:, qs, :].sum(axis=1)
        Fn = S[:, 1] * nx + S[:, 2] * ny
        Pn = np.stack([S[:, 3] * nx + S[:, 4] * ny, S[:, 4] * nx + S[:, 5] * ny], axis=1)
        return Fn, Pn

    Fp, Pp = part(pos)
    Fm, Pm = part(neg)
    return Fp, Fm, Pp, Pm


def inflow_moments(omx, omy, w, I_in, n):
    """(J_in, Pi_in) of an isotropic inflow I_in through a face with outward normal n."""
    on = omx * n[0] + omy * n[1]
    sel = on < 0
    J = float(np.sum(w[sel] * -on[sel])) * I_in
    Pi = np.array([np.sum(w[sel] * omx[sel] * on[sel]), np.sum(w[sel] * omy[sel] * on[sel])]) * I_in
    return J, Pi


def consistent_sources(m: L.Mesh, c, alpha, clo, omx, omy, w, I, I_in_side):
    """(R1, bnd): the first-moment source (flattened [node][dim]) and the
    zeroth-moment face source (replacing the independent boundary source) of
    the consistent method, from the high-order intensity I [d][g][cell][node],
    the closures clo (volume terms) and the gray inflow per side."""
    D = m.dim
    N = m.nnode
    if D == 1:
        qm = half_moments_1d(omx, w, I).reshape(N, 4, 6)
    else:
        qm = quadrant_moments(omx, omy, w, I).reshape(N, 4, 6)
    tot = qm.sum(axis=1)
    phi = tot[:, 0]
    E = phi / c
    F = tot[:, 1:1 + D]
    hr = {}
    for n in ((1.0, 0.0), (-1.0, 0.0), (0.0, 1.0), (0.0, -1.0)):
        hr[n] = half_range(qm, n)
    R0 = np.zeros(N)
    R1 = L.closure_sources(m, clo, face_term=False).reshape(N, D)
    for kind, n, wf, pairs in L.faces(m):
        nv = np.array(n[:D])
        key = (float(n[0]), float(n[1]))
        Fp, Fm, Pp, Pm = hr[key]
        Pp, Pm = Pp[:, :D], Pm[:, :D]
        if kind == "int":
            for n1, n2 in pairs:
                r0 = wf * (F[n1] @ nv + 0.5 * c * alpha * (E[n1] - E[n2]) - Fp[n1] - Fm[n2])
                R0[n1] += r0
                R0[n2] -= r0
                r1 = wf * ((c / 3.0) * nv * E[n2] - Pp[n1] - Pm[n2])
                R1[n1] += r1
                R1[n2] -= r1
        else:
            side = n[2]
            J_in, Pi_in = inflow_moments(omx, omy, w, I_in_side[side], np.array(n[:2]))
            for nb, _ in pairs:
                R0[nb] += wf * (J_in + alpha * phi[nb] - Fp[nb])
                R1[nb] += wf * ((c / 3.0) * nv * E[nb] - Pp[nb] - Pi_in[:D])
    return R1.reshape(-1), R0
