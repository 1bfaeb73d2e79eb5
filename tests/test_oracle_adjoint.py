"""Pins for the oracle's time-dependent forward problem and discrete adjoint
(leakage objective, gradient w.r.t. per-cell opacity scales):

* the transpose of the upwind operator is the upwind operator of the reversed
  directions: <p, A(Omega)^-1 q> = <A(-Omega)^-1 p, q> for every (d, g);
* the opacity shape f_g(Tbar) equals the oracle's opacity / s, and its
  derivative, and dB_g/dT = 4 a c T^3 r_g, agree with central differences;
* the converged forward step satisfies the pointwise energy balance;
* the adjoint gradient agrees with central finite differences of the
  objective (multigroup Larsen-form opacity and gray power law).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2504_21784_gb300 import workloads as W


def _problem(kind=1, G=3, nx=3, ny=2):
    edges = W.log_edges(G) if G > 1 else W.GRAY_EDGES.copy()
    return A.Problem(nx, ny, (0.0, 1.0, 0.0, 0.8), edges, 1, 2, kind,
                     10.0 if kind == 1 else 0.0, (1.0, 0.0, 0.4, 0.0), dt=0.01)


def test_reversed_sweep_is_the_transpose():
    pb = _problem()
    omx, omy, w = O.quadrature(2, 2, 2)
    ncell = pb.nx * pb.ny
    rng = np.random.default_rng(3)
    sigma = np.exp(rng.uniform(-1, 3, (pb.G, ncell)))
    P1 = rng.standard_normal((len(w), pb.G, ncell, 4))
    P2 = rng.standard_normal((len(w), pb.G, ncell, 4))
    zq = np.zeros((pb.G, ncell, 4))
    zin = np.zeros((4, pb.G))
    x = O.sweep(2, pb.nx, pb.ny, pb.extent, omx, omy, sigma, 1.0, zq, P1, zin)
    y = O.sweep(2, pb.nx, pb.ny, pb.extent, -omx, -omy, sigma, 1.0, zq, P2, zin)
    lhs = np.einsum("dgkn,dgkn->dg", P2, x)
    rhs = np.einsum("dgkn,dgkn->dg", y, P1)
    mag = np.einsum("dgkn,dgkn->dg", np.abs(P2), np.abs(x))  # scale of the sums' rounding
    assert np.max(np.abs(lhs - rhs) / mag) < 1e-14


@pytest.mark.parametrize("kind", [0, 1])
def test_opacity_shape_and_derivative(kind):
    pb = _problem(kind=kind, G=4)
    T = np.array([[0.05, 0.07, 0.06, 0.05], [0.8, 1.1, 0.9, 1.0]])
    Tbar = T.mean(axis=1)
    f, df = A.opacity_shape(pb, Tbar)
    ref = O.opacity(kind, pb.opacity_alpha, pb.edges, T, np.ones(2))
    assert np.max(np.abs(f - ref) / np.abs(ref)) < 1e-14
    h = 1e-6 * Tbar
    fp, _ = A.opacity_shape(pb, Tbar + h)
    fm, _ = A.opacity_shape(pb, Tbar - h)
    # the difference cannot resolve changes of f below its rounding, about
    # eps |f| / h (where e^{-E/T} is below double rounding, f is constant to
    # machine precision and its tiny derivative is invisible): the excess over
    # that bound must be below 1e-6 of the derivative
    excess = np.abs((fp - fm) / (2 * h) - df) - 4 * np.finfo(float).eps * np.abs(f) / h[None, :]
    assert np.max(excess / np.abs(df)) < 1e-6


def test_planck_derivative():
    pb = _problem(G=5)
    T = np.array([[0.03, 0.3, 1.0, 3.0]])
    B4, dB = A.planck_parts(pb, T)
    h = 1e-6 * T
    Bp, _ = A.planck_parts(pb, T + h)
    Bm, _ = A.planck_parts(pb, T - h)
    fd = 4.0 * math.pi * (Bp - Bm) / (2 * h[None])
    assert np.max(np.abs(fd - dB) / np.max(np.abs(dB), axis=0, keepdims=True)) < 1e-7


def _setup(kind, G, seed=1, nsteps=3):
    pb = _problem(kind=kind, G=G)
    ncell = pb.nx * pb.ny
    rng = np.random.default_rng(seed)
    scale = np.exp(0.5 * rng.standard_normal(ncell)) * (1.0 if kind == 1 else 2.0)
    cv = np.full((ncell, 4), 0.3)
    T0 = 0.2 + 0.3 * rng.random((ncell, 4))
    omx, omy, w = O.quadrature(2, pb.n_polar, pb.n_azim)
    B4, _ = A.planck_parts(pb, T0)
    I0 = np.broadcast_to(B4[None], (len(w),) + B4.shape).copy()
    return pb, scale, cv, T0, I0, nsteps


def test_forward_step_satisfies_energy_balance():
    pb, scale, cv, T0, I0, n = _setup(1, 3)
    J, Ts, Is, recs = A.forward(pb, scale, cv, T0, I0, 1)
    omx, omy, w = O.quadrature(2, pb.n_polar, pb.n_azim)
    sigma = O.opacity(1, pb.opacity_alpha, pb.edges, T0, scale)
    B4, _ = A.planck_parts(pb, Ts[1])
    phi = np.einsum("d,dgkn->gkn", w, Is[1])
    rhs = np.einsum("gk,gkn->kn", sigma, phi - 4.0 * math.pi * B4)
    lhs = cv * (Ts[1] - T0) / pb.dt
    assert np.max(np.abs(lhs - rhs)) < 1e-9 * np.max(np.abs(lhs))
    assert J > 0.0


@pytest.mark.parametrize("kind,G", [(1, 3), (0, 1)])
def test_adjoint_gradient_matches_finite_differences(kind, G):
    pb, scale, cv, T0, I0, n = _setup(kind, G)
    J, Ts, Is, _ = A.forward(pb, scale, cv, T0, I0, n)
    g = A.adjoint(pb, scale, cv, Ts, Is)
    fd = np.zeros_like(g)
    for k in range(len(scale)):
        h = 1e-5 * scale[k]
        sp, sm = scale.copy(), scale.copy()
        sp[k] += h
        sm[k] -= h
        fd[k] = (A.forward(pb, sp, cv, T0, I0, n)[0] - A.forward(pb, sm, cv, T0, I0, n)[0]) / (2 * h)
    err = np.max(np.abs(g - fd)) / np.max(np.abs(fd))
    print(f"kind {kind}: max |grad - fd| / max |fd| = {err:.2e}")
    assert err < 1e-6
