"""Pins for the oracle's angular moments and closures (Sec. 2: E, F, the SM
tensor T, Eqs. sigmaE, sigmaF, sigma_P, additive_mg_correction; Eq. alpha).

* radiative equilibrium I = a c T^4 b_g / 4pi gives phi = a c T^4, F = 0 and
  T = 0, and sum_g sigma_g E_g = sigma_P a T^4;
* a single non-zero (d, g) intensity isolates every weight and index;
* gray problems reduce to sigma_E = sigma_F = sigma_P = sigma with zero
  additive correction.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_21784_gb300 import workloads as W


def _equilibrium(dim, T, edges, a=1.0, c=1.0, npol=4, naz=3):
    ox, oy, w = O.quadrature(dim, npol, naz) if dim == 2 else O.quadrature(1, npol)
    ncell, nn = T.shape
    G = len(edges) - 1
    I = np.zeros((len(w), G, ncell, nn))
    for k in range(ncell):
        for n in range(nn):
            b, _ = O.group_spectra(edges, T[k, n])
            I[:, :, k, n] = a * c * T[k, n] ** 4 * b[None, :] / (4 * math.pi)
    return ox, oy, w, I


@pytest.mark.parametrize("dim", [1, 2])
def test_equilibrium_moments(dim):
    edges = W.log_edges(6)
    nn = 2 if dim == 1 else 4
    T = W.temperature_random(5, nn, seed=1)
    ox, oy, w, I = _equilibrium(dim, T, edges)
    rng = np.random.default_rng(0)
    sig = rng.uniform(0.1, 10, size=(6, 5))
    mom = O.moments(dim, ox, oy, w, sig, I)
    B = T ** 4
    assert np.allclose(mom[..., 0], B, rtol=1e-14)
    assert np.max(np.abs(mom[..., 1])) < 1e-15 * B.max()
    tens = [2] if dim == 1 else [3, 4, 5]
    for m in tens:
        assert np.max(np.abs(mom[..., m])) < 2e-15 * B.max()
    se = 3 if dim == 1 else 6
    sP = np.zeros_like(T)
    for k in range(5):
        for n in range(nn):
            b, _ = O.group_spectra(edges, T[k, n])
            sP[k, n] = (b * sig[:, k]).sum()
    assert np.allclose(mom[..., se], sP * B, rtol=1e-13)


def test_single_ordinate_isolates_weights():
    ox, oy, w = O.quadrature(2, 2, 2)
    G, ncell = 3, 4
    sig = np.arange(1, G * ncell + 1, dtype=float).reshape(G, ncell)
    d, g, k, n = 5, 2, 3, 1
    I = np.zeros((len(w), G, ncell, 4))
    I[d, g, k, n] = 2.0
    mom = O.moments(2, ox, oy, w, sig, I)
    v = 2.0 * w[d]
    expect = [v, v * ox[d], v * oy[d], v * (ox[d] ** 2 - 1 / 3), v * ox[d] * oy[d],
              v * (oy[d] ** 2 - 1 / 3), sig[g, k] * v, sig[g, k] * v * ox[d], sig[g, k] * v * oy[d]]
    assert np.allclose(mom[k, n], expect, rtol=1e-15)
    mask = np.ones((ncell, 4), bool)
    mask[k, n] = False
    assert np.all(mom[mask] == 0)


@pytest.mark.parametrize("dim", [1, 2])
def test_gray_closures_reduce(dim):
    nn = 2 if dim == 1 else 4
    ox, oy, w = O.quadrature(dim, 4, 2) if dim == 2 else O.quadrature(1, 8)
    rng = np.random.default_rng(3)
    ncell = 6
    sig = rng.uniform(0.5, 5, size=(1, ncell))
    I = rng.uniform(0, 1, size=(len(w), 1, ncell, nn))
    T = W.temperature_random(ncell, nn, seed=4)
    mom = O.moments(dim, ox, oy, w, sig, I)
    out = O.closures(dim, W.GRAY_EDGES, 2.0, sig, T, mom)
    sE, sF, sP = (3, 4, 5) if dim == 1 else (6, 7, 8)
    s = np.repeat(sig[0][:, None], nn, axis=1)
    for j in (sE, sF, sP):
        assert np.allclose(out[..., j], s, rtol=1e-14)
    corr = [6] if dim == 1 else [9, 10]
    for j in corr:
        assert np.max(np.abs(out[..., j])) < 1e-14 * np.abs(mom[..., 1]).max() * s.max()
    assert np.allclose(out[..., 0], mom[..., 0] / 2.0, rtol=1e-15)


def test_multigroup_equilibrium_closures():
    """At equilibrium E_g is proportional to b_g, so sigma_E = sigma_P; with
    all sigma_g equal, sigma_F = sigma too and the correction vanishes."""
    edges = W.log_edges(8)
    T = W.temperature_random(3, 4, seed=7, lo=0.05, hi=1.0)
    ox, oy, w, I = _equilibrium(2, T, edges)
    rng = np.random.default_rng(8)
    sig = np.exp(rng.uniform(-2, 4, size=(8, 3)))
    mom = O.moments(2, ox, oy, w, sig, I)
    out = O.closures(2, edges, 1.0, sig, T, mom)
    assert np.allclose(out[..., 6], out[..., 8], rtol=1e-12)
    sig_eq = np.full((8, 3), 4.0)
    mom2 = O.moments(2, ox, oy, w, sig_eq, I)
    out2 = O.closures(2, edges, 1.0, sig_eq, T, mom2)
    assert np.allclose(out2[..., 6:9], 4.0, rtol=1e-13)


def test_additive_correction_definition():
    """sum_g (sigma_F - sigma_g) F_g with one streaming group."""
    edges = W.log_edges(2)
    ox, oy, w = O.quadrature(2, 2, 2)
    sig = np.array([[3.0], [7.0]])
    I = np.zeros((len(w), 2, 1, 4))
    d = 0
    I[d, 1, 0, :] = 1.0
    T = np.full((1, 4), 0.5)
    mom = O.moments(2, ox, oy, w, sig, I)
    out = O.closures(2, edges, 1.0, sig, T, mom)
    _, r = O.group_spectra(edges, 0.5)
    sF = (r * sig[:, 0]).sum() / r.sum()
    F1 = w[d] * np.array([ox[d], oy[d]])
    assert np.allclose(out[0, :, 9], (sF - 7.0) * F1[0], rtol=1e-13)
    assert np.allclose(out[0, :, 10], (sF - 7.0) * F1[1], rtol=1e-13)
    assert np.allclose(out[0, :, 6], 7.0, rtol=1e-14)


@pytest.mark.parametrize("dim", [1, 2])
def test_sigma_e_falls_back_where_the_energy_weights_are_not_positive(dim):
    """sigma_E = sum_g sigma_g E_g / sum_g E_g (Eq. sigmaE) is a mean of the
    positive group opacities; at nodes where phi <= 0 or SE <= 0 (a lumped
    intensity that dips below zero) it falls back to sigma_P, elsewhere it is
    SE / phi exactly."""
    rng = np.random.default_rng(4)
    edges = W.log_edges(5)
    ncell, nn = 3, 2 if dim == 1 else 4
    nm = 5 if dim == 1 else 9
    T = 0.1 + rng.random((ncell, nn))
    sigma = np.exp(rng.uniform(-1, 3, (5, ncell)))
    mom = rng.uniform(0.1, 1.0, (ncell, nn, nm))
    ise = 3 if dim == 1 else 6
    mom[0, 0, 0] = -0.2            # phi < 0
    mom[1, 1, 0] = 0.0             # phi = 0
    mom[2, 0, ise] = -0.5          # SE < 0
    mom[2, 1, 0] = -0.3            # both negative: a positive ratio, still undefined
    mom[2, 1, ise] = -0.6
    clo = O.closures(dim, edges, 1.0, sigma, T, mom)
    kE, kP = (3, 5) if dim == 1 else (6, 8)
    fallback = {(0, 0), (1, 1), (2, 0), (2, 1)}
    for k in range(ncell):
        for n in range(nn):
            if (k, n) in fallback:
                assert clo[k, n, kE] == clo[k, n, kP]
            else:
                assert clo[k, n, kE] == mom[k, n, ise] / mom[k, n, 0]
