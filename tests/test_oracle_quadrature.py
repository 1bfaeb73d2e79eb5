"""Pins for the oracle's angular quadrature (Sec. 2 {Omega_d, w_d}; Eq. alpha).

Checked against numpy's Gauss-Legendre routine, exact angular moments, and a
closed form for alpha of the product set."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n", list(range(1, 21)) + [32])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 2e-15
    assert np.max(np.abs(w - wr)) < 2e-14


@pytest.mark.parametrize("n", [2, 4, 6, 8, 16])
def test_1d_set_moments(n):
    mu, _, w = O.quadrature(1, n)
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    assert abs((w * mu).sum()) < 1e-14
    assert abs((w * mu * mu).sum() - 4 * math.pi / 3) < 1e-13
    assert np.all(np.diff(mu) > 0)


@pytest.mark.parametrize("npol,naz", [(1, 1), (2, 4), (4, 4), (4, 8), (3, 5)])
def test_2d_set_moments_and_symmetry(npol, naz):
    ox, oy, w = O.quadrature(2, npol, naz)
    assert len(w) == 4 * npol * naz
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    assert abs((w * ox).sum()) < 1e-14 and abs((w * oy).sum()) < 1e-14
    assert abs((w * ox * oy).sum()) < 1e-14
    if npol >= 2:  # second moments need a polar rule exact for degree 2
        assert abs((w * ox * ox).sum() - 4 * math.pi / 3) < 1e-13
        assert abs((w * oy * oy).sum() - 4 * math.pi / 3) < 1e-13
    assert np.all(ox * ox + oy * oy < 1.0)
    # quadrant-major order with signs (+,+), (-,+), (-,-), (+,-)
    k = npol * naz
    signs = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    for q, (sx, sy) in enumerate(signs):
        assert np.all(np.sign(ox[q * k:(q + 1) * k]) == sx)
        assert np.all(np.sign(oy[q * k:(q + 1) * k]) == sy)
    # x <-> y symmetry of the set
    a = np.sort(np.round(np.c_[ox, oy, w], 14), axis=0)
    b = np.sort(np.round(np.c_[oy, ox, w], 14), axis=0)
    assert np.allclose(a, b, atol=1e-14)


@pytest.mark.parametrize("npol,naz", [(2, 4), (4, 4), (4, 8), (8, 16)])
def test_alpha_closed_form(npol, naz):
    """alpha = sum w |Omega_x| / 4pi.  For the product set the azimuthal
    midpoint sum of cos is 1/(2 sin(pi/(4 n_a))), giving
    alpha = [sum_p w_p sqrt(1 - xi_p^2)] / (2 n_a sin(pi/(4 n_a)))."""
    ox, oy, w = O.quadrature(2, npol, naz)
    xg, wg = np.polynomial.legendre.leggauss(2 * npol)
    pos = xg > 0
    expect = (wg[pos] * np.sqrt(1 - xg[pos] ** 2)).sum() / (2 * naz * math.sin(math.pi / (4 * naz)))
    assert abs(O.alpha(ox, w) - expect) < 1e-14
    assert abs(O.alpha(oy, w) - expect) < 1e-14
    assert abs(expect - 0.5) < 0.05


def test_alpha_1d():
    mu, _, w = O.quadrature(1, 8)
    xg, wg = np.polynomial.legendre.leggauss(8)
    assert abs(O.alpha(mu, w) - 0.5 * (wg * np.abs(xg)).sum()) < 1e-14
