"""Pins for the oracle's Planck / Rosseland integrals, opacity and sources
(Sec. 2: Eq. planck, Eq. black_body, b_g, r_g, dB_g/dT = 4acT^3 r_g;
Sec. 3 Rem. opacity; Sec. 6.2 opacity form).

Checked against adaptive quadrature (scipy), the zeta-function closed form of
the Bernoulli numbers (scipy.special.zeta), the normalisations sum b = sum r = 1,
branch agreement, a central difference, and asymptotic limits."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2504_21784_gb300 import workloads as W

C15 = 15 / math.pi ** 4


def _quad_P(x):
    f = lambda t: t ** 3 / math.expm1(t) if t > 0 else 0.0
    return C15 * integrate.quad(f, 0, x, epsabs=1e-300, epsrel=1e-13, limit=400)[0]


def _quad_R(x):
    f = lambda t: t ** 4 * math.exp(t) / math.expm1(t) ** 2 if 0 < t < 700 else 0.0
    return 0.25 * C15 * integrate.quad(f, 0, x, epsabs=1e-300, epsrel=1e-13, limit=400)[0]


XS = [1e-4, 1e-2, 0.3, 1.0, 1.7, 1.99, 2.0, 2.01, 2.5, 4.0, 8.0, 15.0, 30.0]


@pytest.mark.parametrize("x", XS)
def test_P_matches_adaptive_quadrature(x):
    assert abs(O.planck_P(x) - _quad_P(x)) <= 5e-14 * _quad_P(x) + 1e-300


@pytest.mark.parametrize("x", XS)
def test_R_matches_adaptive_quadrature(x):
    assert abs(O.rosseland_R(x) - _quad_R(x)) <= 5e-14 * _quad_R(x) + 1e-300


@pytest.mark.parametrize("x", [2.0, 5.0, 10.0, 30.0])
def test_tail_Q_matches_quadrature_of_tail(x):
    """1 - P(x) from the tail series keeps full relative accuracy."""
    f = lambda t: t ** 3 / math.expm1(t) if t < 700 else 0.0
    tail = C15 * integrate.quad(f, x, np.inf, epsabs=1e-300, epsrel=1e-13, limit=400)[0]
    assert abs(O.planck_Q(x) - tail) <= 1e-13 * tail


@pytest.mark.parametrize("x", [0.5, 1.0, 2.0, 2.5, 3.0])
def test_series_branches_agree(x):
    assert abs(O.planck_P_head(x) - O.planck_P_tail(x)) < 1e-14


def test_limits():
    assert O.planck_P(0.0) == 0.0
    assert O.planck_P(np.inf) == 1.0
    assert abs(O.planck_P(60.0) - 1.0) < 1e-16
    assert O.rosseland_R(np.inf) == 1.0
    # small-x leading term (15/pi^4) x^3 / 3
    x = 1e-3
    assert abs(O.planck_P(x) / (C15 * x ** 3 / 3) - 1) < 1e-3


@pytest.mark.parametrize("k", range(1, 25))
def test_bernoulli_coefficients_zeta(k):
    """B_2k/(2k)! = (-1)^(k+1) 2 zeta(2k) / (2 pi)^(2k)."""
    exact = (-1) ** (k + 1) * 2 * special.zeta(2 * k) / (2 * math.pi) ** (2 * k)
    got = O.bernoulli_over_factorial(2 * k)
    assert abs(got / exact - 1) < 1e-12
    assert O.bernoulli_over_factorial(2 * k + 1) == pytest.approx(0.0, abs=1e-17)
    assert O.bernoulli_over_factorial(1) == pytest.approx(-0.5, abs=1e-16)


@pytest.mark.parametrize("T", [0.01, 0.05, 0.3, 1.0, 7.0])
@pytest.mark.parametrize("G", [1, 3, 16, 64])
def test_group_spectra_normalised(T, G):
    edges = W.log_edges(G)
    b, r = O.group_spectra(edges, T)
    assert abs(b.sum() - 1) < 1e-14 and abs(r.sum() - 1) < 1e-14
    assert np.all(b >= 0) and np.all(r >= 0)


@pytest.mark.parametrize("T", [0.02, 0.2, 1.0])
def test_group_spectra_against_quadrature(T):
    edges = W.log_edges(8)
    b, r = O.group_spectra(edges, T)
    lo = np.r_[0.0, edges[1:-1] / T]
    hi = np.r_[edges[1:-1] / T, np.inf]
    f = lambda t: t ** 3 / math.expm1(t) if 0 < t < 700 else 0.0
    for g in range(8):
        ref = C15 * integrate.quad(f, lo[g], hi[g], epsabs=1e-300, epsrel=1e-12, limit=400)[0]
        assert abs(b[g] - ref) <= 1e-11 * ref + 1e-300


@pytest.mark.parametrize("T", [0.03, 0.25, 1.0])
def test_dBg_dT_is_rosseland(T):
    """dB_g/dT = 4 a c T^3 r_g (Sec. 2), central difference."""
    a, c = 1.7, 0.9
    edges = W.log_edges(12)
    h = 1e-5 * T
    bp, _ = O.group_spectra(edges, T + h)
    bm, _ = O.group_spectra(edges, T - h)
    _, r = O.group_spectra(edges, T)
    Bp = a * c * (T + h) ** 4 * bp
    Bm = a * c * (T - h) ** 4 * bm
    fd = (Bp - Bm) / (2 * h)
    exact = 4 * a * c * T ** 3 * r
    big = exact > 1e-8 * exact.max()
    assert np.max(np.abs(fd[big] - exact[big]) / exact[big]) < 1e-7


def test_emission_sums_to_gray_planck():
    """With equal sigma_g, sum_g q_g = sigma a c T^4 / 4pi (sum b_g = 1)."""
    edges = W.log_edges(10)
    T = W.temperature_random(7, 4, seed=3)
    sig = np.full((10, 7), 2.5)
    q = O.emission(edges, 1.3, 0.7, T, sig)
    assert np.allclose(q.sum(axis=0), 2.5 * 1.3 * 0.7 * T ** 4 / (4 * math.pi), rtol=1e-14)
    assert np.all(q >= 0)


def test_inflow_gray_and_vacuum():
    edges = W.log_edges(5)
    infl = O.inflow(edges, 1.0, 1.0, [1.0, 0.0, 0.5, -1.0])
    assert abs(infl[0].sum() - 1 / (4 * math.pi)) < 1e-15
    assert abs(infl[2].sum() - 0.5 ** 4 / (4 * math.pi)) < 1e-16
    assert np.all(infl[1] == 0) and np.all(infl[3] == 0)


def test_opacity_power_law_and_cell_mean():
    T = np.array([[0.1, 0.1, 0.1, 0.1], [0.1, 0.3, 0.2, 0.2]])
    s = np.array([2.0, 3.0])
    sig = O.opacity(0, 0.0, W.GRAY_EDGES, T, s)
    assert sig.shape == (1, 2)
    assert abs(sig[0, 0] - 2.0 / 0.1 ** 3) < 1e-9
    # cell mean of (0.1, 0.3, 0.2, 0.2) is 0.2; node permutation does not matter
    assert abs(sig[0, 1] - 3.0 / 0.2 ** 3) < 1e-9
    sig2 = O.opacity(0, 0.0, W.GRAY_EDGES, T[:, ::-1].copy(), s)
    assert np.allclose(sig, sig2, rtol=1e-15)


def test_opacity_larsen_limits():
    """sigma_g -> s alpha / E_g^3 (T -> 0) and -> s alpha / (T E_g^2) (T -> inf)."""
    edges = W.log_edges(4)
    Eg = np.sqrt(edges[:-1] * edges[1:])
    cold = O.opacity(1, 10.0, edges, np.full((1, 4), 1e-6), np.array([2.0]))[:, 0]
    assert np.allclose(cold, 2.0 * 10.0 / Eg ** 3, rtol=1e-14)
    hot = O.opacity(1, 10.0, edges, np.full((1, 4), 1e9), np.array([2.0]))[:, 0]
    assert np.allclose(hot, 2.0 * 10.0 / (1e9 * Eg ** 2), rtol=1e-6)
