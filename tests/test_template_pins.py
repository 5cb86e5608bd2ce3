"""Pins for the window-convolution template oracle (Sec. 3.2, Appendix D)."""
import math
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp
from scipy.integrate import quad
from scipy.special import spherical_jn

from oracle import template_oracle as T

F = Fraction


def _coeffs(kind, L, Lp):
    return [sp.Rational(c) for c in T.mixing_coefficients(kind, L, Lp)]


# The paper prints these mixtures in Eq. all_convolutions and in the leakage terms of
# Sec. 4.3 (coefficients of Q_0, Q_2, Q_4, Q_6, Q_8).
PRINTED = {
    ("cross", 2, 2): [1, F(-2, 7), F(1, 21), 0, 0],
    ("cross", 4, 2): [0, F(3, 35), F(-6, 77), F(3, 143), 0],
    ("minus", 4, 4): [1, F(-4, 11), F(18, 143), F(-4, 143), F(7, 2431)],
    ("plus", 0, 0): [1, 0, 0, 0, 0],
    ("plus", 0, 2): [0, F(1, 5), 0, 0, 0],
    ("plus", 0, 4): [0, 0, F(1, 9), 0, 0],
    ("plus", 2, 0): [0, 1, 0, 0, 0],
    ("plus", 2, 2): [1, F(2, 7), F(2, 7), 0, 0],
    ("plus", 2, 4): [0, F(2, 7), F(100, 693), F(25, 143), 0],
    ("plus", 4, 0): [0, 0, 1, 0, 0],
    ("plus", 4, 2): [0, F(18, 35), F(20, 77), F(45, 143), 0],
    ("plus", 4, 4): [1, F(20, 77), F(162, 1001), F(20, 143), F(490, 2431)],
    ("dd", 2, 0): [0, 1, 0, 0, 0],
    ("dd", 0, 0): [1, 0, 0, 0, 0],
}


@pytest.mark.parametrize("key", sorted(PRINTED))
def test_mixing_coefficients_match_paper(key):
    got = _coeffs(*key)
    want = [sp.Rational(f.numerator, f.denominator) for f in map(F, PRINTED[key])]
    assert got == want, (key, got)


@pytest.mark.parametrize("ell", [0, 2, 4])
def test_fftlog_gaussian_pair(ell):
    """int k^(l+2) e^{-a k^2} j_l(kr) dk = sqrt(pi) r^l e^{-r^2/4a} / (2^(l+2) a^(l+3/2))."""
    k, r, delta = T.log_grid()
    a = 25.0
    pk = np.where(np.arange(T.N_FFT) < T.N_IN, k ** ell * np.exp(-a * k * k), 0.0)
    xi = T.hankel_inverse(pk, ell)
    want = (1j ** ell).real / (2 * math.pi ** 2) * math.sqrt(math.pi) * r ** ell * np.exp(-r * r / (4 * a)) / (
        2 ** (ell + 2) * a ** (ell + 1.5))
    sel = (r > 0.5) & (r < 60.0)
    scale = np.abs(want[sel]).max()
    assert np.max(np.abs(xi[sel] - want[sel])) < 1e-7 * scale


@pytest.mark.parametrize("ell", [2, 8, 10, 12])
def test_fftlog_forward_gaussian_pair(ell):
    """The forward transform of the output slots' orders, up to the minus moments L = 10, 12:
    4 pi (-i)^l int r^(l+2) e^{-b r^2} j_l(kr) dr = 4 pi (-i)^l sqrt(pi) k^l e^{-k^2/4b} / (2^(l+2) b^(l+3/2))."""
    k, r, delta = T.log_grid()
    for b in (0.01, 0.001):
        pk = T.hankel_forward(r ** ell * np.exp(-b * r * r), ell)
        want = 4.0 * math.pi * ((-1j) ** ell).real * math.sqrt(math.pi) * k ** ell * np.exp(-k * k / (4 * b)) / (
            2 ** (ell + 2) * b ** (ell + 1.5))
        sel = (k > 1e-3) & (k < 3.0)
        assert np.max(np.abs(pk[sel] - want[sel])) < 1e-10 * np.abs(want[sel]).max()


def test_fftlog_matches_direct_quadrature():
    """H^-1_l of the (tapered) BBKS spectrum against adaptive quadrature of the same integrand."""
    from scipy.interpolate import interp1d
    k, r, delta = T.log_grid()
    params = (1.0, 1.5, 0.8, 0.0, 0.2, 1.0)
    pk = T.linear_pk(params)
    norm = pk[100] / T.bbks_shape(k[100], 0.2, 0.0)
    tp = interp1d(np.log(k[:T.N_IN]), T.taper(), kind="cubic")
    for ell in (0, 2):
        xi = T.hankel_inverse(pk, ell)
        sel = (r > 5.0) & (r < 200.0)
        scale = np.abs(xi[sel]).max()
        for rr in (5.0, 20.0, 80.0, 150.0):
            m = int(np.argmin(np.abs(r - rr)))
            f = lambda kk: (kk * kk * norm * T.bbks_shape(kk, 0.2, 0.0) * float(tp(np.log(kk)))
                            * spherical_jn(ell, kk * r[m]) / (2 * math.pi ** 2))
            val, _ = quad(f, T.K_MIN, T.K_MAX, limit=8000, epsabs=1e-14, epsrel=1e-11)
            val *= (1j ** ell).real
            assert abs(xi[m] - val) < 1e-6 * scale, (ell, rr, xi[m], val)


def test_round_trip_and_unit_window():
    """A window with Q_0 = exp(-(r/R)^2), Q_l>0 = 0 and R large smooths by ~1/R only, so
    Pt^(L)_X tends to the model multipole P^(L)_X at k >> 1/R (the window convolution is the
    identity in that limit, Eq. window_convolution_X_hankel)."""
    k, r, delta = T.log_grid()
    params = (1.2, 1.7, 0.8, 0.05, 0.21, 1.0)
    s = np.geomspace(0.01, 9000.0, 400)
    qt = np.zeros((5, s.size))
    qt[0] = np.exp(-(s / 3000.0) ** 2)
    edges = np.linspace(0.03, 0.2, 10)
    tmpl = T.template(params, qt, s, edges)
    pk = T.linear_pk(params)
    model = T.model_multipoles(params)
    for i, (kind, L) in enumerate(T.SLOTS):
        want = T.bin_average(model[kind].get(L, 0.0) * pk, edges)
        scale = np.abs(T.bin_average(model[kind][min(model[kind])] * pk, edges))
        assert np.max(np.abs(tmpl[i] - want) / scale) < 2e-3, (kind, L, np.max(np.abs(tmpl[i] - want) / scale))


def test_gaussian_sigma_against_monte_carlo():
    """The Gaussian error bars against the scatter of the multipole estimator over Gaussian
    realisations: N_k / 2 independent complex modes per shell, uniform in mu (isotropic
    power; the mu of the modes are fixed by the grid, the same in every realisation),
    P_ab^(l) = (2l+1) <Re(d_a d_b*) L_l(mu)>."""
    from scipy.special import eval_legendre
    rng = np.random.default_rng(12)
    n_k, reals = 400, 20000
    k1 = 0.05
    volume = n_k * 6.0 * math.pi ** 2 / k1 ** 3
    pgg, pee, pbb, pge = 3.0, 2.0, 0.7, 0.9
    chol = np.linalg.cholesky(np.array([[pgg, pge], [pge, pee]]))
    m = n_k // 2
    z = (rng.standard_normal((reals, m, 3)) + 1j * rng.standard_normal((reals, m, 3))) / math.sqrt(2.0)
    dg = chol[0, 0] * z[..., 0]
    de = chol[1, 0] * z[..., 0] + chol[1, 1] * z[..., 1]
    db = math.sqrt(pbb) * z[..., 2]
    mu = -1.0 + (np.arange(m) + 0.5) * (2.0 / m)
    noise_e = 0.5
    p0 = np.array([[pgg], [pge], [pee - noise_e], [pbb - noise_e]])
    want = T.gaussian_sigma(p0, np.array([0.0, k1]), volume, 0.0, noise_e)[:, 0]
    pairs = [(dg, de), (dg, de), (de, de), (de, de), (de, de), (db, db), (db, db), (db, db)]
    for c, (ell, (a, b)) in enumerate(zip([0, 2, 0, 2, 4, 0, 2, 4], pairs)):
        est = (2 * ell + 1) * np.mean((a * np.conj(b)).real * eval_legendre(ell, mu), axis=1)
        got = est.std()
        assert abs(got / want[c] - 1.0) < 0.04, (c, got, want[c])


def _bbks_published(k, gamma, tilt):
    """Bardeen, Bond, Kaiser & Szalay (1986), Eq. G3: T(q) = ln(1 + 2.34 q)/(2.34 q)
    [1 + 3.89 q + (16.1 q)^2 + (5.46 q)^3 + (6.71 q)^4]^(-1/4), q = k / Gamma; P = k^(1+tilt) T^2."""
    q = k / gamma
    t = math.log(1.0 + 2.34 * q) / (2.34 * q) * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3
                                                 + (6.71 * q) ** 4) ** -0.25
    return k ** (1.0 + tilt) * t * t


@pytest.mark.parametrize("params", [(1.0, 1.5, 0.8, 0.0, 0.2, 1.0), (0.3, 2.2, 0.65, -0.15, 0.12, 1.0),
                                    (2.5, 1.1, 0.97, 0.18, 0.29, 0.6)])
def test_linear_pk_sigma8_normalisation(params):
    """sigma_8^2 = int dk/k k^3 P(k) W_TH(8k)^2 / (2 pi^2) with the top hat W(x) = 3 (sin x - x cos x)/x^3.

    The oracle's P(k) must be the published BBKS shape times one constant (checked at every
    tenth grid point), and the integral, done here by adaptive quadrature over the input range
    [1e-4, 10] of the oracle's reading, must equal the requested sigma_8^2 to 1e-8.  Over
    (0, inf) the truncated range costs under 1e-5.  A wrong 2 pi^2, top-hat factor or BBKS
    coefficient fails this test."""
    from scipy.integrate import quad
    k, r, delta = T.log_grid()
    pk = T.linear_pk(params)
    gam, tilt, s8 = params[4], params[3], params[2]
    ratio = np.array([pk[i] / _bbks_published(k[i], gam, tilt) for i in range(0, T.N_IN, 10)])
    norm = ratio[0]
    assert np.max(np.abs(ratio / norm - 1.0)) < 1e-12
    assert np.all(pk[T.N_IN:] == 0.0)

    def w_th(x):
        return 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3

    def f(lk):
        kk = math.exp(lk)
        return kk ** 3 * norm * _bbks_published(kk, gam, tilt) * w_th(8.0 * kk) ** 2 / (2.0 * math.pi ** 2)

    edges = np.log(np.geomspace(T.K_MIN, T.K_MAX, 200))
    s2 = sum(quad(f, a, b, epsabs=0.0, epsrel=1e-13, limit=200)[0] for a, b in zip(edges[:-1], edges[1:]))
    assert s2 == pytest.approx(s8 * s8, rel=1e-8)
    tail = quad(f, math.log(T.K_MAX), math.log(1e3), epsabs=0.0, epsrel=1e-10, limit=4000)[0] + \
        quad(f, math.log(1e-9), math.log(T.K_MIN), epsabs=0.0, epsrel=1e-10)[0]
    assert tail < 1e-5 * s8 * s8


def test_png_response_on_the_right_families():
    """Spin-2 PNG (Sec. 5) through a broad unit window (the identity, as in
    test_round_trip_and_unit_window): the density slots keep the Gaussian model, the cross
    slot follows the model times the response factor once and the plus / minus slots times
    it twice; the factor is 1 + 12 f_NL db_IA / M with M -> (2/3) k^2 (c/H0)^2 / Omega_m at
    small k (T -> 1), c / H0 = 299792.458 km/s over 100 km/s/Mpc.  f_NL = -20 (about the CMB
    bound): a much larger |f_NL| makes the squared factor grow as k^-4 at the lowest k, and that
    power leaks through any window of finite width, so the unit-window identity no longer holds."""
    params = (1.2, 1.7, 0.8, 0.05, 0.21, 1.0)
    png = (-20.0, 0.17, 0.3)
    s = np.geomspace(0.01, 9000.0, 400)
    qt = np.zeros((5, s.size))
    qt[0] = np.exp(-(s / 3000.0) ** 2)
    edges = np.linspace(0.03, 0.2, 10)
    tmpl = T.template(params, qt, s, edges, png=png)
    k, r, delta = T.log_grid()
    pk = T.linear_pk(params)
    f = np.ones(T.N_FFT)
    f[:T.N_IN] = T.png_factor(k[:T.N_IN], params[4], *png)
    model = T.model_multipoles(params)
    power = {"dd": 0, "cross": 1, "plus": 2, "minus": 2}
    for i, (kind, L) in enumerate(T.SLOTS):
        want = T.bin_average(model[kind].get(L, 0.0) * pk * f ** power[kind], edges)
        scale = np.abs(T.bin_average(model[kind][min(model[kind])] * pk * f ** power[kind], edges))
        assert np.max(np.abs(tmpl[i] - want) / scale) < 3e-3, (kind, L)
    # the small-k limit of M, and f_NL = 0 is the Gaussian template
    kk = 1e-6
    m_small = 12.0 * 0.17 * (-180.0) / (T.png_factor(kk, 0.21, -180.0, 0.17, 0.3) - 1.0)
    assert m_small / kk ** 2 == pytest.approx((2.0 / 3.0) * (299792.458 / 100.0) ** 2 / 0.3, rel=1e-4)
    np.testing.assert_array_equal(T.template(params, qt, s, edges, png=(0.0, 0.17, 0.3)),
                                  T.template(params, qt, s, edges))
