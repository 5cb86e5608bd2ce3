"""FP64 CPU oracle for window-convolved theory templates (Sec. 3.2, Appendix D).

TEST INFRASTRUCTURE ONLY: imported by the test-suite and the cpu-baseline leg of the
benchmark, never by the product path; it shares no code with the CUDA library.

The window-convolved multipole of statistic X (Eqs. window_convolution_X,
window_convolution_X_hankel, def_of_Q_llp) is

    Pt^(L)_X(k) = H_L[ sum_L' Q^X_LL'(r) xi^(L')_X(r) ](k),   xi^(L')_X = H^-1_L'[P^(L')_X],
    Q^X_LL'(r) = sum_l'' Q_l''(r) (2L+1) sqrt((L-m)!/(L+m)! (L'+m)!/(L'-m)!)
                 (l'' L L'; 0 0 0)(l'' L L'; 0 m -m),      (X, m) in {(dd,0), (gd,2), (+,0), (-,4)}

with H_l[g](k) = 4 pi (-i)^l int r^2 dr j_l(kr) g(r) and
H^-1_l[P](r) = i^l int k^2 dk/(2 pi^2) j_l(kr) P(k) (Sec. 1 conventions).

Hankel transforms use the FFTLog method of Hamilton (2000), which the paper cites (Sec. 3.2):
A(k) k^-q is expanded in a discrete Fourier series in ln k, each term transformed with
the Mellin transform of j_l,

    int_0^inf x^(s-1) j_l(x) dx = 2^(s-2) sqrt(pi) Gamma((l+s)/2) / Gamma((3+l-s)/2).

Readings where the paper is silent: 2048 log-spaced k in [1e-4, 10],
zero padding to 4096, k_0 r_0 = exp(-(N-1) Delta), biases q = 1.5 (inverse) and 0.5
(forward), the Nyquist coefficient replaced by its real part; the input spectrum tapered
to zero over the lowest and highest 10% of the log-k range by t - sin(2 pi t)/(2 pi) (a
hard cut at k = 10 would make the log-Fourier series ring); Q_l(r) linearly interpolated
from the measured table, held at its first value below the first separation and zero
beyond the last; bin averages weighted by k^3 on the log grid; the tidal-alignment model
with shapes e = -A T and galaxies b_g delta (Eq. power_for_validation scaled), BBKS P(k)
normalised to sigma_8 by trapezoid quadrature on the same log grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import loggamma

N_IN = 2048
N_FFT = 4096
K_MIN = 1.0e-4
K_MAX = 10.0
Q_INV = 1.5
Q_FWD = 0.5

# output slots in the order of the estimator (dd0, cross2,4,6, plus0,2,4, minus4,6,8, dd2,4,
# minus10,12); the density quadrupole and hexadecapole of the model (no redshift-space
# distortions) are pure window leakage of the monopole, the mixtures Q^dd_20 and Q^dd_40
# (Sec. 4.3), and so are the minus moments L = 10, 12 of the minus hexadecapole (Q^-_L4 with
# the window multipoles l'' = 6, 8 for L = 10 and l'' = 8 for L = 12)
SLOTS = [("dd", 0), ("cross", 2), ("cross", 4), ("cross", 6), ("plus", 0), ("plus", 2), ("plus", 4),
         ("minus", 4), ("minus", 6), ("minus", 8), ("dd", 2), ("dd", 4), ("minus", 10), ("minus", 12)]
M_OF = {"dd": 0, "cross": 2, "plus": 0, "minus": 4}


def log_grid():
    """k_n (N_IN points), Delta, the padded k grid and the r grid with k_0 r_0 = e^{-(N-1) Delta}."""
    delta = math.log(K_MAX / K_MIN) / (N_IN - 1)
    n = np.arange(N_FFT)
    k = K_MIN * np.exp(n * delta)
    r0 = math.exp(-(N_FFT - 1) * delta) / K_MIN
    r = r0 * np.exp(n * delta)
    return k, r, delta


# ------------------------------------------------------------------ Wigner mixing
def wigner3j(j1, j2, j3, m1, m2, m3):
    from sympy.physics.wigner import wigner_3j
    return wigner_3j(j1, j2, j3, m1, m2, m3)


def mixing_coefficients(kind: str, L: int, Lp: int, lmax: int = 8):
    """Exact coefficients of Q_l'' (l'' = 0, 2, ..., lmax) in Q^X_LL' (Eq. def_of_Q_llp)."""
    import sympy as sp
    m = M_OF[kind]
    pref = (2 * L + 1) * sp.sqrt(sp.factorial(L - m) / sp.factorial(L + m) * sp.factorial(Lp + m) / sp.factorial(Lp - m))
    out = []
    for lpp in range(0, lmax + 1, 2):
        out.append(sp.nsimplify(sp.simplify(pref * wigner3j(lpp, L, Lp, 0, 0, 0) * wigner3j(lpp, L, Lp, 0, m, -m))))
    return out


# ------------------------------------------------------------------ FFTLog
def mellin_jl(ell: int, s: np.ndarray) -> np.ndarray:
    """int_0^inf x^(s-1) j_l(x) dx for complex s with -l < Re s < 2."""
    return np.exp((s - 2.0) * math.log(2.0) + 0.5 * math.log(math.pi)
                  + loggamma(0.5 * (ell + s)) - loggamma(0.5 * (3.0 + ell - s)))


def fftlog_kernel(ell: int, q: float, delta: float, kr0: float) -> np.ndarray:
    """u_alpha = (k_0 r_0)^{-i eta} M_l(q + i eta), eta = 2 pi alpha / (N Delta), alpha in DFT order."""
    alpha = np.fft.fftfreq(N_FFT, d=1.0 / N_FFT)
    eta = 2.0 * math.pi * alpha / (N_FFT * delta)
    u = np.exp(-1j * eta * math.log(kr0)) * mellin_jl(ell, q + 1j * eta)
    u[N_FFT // 2] = u[N_FFT // 2].real   # Nyquist term (alpha = -N/2) kept real
    return u


def fftlog(a: np.ndarray, x_in: np.ndarray, x_out: np.ndarray, ell: int, q: float, delta: float) -> np.ndarray:
    """T[a](y_m) = int_0^inf (dx/x) a(x) j_l(x y_m) on log grids x_n = x_0 e^{n Delta}, y_m = y_0 e^{m Delta}."""
    c = np.fft.fft(a * x_in ** (-q)) / N_FFT
    u = fftlog_kernel(ell, q, delta, x_in[0] * x_out[0])
    return np.real(np.fft.fft(c * u)) * x_out ** (-q)


def hankel_inverse(pk: np.ndarray, ell: int):
    """xi(r) = H^-1_l[P](r) = i^l int k^2 dk/(2 pi^2) j_l(kr) P(k) on the r grid (P tapered at the ends)."""
    k, r, delta = log_grid()
    tp = np.zeros(N_FFT)
    tp[:N_IN] = taper()
    return (1j ** ell).real / (2.0 * math.pi ** 2) * fftlog(k ** 3 * pk * tp, k, r, ell, Q_INV, delta)


def hankel_forward(g: np.ndarray, ell: int):
    """P(k) = H_l[g](k) = 4 pi (-i)^l int r^2 dr j_l(kr) g(r) on the k grid."""
    k, r, delta = log_grid()
    return 4.0 * math.pi * ((-1j) ** ell).real * fftlog(r ** 3 * g, r, k, ell, Q_FWD, delta)


# ------------------------------------------------------------------ model
def top_hat(x):
    x = np.asarray(x, dtype=np.float64)
    small = x < 1e-2
    xs = np.where(small, 1.0, x)
    big = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(small, 1.0 - x * x / 10.0 + x ** 4 / 280.0, big)


def bbks_shape(k, gamma, tilt):
    q = k / gamma
    t = np.log(1.0 + 2.34 * q) / (2.34 * q) * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3
                                               + (6.71 * q) ** 4) ** -0.25
    return k ** (1.0 + tilt) * t * t


TAPER = 0.1


def taper(n_in: int = N_IN):
    """Smooth edges of the input range: t - sin(2 pi t)/(2 pi) over the first and last TAPER of it."""
    x = np.arange(n_in) / (n_in - 1)
    out = np.ones(n_in)
    for t in (x / TAPER, (1.0 - x) / TAPER):
        tt = np.clip(t, 0.0, 1.0)
        out *= np.where(t >= 1.0, 1.0, tt - np.sin(2.0 * math.pi * tt) / (2.0 * math.pi))
    return out


def linear_pk(params):
    """BBKS P(k) on the k grid (zero beyond the N_IN input points), sigma_8-normalised (untapered)."""
    a_ia, b_g, s8, tilt, gam, shot = params
    k, r, delta = log_grid()
    kin = k[:N_IN]
    shape = bbks_shape(kin, gam, tilt)
    integrand = kin ** 3 * shape / (2.0 * math.pi ** 2) * top_hat(8.0 * kin) ** 2
    w = np.full(N_IN, delta)
    w[0] = w[-1] = 0.5 * delta
    s2 = float(np.sum(w * integrand))
    pk = np.zeros(N_FFT)
    pk[:N_IN] = shape * (s8 * s8 / s2)
    return pk


C_OVER_H0 = 2997.92458   # Mpc/h: the speed of light over 100 km/s/Mpc


def bbks_transfer(k, gamma):
    """BBKS transfer function T(k / Gamma) (Bardeen et al. 1986), the shape's T in bbks_shape."""
    q = k / gamma
    return np.log(1.0 + 2.34 * q) / (2.34 * q) * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3
                                                  + (6.71 * q) ** 4) ** -0.25


def png_factor(k, gamma, f_nl, db_ia, omega_m):
    """Response of a galaxy-shape field to spin-2 local primordial non-Gaussianity (Sec. 5):
    P -> [1 + 12 f_NL delta b_IA / M(k)] P with M(k) = (2/3) k^2 T(k) D (c/H0)^2 / Omega_m, D = 1.
    Reading: the factor multiplies each shape field, so P_gd carries it once and P_+- twice."""
    mk = (2.0 / 3.0) * k * k * bbks_transfer(k, gamma) * C_OVER_H0 ** 2 / omega_m
    return 1.0 + 12.0 * f_nl * db_ia / mk


def model_multipoles(params):
    """Native multipoles P^(L')_X of the tidal-alignment model (Eq. power_for_validation with e = -A T,
    galaxies b_g delta): dd {0: b^2}, cross {2: -A b / 6}, plus {0: 2A^2/15, 2: -4A^2/21, 4: 2A^2/35},
    minus {4: A^2/420}, each times the linear P(k)."""
    a_ia, b_g = params[0], params[1]
    return {"dd": {0: b_g * b_g}, "cross": {2: -a_ia * b_g / 6.0},
            "plus": {0: 2.0 * a_ia ** 2 / 15.0, 2: -4.0 * a_ia ** 2 / 21.0, 4: 2.0 * a_ia ** 2 / 35.0},
            "minus": {4: a_ia ** 2 / 420.0}}


def q_on_r(q_table, s, r):
    """Q_l(r) for l = 0..8 even from a table at separations s: linear, held below s_0, zero beyond s_last."""
    out = np.zeros((5, r.size))
    for li in range(5):
        v = np.interp(r, s, q_table[li], left=q_table[li][0], right=0.0)
        v = np.where(r > s[-1], 0.0, v)
        out[li] = v
    return out


def bin_average(pk_grid, k_edges):
    """sum k^3 P / sum k^3 over the grid points of each shell [e_b, e_b+1)."""
    k, r, delta = log_grid()
    kin = k[:N_IN]
    out = np.zeros(len(k_edges) - 1)
    for b in range(len(k_edges) - 1):
        sel = (kin >= k_edges[b]) & (kin < k_edges[b + 1])
        wk = kin[sel] ** 3
        out[b] = np.sum(wk * pk_grid[:N_IN][sel]) / np.sum(wk) if wk.size else 0.0
    return out


def template(params, q_table, s, k_edges, shot_plus: float = 0.0, mixing=None, png=None):
    """All fourteen window-convolved native multipoles of one parameter set, shell-averaged: (14, nb).
    png = (f_NL, delta b_IA, Omega_m): the shape spectra carry png_factor (cross once, plus and
    minus twice; Sec. 5), the density spectrum not."""
    k, r, delta = log_grid()
    pk = linear_pk(params)
    spec = {"dd": pk, "cross": pk, "plus": pk, "minus": pk}
    if png is not None:
        f = np.ones(N_FFT)
        f[:N_IN] = png_factor(k[:N_IN], params[4], *png)
        spec = {"dd": pk, "cross": pk * f, "plus": pk * f * f, "minus": pk * f * f}
    qr = q_on_r(np.asarray(q_table, dtype=np.float64), np.asarray(s, dtype=np.float64), r)
    model = model_multipoles(params)
    xi = {(kind, lp): hankel_inverse(spec[kind], lp) for kind in model for lp in model[kind]}
    out = np.zeros((len(SLOTS), len(k_edges) - 1))
    for i, (kind, L) in enumerate(SLOTS):
        g = np.zeros(N_FFT)
        for lp, coef in model[kind].items():
            mix = mixing[(kind, L, lp)] if mixing else [float(c) for c in mixing_coefficients(kind, L, lp)]
            qx = sum(mix[j] * qr[j] for j in range(5))
            g += coef * qx * xi[(kind, lp)]
        pt = hankel_forward(g, L)
        if kind == "plus" and L == 0:
            pt = pt + params[5] * shot_plus
        out[i] = bin_average(pt, k_edges)
    return out


def mixing_table():
    """All (X, L, L') mixing coefficient lists the template needs, as floats."""
    tab = {}
    for kind, L in SLOTS:
        for lp in model_multipoles((1.0, 1.0, 0.8, 0.0, 0.2, 1.0))[kind]:
            tab[(kind, L, lp)] = [float(c) for c in mixing_coefficients(kind, L, lp)]
    return tab


def gaussian_sigma(p0, k_edges, volume, noise_g, noise_e):
    """Gaussian error bars of the derived multipoles (gE_0,2, EE_0,2,4, BB_0,2,4).

    The paper states no covariance; the reading used is the disconnected Gaussian one with
    isotropic power: a shell holding N_k = V * (4 pi / 3) (k_hi^3 - k_lo^3) / (2 pi)^3 modes
    (k and -k both counted, so N_k / 2 independent complex amplitudes at fixed mu) and the
    Legendre-weighted estimator of multipole l give var(P_ab^(l)) = (2l+1) (P_aa P_bb + P_ab^2) / N_k,
    which for an auto spectrum is 2 (2l+1) P^2 / N_k.  p0 = [P_gg, P_gE, P_EE, P_BB] monopoles
    without shot noise; noise_g is added to P_gg and noise_e to P_EE and P_BB."""
    p0 = np.asarray(p0, dtype=np.float64).reshape(4, -1)
    e = np.asarray(k_edges, dtype=np.float64)
    nk = volume * (4.0 * math.pi / 3.0) * (e[1:] ** 3 - e[:-1] ** 3) / (2.0 * math.pi) ** 3
    gg, ge, ee, bb = p0[0] + noise_g, p0[1], p0[2] + noise_e, p0[3] + noise_e
    out = np.zeros((8, p0.shape[1]))
    for c, ell in enumerate([0, 2, 0, 2, 4, 0, 2, 4]):
        f = 2 * ell + 1
        if c < 2:
            var = f * (gg * ee + ge * ge) / nk
        elif c < 5:
            var = 2 * f * ee * ee / nk
        else:
            var = 2 * f * bb * bb / nk
        out[c] = np.sqrt(var)
    return out
