"""FP64 CPU oracle for the LPP projected-tensor multipole estimator (Kurita & Takada 2022).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain statement of what the
CUDA path computes.  Only the test-suite, the package's ``smoke()`` check and the
``cpu_baseline``/reference leg of ``bench.py`` may import it; the product path
never does, and it shares no code with the CUDA library.

It follows the paper's own Cartesian form of the estimators:

* cross (Eq. lpp_estimator_cross_Xiij, Eq. def_of_Xiij)
      P^(L)_gd(k) = (2L+1)(L-2)!/(L+2)! < Xi^(L)_ij(k) k_i k_j delta(-k) >_shell
      Xi^(L)_ij(k) = FT[ gamma 2 e*_ij(x) Lm2_L(k.x) / (1-(k.x)^2) ]
* plus (Eq. lpp_estimator_auto_+)
      P^(l)_+(k) = (2l+1) < gamma^(l)(k) gamma*(-k) >_shell,  gamma^(l) = FT[gamma L_l(k.x)]
* minus (Eq. lpp_estimator_auto_-, Eq. def_of_Xiijkl), L = 4, 6, ..., 12
      P^(L)_-(k) = (2L+1)(L-4)!/(L+4)! < Xi^(L)_ijkl(k) k_i k_j k_k k_l gamma(-k) >_shell
      Xi^(L)_ijkl = FT[ gamma 4 e*_ij e*_kl Lm4_L(k.x) / (1-(k.x)^2)^2 ]

with gamma = e_ij(x) s_ij (Eq. gamma_def), e_ij = e+_i e+_j, e+ = (e_theta + i e_phi)/sqrt2
(Eqs. def_of_eij_+2, def_polarization_vector), and the associated Legendre functions
Lm_L(mu) = (-1)^m (1-mu^2)^(m/2) d^m/dmu^m L_L(mu) (Eq. def_of_asso).  Every ratio
Lm_L/(1-mu^2)^(m/2) is a polynomial in mu = k.x, expanded here into products of
Cartesian components of k and x (Sec. 3.1.2: "Cartesian components"), so each
needed field is a plain FFT of gamma * (tensor component) * (monomial of x).

Readings where the paper is silent:
* sky frame: e_phi = unit(p x xhat), e_theta = e_phi x xhat for a plan pole p
  (the spherical frame about p; the paper's S(d) matrix is the case p = z);
* galaxies enter as weighted Dirac deltas, gridded by CIC/TSC (optionally with
  half-cell interlacing) and deconvolved by the assignment window;
* delta(-k) := conj(D(k)) for the real density field, gamma*(-k) := conj(FT[gamma]),
  gamma(-k) := conj(FT[gamma*]);  the shell average is the mean over all modes of the
  n^3 DFT grid (numpy fftfreq frequencies) with kf*sqrt(n^2) in [edge_b, edge_b+1), k != 0;
* normalisation I: periodic box (Sum w)^2/V (auto) and (Sum w_s)(Sum w_d)/V (cross),
  with randoms alpha * Sum_r nbar w^2; shot noise Sum_s w^2|gamma|^2 / I on P_+^(0) only;
  a shell that contains no mode of the grid reports 0 (no estimate, no shot-noise term).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from itertools import combinations_with_replacement

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

# moments this oracle evaluates, in a fixed order: the density monopole, the ten of the paper's
# headline set (cross L <= 6, plus l <= 4, minus L <= 8), then the minus moments L = 10, 12 that
# continue the expansion of P_-(k, mu) in Lm4_L (Sec. 2.4); a Plan evaluates DEFAULT_MOMENTS
# unless told otherwise
MOMENTS = [("dd", 0), ("cross", 2), ("cross", 4), ("cross", 6), ("plus", 0), ("plus", 2),
           ("plus", 4), ("minus", 4), ("minus", 6), ("minus", 8), ("minus", 10), ("minus", 12)]
DEFAULT_MOMENTS = MOMENTS[:10]
M_INDEX = {m: i for i, m in enumerate(MOMENTS)}


# ----------------------------------------------------------------- polynomials
def legendre_coeffs(ell: int) -> np.ndarray:
    """Power-series coefficients of the Legendre polynomial L_ell(mu)."""
    c = np.zeros(ell + 1)
    c[ell] = 1.0
    return npleg.leg2poly(c)


def reduced_assoc_legendre(m: int, L: int) -> np.ndarray:
    """Coefficients of Lm_L(mu)/(1-mu^2)^(m/2) = (-1)^m d^m L_L/dmu^m (Eq. def_of_asso), m even."""
    assert m % 2 == 0
    c = legendre_coeffs(L)
    d = nppoly.polyder(c, m) if m else c
    return ((-1) ** m) * d


def norm_factor(m: int, L: int) -> float:
    """(2L+1) (L-m)!/(L+m)!: the prefactor of Eqs. multipole_cross_def and Hankel_trs_-."""
    return (2 * L + 1) * math.factorial(L - m) / math.factorial(L + m)


def legendre_fraction(ell: int):
    """Exact Legendre coefficients from Rodrigues' formula d^l/dmu^l (mu^2-1)^l / (2^l l!)."""
    # (mu^2 - 1)^l expanded
    p = [Fraction(0)] * (2 * ell + 1)
    for j in range(ell + 1):
        p[2 * j] = Fraction(math.comb(ell, j) * (-1) ** (ell - j))
    for _ in range(ell):
        p = [p[i] * i for i in range(1, len(p))]
    s = Fraction(1, 2 ** ell * math.factorial(ell))
    return [c * s for c in p]


def _poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_int_m1_1(a) -> Fraction:
    return sum((c * Fraction(2, i + 1) for i, c in enumerate(a) if i % 2 == 0), Fraction(0))


def assoc_legendre_fraction(m: int, L: int):
    """Exact coefficients of Lm_L(mu) for even m (Eq. def_of_asso)."""
    d = legendre_fraction(L)
    for _ in range(m):
        d = [d[i] * i for i in range(1, len(d))] or [Fraction(0)]
    one_minus = [Fraction(1), Fraction(0), Fraction(-1)]
    f = [Fraction(1)]
    for _ in range(m // 2):
        f = _poly_mul(f, one_minus)
    return [c * (-1) ** m for c in _poly_mul(f, d)]


def legendre_projection_matrix(m: int, ells, Ls):
    """M[l][L] = (2l+1)/2 int_{-1}^{1} Lm_L(mu) L_l(mu) dmu, exact rationals.

    Maps associated-Legendre moments (Eqs. multipole_cross_def, Hankel_trs_-) onto
    ordinary Legendre multipoles of the same function of mu (completeness, Sec. 2.4).
    """
    out = []
    for ell in ells:
        row = []
        pl = legendre_fraction(ell)
        for L in Ls:
            row.append(Fraction(2 * ell + 1, 2) * _poly_int_m1_1(_poly_mul(assoc_legendre_fraction(m, L), pl)))
        out.append(row)
    return out


# ------------------------------------------------------------- sky frame & shear
def line_of_sight(pos: np.ndarray, observer) -> np.ndarray:
    """Unit vectors xhat from the observer to each position, (n, 3)."""
    r = pos.T.astype(np.float64) - np.asarray(observer, dtype=np.float64)[None, :]
    return r / np.linalg.norm(r, axis=1)[:, None]


def sky_frame(xhat: np.ndarray, pole):
    """Spherical frame about the pole p: e_phi = unit(p x xhat), e_theta = e_phi x xhat."""
    p = np.asarray(pole, dtype=np.float64)
    p = p / np.linalg.norm(p)
    ephi = np.cross(np.broadcast_to(p, xhat.shape), xhat)
    ephi = ephi / np.linalg.norm(ephi, axis=1)[:, None]
    etheta = np.cross(ephi, xhat)
    return etheta, ephi


def helicity_tensor(etheta: np.ndarray, ephi: np.ndarray) -> np.ndarray:
    """e_ij = e+_i e+_j with e+ = (e_theta + i e_phi)/sqrt(2); (n, 3, 3) complex."""
    ep = (etheta + 1j * ephi) / math.sqrt(2.0)
    return ep[:, :, None] * ep[:, None, :]


def full_tensor(s6: np.ndarray) -> np.ndarray:
    """(6, n) components (xx, yy, zz, xy, xz, yz) -> (n, 3, 3)."""
    s = np.zeros((s6.shape[1], 3, 3))
    order = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for c, (i, j) in enumerate(order):
        s[:, i, j] = s6[c]
        s[:, j, i] = s6[c]
    return s


def shear(s6: np.ndarray | None, g12: np.ndarray | None, e: np.ndarray) -> np.ndarray:
    """gamma = gamma_1 + i gamma_2 = e_ij s_ij (Eq. gamma_def), or the given (gamma_1, gamma_2)."""
    if s6 is not None:
        return np.einsum("nij,nij->n", e, full_tensor(np.asarray(s6, dtype=np.float64)))
    g = np.asarray(g12, dtype=np.float64)
    return g[0] + 1j * g[1]


# ------------------------------------------------------------------- assignment
def assignment_stencil(pos: np.ndarray, n: int, box: float, origin, scheme: int, shift: float):
    """Flat cell indices (np, p^3) and weights for CIC (p=2) or TSC (p=3), periodic.

    Grid nodes sit at origin + (i + shift) H, H = box/n.  CIC: w(s) = 1 - |s|;
    TSC: w(s) = 3/4 - s^2 (|s| <= 1/2), (3/2 - |s|)^2 / 2 (1/2 <= |s| < 3/2).
    """
    h = box / n
    idx1d, w1d = [], []
    for a in range(3):
        u = (pos[a].astype(np.float64) - origin[a]) / h - shift
        if scheme == 2:
            i0 = np.floor(u)
            f = u - i0
            cells = np.stack([i0, i0 + 1], axis=1)
            wts = np.stack([1.0 - f, f], axis=1)
        elif scheme == 3:
            ic = np.floor(u + 0.5)
            d = u - ic
            cells = np.stack([ic - 1, ic, ic + 1], axis=1)
            wts = np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2], axis=1)
        else:
            raise ValueError("scheme must be 2 (CIC) or 3 (TSC)")
        idx1d.append(np.mod(cells.astype(np.int64), n))
        w1d.append(wts)
    p = scheme
    flat = (idx1d[0][:, :, None, None] * n + idx1d[1][:, None, :, None]) * n + idx1d[2][:, None, None, :]
    wt = w1d[0][:, :, None, None] * w1d[1][:, None, :, None] * w1d[2][:, None, None, :]
    return flat.reshape(-1, p ** 3), wt.reshape(-1, p ** 3)


def grid_from_stencil(stencil, values: np.ndarray, n: int) -> np.ndarray:
    """Sum values (np,) complex or real onto the n^3 grid through the stencil."""
    flat, wt = stencil
    contrib = values[:, None] * wt
    if np.iscomplexobj(contrib):
        g = (np.bincount(flat.ravel(), weights=contrib.real.ravel(), minlength=n ** 3)
             + 1j * np.bincount(flat.ravel(), weights=contrib.imag.ravel(), minlength=n ** 3))
    else:
        g = np.bincount(flat.ravel(), weights=contrib.ravel(), minlength=n ** 3)
    return g.reshape(n, n, n)


@dataclass
class ModeGrid:
    """Integer frequencies (numpy fftfreq ordering) of the n^3 DFT grid."""
    n: int
    box: float

    def __post_init__(self):
        f = np.fft.fftfreq(self.n, d=1.0 / self.n)
        self.nx, self.ny, self.nz = np.meshgrid(f, f, f, indexing="ij")
        self.n2 = self.nx ** 2 + self.ny ** 2 + self.nz ** 2
        kf = 2.0 * math.pi / self.box
        self.kmag = kf * np.sqrt(self.n2)
        nrm = np.sqrt(self.n2)
        nrm[0, 0, 0] = 1.0
        self.khat = (self.nx / nrm, self.ny / nrm, self.nz / nrm)


def window_compensation(mg: ModeGrid, scheme: int) -> np.ndarray:
    """W(k) = prod_a sinc(pi n_a / n)^p of the CIC/TSC assignment kernel."""
    w = np.ones_like(mg.nx)
    for na in (mg.nx, mg.ny, mg.nz):
        w = w * np.sinc(na / mg.n) ** scheme
    return w


class FieldTransformer:
    """Grid assignment + DFT + window deconvolution + interlacing of per-particle values."""

    def __init__(self, pos, n, box, origin, scheme, interlace, compensate, mg: ModeGrid):
        self.n = n
        self.st0 = assignment_stencil(pos, n, box, origin, scheme, 0.0)
        self.st1 = assignment_stencil(pos, n, box, origin, scheme, 0.5) if interlace else None
        self.inv_w = 1.0 / window_compensation(mg, scheme) if compensate else None
        # half-cell shift phase e^{-i (kx+ky+kz) H/2}
        self.phase = np.exp(-1j * math.pi * (mg.nx + mg.ny + mg.nz) / n) if interlace else None

    def ft(self, values: np.ndarray) -> np.ndarray:
        f = np.fft.fftn(grid_from_stencil(self.st0, values, self.n))
        if self.st1 is not None:
            f2 = np.fft.fftn(grid_from_stencil(self.st1, values, self.n))
            f = 0.5 * (f + self.phase * f2)
        if self.inv_w is not None:
            f = f * self.inv_w
        return f


# ------------------------------------------------------------- Cartesian expansion
def monomials(degree: int):
    """Exponent triples (a, b, c), a+b+c = degree, with multinomial counts."""
    out = []
    for combo in combinations_with_replacement(range(3), degree):
        e = (combo.count(0), combo.count(1), combo.count(2))
        out.append(e)
    uniq = sorted(set(out))
    return [(e, math.factorial(degree) // (math.factorial(e[0]) * math.factorial(e[1]) * math.factorial(e[2])))
            for e in uniq]


def _pow3(v, e):
    return v[0] ** e[0] * v[1] ** e[1] * v[2] ** e[2]


def sym_index_sets(rank: int):
    """Distinct sorted index tuples of a symmetric rank-`rank` tensor in 3D with multiplicity."""
    out = []
    for t in combinations_with_replacement(range(3), rank):
        cnt = [t.count(i) for i in range(3)]
        mult = math.factorial(rank)
        for c in cnt:
            mult //= math.factorial(c)
        out.append((t, mult))
    return out


def xi_contracted(ft: FieldTransformer, mg: ModeGrid, base: np.ndarray, tensor: np.ndarray,
                  rank: int, radial_poly: np.ndarray, xhat: np.ndarray) -> np.ndarray:
    """sum_{i..} khat_i.. Xi_{i..}(k) with Xi_{i..} = FT[base * tensor_{i..} * P(k.x)].

    P(mu) = sum_p c_p mu^p is expanded as sum_p c_p sum_|a|=p multinom(a) khat^a xhat^a,
    i.e. one FFT per (symmetric tensor component, x-monomial) pair, as in Eq. def_of_Xiij.
    """
    out = np.zeros((mg.n,) * 3, dtype=np.complex128)
    kh = mg.khat
    for idx, mult in sym_index_sets(rank):
        comp = tensor[(slice(None),) + idx]
        kcomp = np.ones_like(mg.nx)
        for i in idx:
            kcomp = kcomp * kh[i]
        for p, cp in enumerate(radial_poly):
            if cp == 0.0:
                continue
            for e, mn in monomials(p):
                vals = base * comp * _pow3(xhat.T, e)
                out += (mult * cp * mn) * kcomp * _pow3(kh, e) * ft.ft(vals)
    return out


def moment_field(kind: str, L: int, ft: FieldTransformer, mg: ModeGrid, w: np.ndarray,
                 gamma: np.ndarray, e: np.ndarray, xhat: np.ndarray, with_b: bool = True) -> np.ndarray:
    """The k-space field contracted with the partner for one moment.

    cross: Xi^(L)_ij khat_i khat_j (Eq. def_of_Xiij); its real part is the E part
           (Re[gamma 2e*_ij] = gamma_ij) and its imaginary part the B part.  With
           ``with_b`` False only the E part is formed (from the real tensor gamma_ij).
    plus : gamma^(l)(k) (Eq. lpp_estimator_auto_+).
    minus: Xi^(L)_ijkl khat_i khat_j khat_k khat_l (Eq. def_of_Xiijkl).
    """
    if kind == "cross":
        t2 = 2.0 * np.conj(e)
        q = reduced_assoc_legendre(2, L)
        if with_b:
            return xi_contracted(ft, mg, w * gamma, t2, 2, q, xhat)
        gij = (gamma[:, None, None] * t2).real
        return xi_contracted(ft, mg, w, gij, 2, q, xhat)
    if kind == "plus":
        return xi_contracted(ft, mg, w * gamma, np.ones(w.shape[0]), 0, legendre_coeffs(L), xhat)
    if kind == "minus":
        t4 = 4.0 * np.conj(e)[:, :, :, None, None] * np.conj(e)[:, None, None, :, :]
        return xi_contracted(ft, mg, w * gamma, t4, 4, reduced_assoc_legendre(4, L), xhat)
    raise ValueError(kind)


# -------------------------------------------------------------------- estimator
@dataclass
class Plan:
    n: int
    box: float
    origin: tuple = (0.0, 0.0, 0.0)
    observer: tuple = (0.0, 0.0, 0.0)
    pole: tuple = (-1.0, 0.0, 0.0)
    scheme: int = 2
    interlace: bool = False
    compensate: bool = True
    los_proj_global: bool = False   # True: project shapes with the global n (case (c))
    los_est_global: bool = False    # True: estimator uses the global n (cases (b), (c))
    los_global: tuple = (0.0, 0.0, 1.0)
    moments: tuple = tuple(DEFAULT_MOMENTS)
    cross_b: bool = False
    k_edges: np.ndarray = field(default_factory=lambda: np.zeros(0))
    norm_override: float = 0.0
    subtract_shot: bool = True


@dataclass
class Result:
    p: np.ndarray          # (10, nb) complex, normalised
    raw: np.ndarray        # (10, nb) complex, shell means before normalisation and shot noise
    n_modes: np.ndarray
    k_mean: np.ndarray
    norm_auto: float
    norm_cross: float
    norm_dd: float
    shot_plus: float
    shot_dd: float
    alpha: float


def _bins(mg: ModeGrid, edges: np.ndarray):
    b = np.searchsorted(edges, mg.kmag, side="right") - 1
    nb = len(edges) - 1
    valid = (b >= 0) & (b < nb) & (mg.n2 > 0)
    return np.where(valid, b, nb), nb


def _shell_sum(vals: np.ndarray, b: np.ndarray, nb: int) -> np.ndarray:
    re = np.bincount(b.ravel(), weights=vals.real.ravel(), minlength=nb + 1)[:nb]
    im = np.bincount(b.ravel(), weights=vals.imag.ravel(), minlength=nb + 1)[:nb]
    return re + 1j * im


def multipoles(plan: Plan, shapes_pos, shapes_w=None, shapes_s6=None, shapes_g12=None,
               dens_pos=None, dens_w=None, rand_pos=None, rand_w=None, rand_nbar=None) -> Result:
    """All native multipoles of the LPP estimator on one catalogue set (FP64)."""
    n, box = plan.n, plan.box
    vol = box ** 3
    mg = ModeGrid(n, box)
    edges = np.asarray(plan.k_edges, dtype=np.float64)
    b, nb = _bins(mg, edges)
    n_modes = np.bincount(b.ravel(), minlength=nb + 1)[:nb].astype(np.int64)
    ksum = np.bincount(b.ravel(), weights=mg.kmag.ravel(), minlength=nb + 1)[:nb]
    k_mean = np.where(n_modes > 0, ksum / np.maximum(n_modes, 1), 0.0)

    sp = np.asarray(shapes_pos, dtype=np.float64)
    ns = sp.shape[1]
    ws = np.ones(ns) if shapes_w is None else np.asarray(shapes_w, dtype=np.float64)
    # line of sight used for the projection (Eq. 2Dshear_from_3Dshape) and for the estimator
    x_loc = line_of_sight(sp, plan.observer)
    nglob = np.asarray(plan.los_global, dtype=np.float64)
    nglob = nglob / np.linalg.norm(nglob)
    x_proj = np.broadcast_to(nglob, x_loc.shape).copy() if plan.los_proj_global else x_loc
    x_est = np.broadcast_to(nglob, x_loc.shape).copy() if plan.los_est_global else x_loc
    eth_p, eph_p = sky_frame(x_proj, plan.pole)
    gamma = shear(shapes_s6, shapes_g12, helicity_tensor(eth_p, eph_p))
    eth, eph = sky_frame(x_est, plan.pole)
    e_est = helicity_tensor(eth, eph)

    ft_s = FieldTransformer(sp, n, box, plan.origin, plan.scheme, plan.interlace, plan.compensate, mg)

    # density tracer and randoms
    if dens_pos is None:
        dp, wd, ft_d = sp, ws, ft_s
    else:
        dp = np.asarray(dens_pos, dtype=np.float64)
        wd = np.ones(dp.shape[1]) if dens_w is None else np.asarray(dens_w, dtype=np.float64)
        ft_d = FieldTransformer(dp, n, box, plan.origin, plan.scheme, plan.interlace, plan.compensate, mg)
    dens_ft = ft_d.ft(wd.astype(np.complex128))
    if rand_pos is not None:
        rp = np.asarray(rand_pos, dtype=np.float64)
        wr = np.ones(rp.shape[1]) if rand_w is None else np.asarray(rand_w, dtype=np.float64)
        nbr = np.ones(rp.shape[1]) if rand_nbar is None else np.asarray(rand_nbar, dtype=np.float64)
        alpha = wd.sum() / wr.sum()
        ft_r = FieldTransformer(rp, n, box, plan.origin, plan.scheme, plan.interlace, plan.compensate, mg)
        dens_ft = dens_ft - alpha * ft_r.ft(wr.astype(np.complex128))
        norm = alpha * np.sum(nbr * wr * wr)
        norm_auto = norm_cross = norm_dd = norm
        shot_dd_num = np.sum(wd * wd) + alpha * alpha * np.sum(wr * wr)
    else:
        alpha = 0.0
        norm_auto = ws.sum() ** 2 / vol
        norm_cross = ws.sum() * wd.sum() / vol
        norm_dd = wd.sum() ** 2 / vol
        shot_dd_num = np.sum(wd * wd)
    if plan.norm_override > 0:
        norm_auto = norm_cross = norm_dd = plan.norm_override
    shot_plus = np.sum(ws * ws * np.abs(gamma) ** 2) / norm_auto if plan.subtract_shot else 0.0
    shot_dd = shot_dd_num / norm_dd if plan.subtract_shot else 0.0

    wg = ws * gamma                              # weighted complex shear
    g_ft = ft_s.ft(wg)                           # gamma(k)
    gc_ft = ft_s.ft(np.conj(wg))                 # FT[gamma*]
    partner = {
        "cross": np.conj(dens_ft),               # delta(-k), delta real
        "plus": np.conj(g_ft),                   # gamma*(-k) = conj(FT[gamma])
        "minus": np.conj(gc_ft),                 # gamma(-k)  = conj(FT[gamma*])
    }
    raw = np.zeros((len(MOMENTS), nb), dtype=np.complex128)
    nm = np.maximum(n_modes, 1)
    for (kind, L) in plan.moments:
        i = M_INDEX[(kind, L)]
        if kind == "dd":
            raw[i] = _shell_sum(dens_ft * np.conj(dens_ft), b, nb) / nm
            continue
        f = moment_field(kind, L, ft_s, mg, ws, gamma, e_est, x_est, plan.cross_b)
        fac = norm_factor({"cross": 2, "plus": 0, "minus": 4}[kind], L)
        raw[i] = fac * _shell_sum(f * partner[kind], b, nb) / nm
    p = np.zeros_like(raw)
    for (kind, L) in plan.moments:
        i = M_INDEX[(kind, L)]
        nrm = {"dd": norm_dd, "cross": norm_cross}.get(kind, norm_auto)
        p[i] = raw[i] / nrm
        if kind == "plus" and L == 0:
            p[i] = p[i] - shot_plus
        if kind == "dd":
            p[i] = p[i] - shot_dd
        p[i] = np.where(n_modes > 0, p[i], 0.0)   # a shell without modes has no estimate: report 0
    return Result(p, raw, n_modes, k_mean, norm_auto, norm_cross, norm_dd, shot_plus, shot_dd, alpha)


# ---------------------------------------------------------------- derived E/B
def derived_eb(p: np.ndarray):
    """Legendre multipoles of P_gE (l=0,2) and P_EE/P_BB (l=0,2,4) from the native moments.

    P_gE(mu) = Re sum_L P^(L)_gd Lm2_L(mu), P_-(mu) = sum_L P^(L)_- Lm4_L(mu) (Sec. 2.4
    completeness), P_EE/BB = (P_+ +- P_-)/2 (Eq. relation_pm_EB), projected on L_l.
    """
    n_mat = legendre_projection_matrix(2, (0, 2), (2, 4, 6))
    m_mat = legendre_projection_matrix(4, (0, 2, 4), (4, 6, 8))
    cross = np.stack([p[M_INDEX[("cross", L)]].real for L in (2, 4, 6)])
    minus = np.stack([p[M_INDEX[("minus", L)]].real for L in (4, 6, 8)])
    plus = np.stack([p[M_INDEX[("plus", l)]].real for l in (0, 2, 4)])
    ge = np.array([[float(c) for c in row] for row in n_mat]) @ cross
    mm = np.array([[float(c) for c in row] for row in m_mat]) @ minus
    return ge, 0.5 * (plus + mm), 0.5 * (plus - mm)


# ------------------------------------------------------------ density multipoles
@dataclass
class DensityResult:
    ells: tuple
    p: np.ndarray          # (len(ells), nb) complex, normalised (shot noise on l = 0 only)
    raw: np.ndarray        # (len(ells), nb) complex, shell means before normalisation
    n_modes: np.ndarray
    k_mean: np.ndarray
    norm: float
    shot: float


def density_ell_field(plan: Plan, mg: ModeGrid, pos, w, ell: int) -> np.ndarray:
    """delta^(l)(k) = FT[w L_l(khat . xhat)] of one catalogue (Eq. delta_ell, endpoint line of
    sight xhat toward each galaxy, or the plan's global n for the GPP form Eq. gpp_dens),
    with L_l(khat . xhat) expanded into Cartesian products of khat and xhat as for the
    tensor moments (one FFT per monomial of xhat)."""
    pos = np.asarray(pos, dtype=np.float64)
    xl = line_of_sight(pos, plan.observer)
    if plan.los_est_global:
        ng = np.asarray(plan.los_global, dtype=np.float64)
        xl = np.broadcast_to(ng / np.linalg.norm(ng), xl.shape).copy()
    ft = FieldTransformer(pos, plan.n, plan.box, plan.origin, plan.scheme, plan.interlace, plan.compensate, mg)
    return xi_contracted(ft, mg, np.asarray(w, dtype=np.float64), np.ones(pos.shape[1]), 0, legendre_coeffs(ell), xl)


def density_multipoles(plan: Plan, dens_pos, dens_w=None, rand_pos=None, rand_w=None, rand_nbar=None,
                       ells=(0, 2, 4)) -> DensityResult:
    """Yamamoto (LPP) multipoles of the galaxy density (Eq. lpp_dens_app):
        P^(l)(k) = (2l+1) < delta^(l)(k) delta(-k) >_shell / I  -  [l = 0] N,
    delta = data - alpha randoms, each catalogue's delta^(l) from its own lines of sight;
    I and the shot noise N as for the density monopole slot of `multipoles`."""
    n, box = plan.n, plan.box
    mg = ModeGrid(n, box)
    edges = np.asarray(plan.k_edges, dtype=np.float64)
    b, nb = _bins(mg, edges)
    n_modes = np.bincount(b.ravel(), minlength=nb + 1)[:nb].astype(np.int64)
    ksum = np.bincount(b.ravel(), weights=mg.kmag.ravel(), minlength=nb + 1)[:nb]
    k_mean = np.where(n_modes > 0, ksum / np.maximum(n_modes, 1), 0.0)
    dp = np.asarray(dens_pos, dtype=np.float64)
    wd = np.ones(dp.shape[1]) if dens_w is None else np.asarray(dens_w, dtype=np.float64)
    if rand_pos is not None:
        rp = np.asarray(rand_pos, dtype=np.float64)
        wr = np.ones(rp.shape[1]) if rand_w is None else np.asarray(rand_w, dtype=np.float64)
        nbr = np.ones(rp.shape[1]) if rand_nbar is None else np.asarray(rand_nbar, dtype=np.float64)
        alpha = wd.sum() / wr.sum()
        norm = alpha * np.sum(nbr * wr * wr)
        shot_num = np.sum(wd * wd) + alpha * alpha * np.sum(wr * wr)
    else:
        alpha, norm, shot_num = 0.0, wd.sum() ** 2 / box ** 3, np.sum(wd * wd)
    if plan.norm_override > 0:
        norm = plan.norm_override
    shot = shot_num / norm if plan.subtract_shot else 0.0

    def field_of(ell):
        f = density_ell_field(plan, mg, dp, wd, ell)
        if rand_pos is not None:
            f = f - alpha * density_ell_field(plan, mg, rp, wr, ell)
        return f

    delta = field_of(0)
    nm = np.maximum(n_modes, 1)
    raw = np.zeros((len(ells), nb), dtype=np.complex128)
    p = np.zeros_like(raw)
    for i, ell in enumerate(ells):
        f = delta if ell == 0 else field_of(ell)
        raw[i] = (2 * ell + 1) * _shell_sum(f * np.conj(delta), b, nb) / nm
        p[i] = raw[i] / norm - (shot if ell == 0 else 0.0)
        p[i] = np.where(n_modes > 0, p[i], 0.0)
    return DensityResult(tuple(ells), p, raw, n_modes, k_mean, norm, shot)


# --------------------------------------------------------------- direct sums (pins)
def direct_kernel(kind: str, L: int, khat: np.ndarray, xhat, etheta, ephi, gamma):
    """K_X(khat; x, gamma) evaluated directly (no Cartesian expansion), shape (nk, np).

    cross: gamma (2 e*_ij khat_i khat_j) Lm2_L(mu)/(1-mu^2), 2e*_ij k_i k_j = (k.e_theta - i k.e_phi)^2
    plus : gamma L_l(mu);  minus: gamma (2 e*_ij k_i k_j)^2 Lm4_L(mu)/(1-mu^2)^2.
    The Legendre functions come from scipy.special.lpmv (Condon-Shortley phase included).
    """
    from scipy.special import lpmv
    mu = khat @ xhat.T
    a = khat @ etheta.T
    bb = khat @ ephi.T
    ph = (a - 1j * bb) ** 2
    if kind == "plus":
        return gamma[None, :] * lpmv(0, L, mu)
    m = 2 if kind == "cross" else 4
    red = lpmv(m, L, mu) / (1.0 - mu * mu) ** (m // 2)
    return gamma[None, :] * (ph if m == 2 else ph * ph) * red


def direct_ft(kvec: np.ndarray, pos: np.ndarray, values: np.ndarray) -> np.ndarray:
    """sum_g values[k, g] e^{-i k.x_g} for wave vectors kvec (nk, 3)."""
    phase = np.exp(-1j * (kvec @ pos))
    return np.sum(values * phase, axis=1)


# ------------------------------------------------------------------ window multipoles
@dataclass
class WindowResult:
    q: np.ndarray          # (5, nb) for l = 0, 2, 4, 6, 8
    n_points: np.ndarray   # separation grid points per shell
    s_mean: np.ndarray
    norm: float


def _separations(n: int, box: float):
    """Minimal-image separation of every grid offset (same index order as the DFT grid)."""
    h = box / n
    f = np.fft.fftfreq(n, d=1.0 / n)
    sx, sy, sz = np.meshgrid(f, f, f, indexing="ij")
    return sx, sy, sz, h


def window_multipoles(n: int, box: float, origin, observer, rand_pos, rand_w, rand_nbar, alpha: float,
                      s_edges, scheme: int = 2, compensate: bool = True, ells=(0, 2, 4, 6, 8)) -> WindowResult:
    """Q_l(s) = (2l+1) < int_x W(x) W(x+s) L_l(s.x) >_shell / I (Eq. windowQ_ell, endpoint d = x).

    W(x) = alpha sum_r w_r delta_D(x - x_r) from the randoms; I = alpha sum_r nbar w^2 (the
    estimator's normalisation, so that Q_0 -> 1 at small s for a window much larger than s).
    L_l(s.x) is expanded into Cartesian monomials of s and x; every monomial field is
    cross-correlated with W by FFT (sum_x A(x) B(x+s) = IFFT[conj FT A . FT B](s)); the shell
    average runs over the grid separations s (minimal image) with h sqrt(q) in [edge_b,
    edge_b+1), s = 0 excluded.
    """
    rp = np.asarray(rand_pos, dtype=np.float64)
    nr = rp.shape[1]
    w = np.ones(nr) if rand_w is None else np.asarray(rand_w, dtype=np.float64)
    nb_ = np.ones(nr) if rand_nbar is None else np.asarray(rand_nbar, dtype=np.float64)
    norm = alpha * np.sum(nb_ * w * w)
    mg = ModeGrid(n, box)
    ft = FieldTransformer(rp, n, box, origin, scheme, False, compensate, mg)
    bft = ft.ft(w.astype(np.complex128))
    xh = line_of_sight(rp, observer)
    sx, sy, sz, h = _separations(n, box)
    q2 = sx * sx + sy * sy + sz * sz
    smag = h * np.sqrt(q2)
    edges = np.asarray(s_edges, dtype=np.float64)
    b = np.searchsorted(edges, smag, side="right") - 1
    nbins = len(edges) - 1
    valid = (b >= 0) & (b < nbins) & (q2 > 0)
    b = np.where(valid, b, nbins)
    npts = np.bincount(b.ravel(), minlength=nbins + 1)[:nbins]
    smean = np.bincount(b.ravel(), weights=smag.ravel(), minlength=nbins + 1)[:nbins] / np.maximum(npts, 1)
    rn = np.sqrt(np.maximum(q2, 1e-300))
    shat = (sx / rn, sy / rn, sz / rn)
    out = np.zeros((len(ells), nbins))
    for li, ell in enumerate(ells):
        c = legendre_coeffs(ell)
        acc = np.zeros((n, n, n))
        for p, cp in enumerate(c):
            if cp == 0.0:
                continue
            for e, mn in monomials(p):
                aft = ft.ft((w * _pow3(xh.T, e)).astype(np.complex128))
                corr = np.real(np.fft.ifftn(np.conj(aft) * bft))
                acc += (cp * mn) * _pow3(shat, e) * corr
        vals = (2 * ell + 1) * alpha * alpha * acc / (h ** 3 * norm)
        out[li] = np.bincount(b.ravel(), weights=vals.ravel(), minlength=nbins + 1)[:nbins] / np.maximum(npts, 1)
    out = np.where(npts[None, :] > 0, out, 0.0)
    return WindowResult(out, npts.astype(np.int64), np.where(npts > 0, smean, 0.0), norm)


def window_pair_count(n: int, box: float, observer, rand_pos, rand_w, rand_nbar, alpha: float, s_edges,
                      ells=(0, 2, 4, 6, 8)) -> np.ndarray:
    """Brute-force endpoint pair sums for particles on grid nodes (pin of window_multipoles):
    Q_l(b) = (2l+1) alpha^2 / (N_b h^3 I) sum_{r,r'} w w' L_l(s_rr'.x_r) [s_rr' in b], with the
    minimal-image separation s_rr' = x_r' - x_r and N_b the grid separations in shell b."""
    from scipy.special import eval_legendre
    rp = np.asarray(rand_pos, dtype=np.float64)
    nr = rp.shape[1]
    w = np.ones(nr) if rand_w is None else np.asarray(rand_w, dtype=np.float64)
    nb_ = np.ones(nr) if rand_nbar is None else np.asarray(rand_nbar, dtype=np.float64)
    norm = alpha * np.sum(nb_ * w * w)
    d = rp.T[None, :, :] - rp.T[:, None, :]          # [r, r', 3] = x_r' - x_r
    d = d - box * np.round(d / box)
    s = np.linalg.norm(d, axis=2)
    xh = line_of_sight(rp, observer)
    sx, sy, sz, h = _separations(n, box)
    q2 = sx * sx + sy * sy + sz * sz
    edges = np.asarray(s_edges, dtype=np.float64)
    bg = np.searchsorted(edges, h * np.sqrt(q2), side="right") - 1
    nbins = len(edges) - 1
    npts = np.array([np.sum((bg == i) & (q2 > 0)) for i in range(nbins)])
    # separations of node pairs are exact multiples of h: bin them through the same expression
    qpair = np.round(np.sum((d / h) ** 2, axis=2))
    bp = np.searchsorted(edges, h * np.sqrt(qpair), side="right") - 1
    ok = (qpair > 0) & (bp >= 0) & (bp < nbins)
    mu = np.einsum("rsa,ra->rs", d, xh) / np.where(s > 0, s, 1.0)
    ww = w[:, None] * w[None, :]
    out = np.zeros((len(ells), nbins))
    for li, ell in enumerate(ells):
        val = (2 * ell + 1) * ww * eval_legendre(ell, mu)
        out[li] = np.bincount(bp[ok], weights=val[ok], minlength=nbins)[:nbins]
    out = out * alpha * alpha / (np.maximum(npts, 1)[None, :] * h ** 3 * norm)
    return np.where(npts[None, :] > 0, out, 0.0)


def window_pair_count_shells(rand_pos, rand_w, rand_nbar, alpha: float, observer, s_edges, box: float = 0.0,
                             ells=(0, 2, 4, 6, 8)) -> np.ndarray:
    """Window multipoles by pair counting (the paper's method for Q_l, Sec. 4.3, after
    Eq. windowQ_ell with W = alpha sum_r w_r delta_D(x - x_r) and the endpoint line of sight):

        Q_l(b) = (2l+1) alpha^2 / (I V_b) sum_{r != r', s_rr' in b} w_r w_r' L_l(shat_rr' . xhat_r),

    s_rr' = x_r' - x_r (minimal image when box > 0), V_b = 4 pi (e_{b+1}^3 - e_b^3) / 3 the
    volume of shell b = [e_b, e_{b+1}), I = alpha sum_r nbar w^2 (the estimator's normalisation)
    and xhat_r the unit vector from the observer to x_r.  The direction average over the shell
    (int dOmega / 4 pi at fixed |s|) is the pair sum divided by the shell volume.  Shell of a
    pair: e_b <= sqrt(dx^2 + dy^2 + dz^2) < e_{b+1} in FP64, pairs at s = 0 excluded."""
    from scipy.special import eval_legendre
    rp = np.asarray(rand_pos, dtype=np.float64)
    nr = rp.shape[1]
    w = np.ones(nr) if rand_w is None else np.asarray(rand_w, dtype=np.float64)
    nb_ = np.ones(nr) if rand_nbar is None else np.asarray(rand_nbar, dtype=np.float64)
    norm = alpha * np.sum(nb_ * w * w)
    edges = np.asarray(s_edges, dtype=np.float64)
    nbins = len(edges) - 1
    xh = line_of_sight(rp, observer)
    out = np.zeros((len(ells), nbins))
    for i in range(nr):
        d = rp - rp[:, i:i + 1]                       # [3, r'] = x_r' - x_i
        if box > 0:
            d = d - box * np.round(d / box)
        s = np.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
        b = np.searchsorted(edges, s, side="right") - 1
        ok = (s > 0) & (b >= 0) & (b < nbins)
        mu = (xh[i] @ d[:, ok]) / s[ok]
        ww = w[i] * w[ok]
        for li, ell in enumerate(ells):
            out[li] += np.bincount(b[ok], weights=ww * eval_legendre(ell, mu), minlength=nbins)[:nbins]
    vol = 4.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3) / 3.0
    ell_fac = np.array([2 * ell + 1 for ell in ells], dtype=np.float64)[:, None]
    return ell_fac * alpha * alpha * out / (norm * vol[None, :])
