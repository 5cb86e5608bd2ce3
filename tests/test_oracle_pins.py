"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers the
paper prints, library special functions, closed-form identities, or a direct
(unexpanded) evaluation of the paper's kernels.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy.special import lpmv

from oracle import lpp_oracle as O
from paper_2202_11839_gb300 import synthetic as S

GL_X, GL_W = npleg.leggauss(40)


def _poly(c, x):
    return np.polynomial.polynomial.polyval(x, c)


# ----------------------------------------------------------------- Legendre pins
@pytest.mark.parametrize("m,L", [(2, 2), (2, 4), (2, 6), (4, 4), (4, 6), (4, 8), (4, 10), (4, 12), (0, 2), (0, 4)])
def test_reduced_assoc_legendre_matches_scipy(m, L):
    """(1-mu^2)^(m/2) * reduced poly == scipy lpmv (Condon-Shortley phase included; Eq. def_of_asso)."""
    mu = np.linspace(-0.97, 0.97, 41)
    ours = (1 - mu * mu) ** (m // 2) * _poly(O.reduced_assoc_legendre(m, L), mu)
    np.testing.assert_allclose(ours, lpmv(m, L, mu), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("m", [2, 4])
def test_assoc_legendre_orthogonality(m):
    """int dmu/2 Lm_L Lm_L' = (L+m)!/((2L+1)(L-m)!) delta_LL' (Eq. ortho_asso_legendre)."""
    Ls = [L for L in range(m, 15, 2)]
    for L in Ls:
        for Lp in Ls:
            a = (1 - GL_X ** 2) ** (m // 2) * _poly(O.reduced_assoc_legendre(m, L), GL_X)
            b = (1 - GL_X ** 2) ** (m // 2) * _poly(O.reduced_assoc_legendre(m, Lp), GL_X)
            val = 0.5 * np.sum(GL_W * a * b)
            nrm = lambda j: math.factorial(j + m) / ((2 * j + 1) * math.factorial(j - m))
            want = nrm(L) if L == Lp else 0.0
            assert abs(val - want) <= 1e-12 * math.sqrt(nrm(L) * nrm(Lp))


def test_tidal_model_normalisation_coefficients():
    """Multipoles of P_gd = (1-mu^2)P/2, P_+ = P_- = (1-mu^2)^2 P/4 (Eq. power_for_validation)
    with the paper's prefactors reproduce the printed coefficients of
    Eq. xi_relations_normalization_coefficients: 1/6; 2/15, -4/21, 2/35; 1/420."""
    mu, w = GL_X, GL_W
    cross = lambda L: O.norm_factor(2, L) * 0.5 * np.sum(
        w * 0.5 * (1 - mu ** 2) * (1 - mu ** 2) * _poly(O.reduced_assoc_legendre(2, L), mu))
    plus = lambda l: (2 * l + 1) * 0.5 * np.sum(w * 0.25 * (1 - mu ** 2) ** 2 * _poly(O.legendre_coeffs(l), mu))
    minus = lambda L: O.norm_factor(4, L) * 0.5 * np.sum(
        w * 0.25 * (1 - mu ** 2) ** 2 * (1 - mu ** 2) ** 2 * _poly(O.reduced_assoc_legendre(4, L), mu))
    assert cross(2) == pytest.approx(1 / 6, abs=1e-14)
    assert cross(4) == pytest.approx(0.0, abs=1e-13)
    assert cross(6) == pytest.approx(0.0, abs=1e-12)
    assert plus(0) == pytest.approx(2 / 15, abs=1e-14)
    assert plus(2) == pytest.approx(-4 / 21, abs=1e-14)
    assert plus(4) == pytest.approx(2 / 35, abs=1e-14)
    assert plus(6) == pytest.approx(0.0, abs=1e-13)
    assert minus(4) == pytest.approx(1 / 420, abs=1e-15)
    assert minus(6) == pytest.approx(0.0, abs=1e-13)
    assert minus(8) == pytest.approx(0.0, abs=1e-12)
    assert minus(10) == pytest.approx(0.0, abs=1e-12)
    assert minus(12) == pytest.approx(0.0, abs=1e-12)


def test_exact_legendre_fractions_match_float():
    for m, L in [(2, 2), (2, 6), (4, 8), (0, 4)]:
        fr = O.assoc_legendre_fraction(m, L)
        mu = np.linspace(-1, 1, 9)
        ex = sum(float(c) * mu ** i for i, c in enumerate(fr))
        np.testing.assert_allclose(ex, lpmv(m, L, mu), rtol=1e-12, atol=1e-10)


def test_derived_eb_on_tidal_model():
    """Derived Legendre multipoles reproduce direct quadrature of P_gE = (1-mu^2)/2,
    P_EE = (1-mu^2)^2/4, P_BB = 0 (Eqs. power_for_validation, relation_pm_EB)."""
    p = np.zeros((10, 1), dtype=complex)
    p[O.M_INDEX[("cross", 2)]] = 1 / 6
    p[O.M_INDEX[("plus", 0)]] = 2 / 15
    p[O.M_INDEX[("plus", 2)]] = -4 / 21
    p[O.M_INDEX[("plus", 4)]] = 2 / 35
    p[O.M_INDEX[("minus", 4)]] = 1 / 420
    ge, ee, bb = O.derived_eb(p)
    leg = lambda l: _poly(O.legendre_coeffs(l), GL_X)
    for i, l in enumerate((0, 2)):
        want = (2 * l + 1) * 0.5 * np.sum(GL_W * 0.5 * (1 - GL_X ** 2) * leg(l))
        assert ge[i, 0] == pytest.approx(want, abs=1e-14)
    for i, l in enumerate((0, 2, 4)):
        want = (2 * l + 1) * 0.5 * np.sum(GL_W * 0.25 * (1 - GL_X ** 2) ** 2 * leg(l))
        assert ee[i, 0] == pytest.approx(want, abs=1e-14)
        assert bb[i, 0] == pytest.approx(0.0, abs=1e-14)


def test_projection_matrix_values():
    assert O.legendre_projection_matrix(2, (0, 2), (2, 4, 6)) == [[2, 2, 2], [-2, 10, 10]]
    assert O.legendre_projection_matrix(4, (0, 2, 4), (4, 6, 8)) == [
        [56, 144, 264], [-80, 360, 960], [24, -864, 216]]


# ------------------------------------------------------------------ frame pins
def test_frame_matches_standard_rotation_for_z_pole():
    """With the pole along z the frame is the columns of S(d) (Eq. def_standard_rotation)."""
    rng = np.random.default_rng(1)
    th = rng.uniform(0.1, 3.0, 20)
    ph = rng.uniform(0, 2 * np.pi, 20)
    d = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    et, ep = O.sky_frame(d, (0, 0, 1))
    np.testing.assert_allclose(et, np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1), atol=1e-14)
    np.testing.assert_allclose(ep, np.stack([-np.sin(ph), np.cos(ph), 0 * ph], 1), atol=1e-14)


def test_helicity_identities_and_projection():
    """e_ii = e_ij e_ij = 0, e_ij e*_ij = 1 (Sec. 2.2); gamma_ij = 2Re(gamma e*_ij) is traceless and
    transverse, and equals Lambda^(2)_ij,kl(x) s_kl (Eqs. Lambda2_def, 2Dshear_from_3Dshape)."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((30, 3))
    x /= np.linalg.norm(x, axis=1)[:, None]
    et, ep = O.sky_frame(x, (-1, 0, 0))
    e = O.helicity_tensor(et, ep)
    assert np.allclose(np.einsum("nii->n", e), 0, atol=1e-14)
    assert np.allclose(np.einsum("nij,nij->n", e, e), 0, atol=1e-14)
    assert np.allclose(np.einsum("nij,nij->n", e, np.conj(e)), 1, atol=1e-14)
    s6 = rng.standard_normal((6, 30))
    g = O.shear(s6, None, e)
    gij = 2 * np.real(g[:, None, None] * np.conj(e))
    assert np.allclose(np.einsum("nii->n", gij), 0, atol=1e-13)
    assert np.allclose(np.einsum("nij,nj->ni", gij, x), 0, atol=1e-13)
    s = O.full_tensor(s6)
    P = np.eye(3)[None] - x[:, :, None] * x[:, None, :]
    lam = 0.5 * (np.einsum("nik,njl->nijkl", P, P) + np.einsum("nil,njk->nijkl", P, P)
                 - np.einsum("nij,nkl->nijkl", P, P))
    np.testing.assert_allclose(np.einsum("nijkl,nkl->nij", lam, s), gij, atol=1e-13)


# ------------------------------------------------ expansion vs direct evaluation
def _on_node_catalogue(n, box, count, seed):
    rng = np.random.default_rng(seed)
    cells = rng.choice(n ** 3, size=count, replace=False)
    ix, iy, iz = np.unravel_index(cells, (n, n, n))
    h = box / n
    pos = np.stack([ix * h, iy * h, iz * h]).astype(np.float64)
    s6 = rng.standard_normal((6, count))
    w = rng.uniform(0.5, 1.5, count)
    return pos, s6, w


@pytest.mark.parametrize("kind,L", [("cross", 2), ("cross", 4), ("cross", 6), ("plus", 2), ("plus", 4),
                                    ("minus", 4), ("minus", 6), ("minus", 8), ("minus", 10), ("minus", 12)])
def test_cartesian_expansion_equals_direct_sum_on_nodes(kind, L):
    """Particles on grid nodes, CIC, no deconvolution/interlacing: the gridded Cartesian
    expansion equals the direct per-mode sum sum_g w K_X(k; x_g) e^{-ik.x_g} to rounding."""
    n, box = 12, 100.0
    pos, s6, w = _on_node_catalogue(n, box, 60, 3)
    obs = (-40.0, 30.0, -250.0)
    mg = O.ModeGrid(n, box)
    ft = O.FieldTransformer(pos, n, box, (0, 0, 0), 2, False, False, mg)
    xh = O.line_of_sight(pos, obs)
    et, ep = O.sky_frame(xh, (-1, 0, 0))
    e = O.helicity_tensor(et, ep)
    g = O.shear(s6, None, e)
    f = O.moment_field(kind, L, ft, mg, w, g, e, xh, with_b=True)
    rng = np.random.default_rng(4)
    picks = rng.choice(n ** 3 - 1, 25, replace=False) + 1
    ii = np.unravel_index(picks, (n, n, n))
    kint = np.stack([mg.nx[ii], mg.ny[ii], mg.nz[ii]], 1)
    kvec = kint * (2 * np.pi / box)
    khat = kint / np.linalg.norm(kint, axis=1)[:, None]
    kern = O.direct_kernel(kind, L, khat, xh, et, ep, g)
    want = O.direct_ft(kvec, pos, w[None, :] * kern)
    np.testing.assert_allclose(f[ii], want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def test_pair_sum_equals_factorised_product():
    """The endpoint pair double-sum (Eq. lpp_estimator_cross with d -> x) equals the product of
    the two single sums used by the FFT form, mode by mode (tiny input)."""
    rng = np.random.default_rng(5)
    npart = 40
    pos = rng.uniform(0, 50, (3, npart))
    xh = O.line_of_sight(pos, (0, 0, -300))
    et, ep = O.sky_frame(xh, (-1, 0, 0))
    g = O.shear(rng.standard_normal((6, npart)), None, O.helicity_tensor(et, ep))
    dens = rng.uniform(0.5, 2, npart)
    kvec = rng.standard_normal((7, 3)) * 0.2
    khat = kvec / np.linalg.norm(kvec, axis=1)[:, None]
    kern = O.direct_kernel("cross", 4, khat, xh, et, ep, g)
    single = O.direct_ft(kvec, pos, kern) * np.conj(O.direct_ft(kvec, pos, np.broadcast_to(dens, kern.shape)))
    dx = pos[:, :, None] - pos[:, None, :]
    pair = np.einsum("kg,h,kgh->k", kern, dens, np.exp(-1j * np.einsum("ka,agh->kgh", kvec, dx)))
    np.testing.assert_allclose(single, pair, rtol=1e-12)


def test_aliasing_bound_off_node_tsc_interlaced():
    """Off-node particles: TSC + interlacing + window deconvolution approaches the exact
    direct sum at low k (relative error < 1e-3 for k < k_Ny/4)."""
    n, box = 32, 200.0
    rng = np.random.default_rng(6)
    pos = rng.uniform(0, box, (3, 400))
    w = rng.uniform(0.5, 1.5, 400)
    mg = O.ModeGrid(n, box)
    ft = O.FieldTransformer(pos, n, box, (0, 0, 0), 3, True, True, mg)
    f = ft.ft(w.astype(complex))
    sel = (mg.n2 > 0) & (np.sqrt(mg.n2) < n / 8)
    kint = np.stack([mg.nx[sel], mg.ny[sel], mg.nz[sel]], 1)
    want = O.direct_ft(kint * 2 * np.pi / box, pos, np.broadcast_to(w, (kint.shape[0], 400)))
    err = np.abs(f[sel] - want) / np.abs(want).max()
    assert err.max() < 1e-3
    # without interlacing the error is clearly larger (the half-cell phase matters)
    ft2 = O.FieldTransformer(pos, n, box, (0, 0, 0), 3, False, True, mg)
    err2 = np.abs(ft2.ft(w.astype(complex))[sel] - want) / np.abs(want).max()
    assert err2.max() > 2 * err.max()


# --------------------------------------------------------------- GPP and tidal pins
def _grid_catalogues(n, box, dk):
    """Grid-defined fields (the paper's Sec. 4 setting): one particle per node."""
    h = box / n
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = np.stack([ix.ravel() * h, iy.ravel() * h, iz.ravel() * h])
    delta = S.real_space(dk, box).ravel()
    tij = S.tidal_tensor_grids(dk, box).reshape(6, -1)
    return pos, delta, tij


def test_gpp_identity_per_mode():
    """With x := n everywhere the LPP machinery equals the per-mode GPP estimator
    C <gamma(k) e^{-2i phi_k} Lm2_L(mu_k) delta*(k)> (Eq. gpp_estimator_cross), and likewise
    (2l+1)<gamma(k) L_l(mu) gamma*(k)> and C<gamma(k) e^{-4i phi} Lm4_L gamma(-k)> (minus L up to 12)."""
    n, box = 12, 300.0
    rng = np.random.default_rng(7)
    pos = rng.uniform(0, box, (3, 200))
    s6 = rng.standard_normal((6, 200))
    dens_w = rng.uniform(0.5, 1.5, 200)
    nvec = np.array([0.3, -0.2, 0.93])
    nvec /= np.linalg.norm(nvec)
    edges = np.linspace(0, np.pi * n / box, 6)
    plan = O.Plan(n=n, box=box, observer=(0, 0, -1e4), scheme=2, compensate=False,
                  los_proj_global=True, los_est_global=True, los_global=tuple(nvec), cross_b=True,
                  k_edges=edges, norm_override=1.0, subtract_shot=False, moments=tuple(O.MOMENTS))
    res = O.multipoles(plan, pos, shapes_s6=s6, dens_pos=pos, dens_w=dens_w)
    mg = O.ModeGrid(n, box)
    st = O.assignment_stencil(pos, n, box, (0, 0, 0), 2, 0.0)
    et, ep = O.sky_frame(nvec[None, :], (-1, 0, 0))
    e = O.helicity_tensor(et, ep)[0]
    gam = np.einsum("ij,nij->n", e, O.full_tensor(s6))
    G = np.fft.fftn(O.grid_from_stencil(st, gam, n))
    Gc = np.fft.fftn(O.grid_from_stencil(st, np.conj(gam), n))
    D = np.fft.fftn(O.grid_from_stencil(st, dens_w, n))
    kh = np.stack([mg.khat[0], mg.khat[1], mg.khat[2]], -1)
    mu = kh @ nvec
    phi = np.arctan2(kh @ ep[0], kh @ et[0])
    b, nb = O._bins(mg, edges)
    nm = np.maximum(np.bincount(b.ravel(), minlength=nb + 1)[:nb], 1)
    for L in (2, 4, 6):
        v = G * np.exp(-2j * phi) * lpmv(2, L, mu) * np.conj(D)
        want = O.norm_factor(2, L) * O._shell_sum(v, b, nb) / nm
        np.testing.assert_allclose(res.p[O.M_INDEX[("cross", L)]], want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    for l in (0, 2, 4):
        v = G * lpmv(0, l, mu) * np.conj(G)
        want = (2 * l + 1) * O._shell_sum(v, b, nb) / nm
        np.testing.assert_allclose(res.p[O.M_INDEX[("plus", l)]], want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    for L in (4, 6, 8, 10, 12):
        v = G * np.exp(-4j * phi) * lpmv(4, L, mu) * np.conj(Gc)
        want = O.norm_factor(4, L) * O._shell_sum(v, b, nb) / nm
        np.testing.assert_allclose(res.p[O.M_INDEX[("minus", L)]], want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_fixed_amplitude_tidal_field_closed_form():
    """Grid tidal field with |delta(k)|^2 fixed, GPP (case (c)): each multipole equals the
    finite shell average of C_X * kernel * (1-mu^2)/2 or (1-mu^2)^2/4 times |delta_k|^2
    (Eq. power_for_validation), B = 0, and P_+ / P_- closed forms hold."""
    n, box = 16, 400.0
    pk = S.power_law_pk(1e4, 0.1, -1.5)
    dk = S.gaussian_field_k(n, box, pk, seed=3, fixed_amplitude=True)
    pos, delta, tij = _grid_catalogues(n, box, dk)
    nvec = np.array([0.0, 0.0, 1.0])
    edges = np.linspace(0, np.pi * n / box, 7)
    plan = O.Plan(n=n, box=box, observer=(0, 0, -1e5), scheme=2, compensate=False,
                  los_proj_global=True, los_est_global=True, los_global=tuple(nvec), cross_b=True,
                  k_edges=edges, norm_override=1.0, subtract_shot=False, moments=tuple(O.MOMENTS))
    res = O.multipoles(plan, pos, shapes_s6=tij, dens_pos=pos, dens_w=delta)
    mg = O.ModeGrid(n, box)
    D = np.fft.fftn(delta.reshape(n, n, n))
    p2 = np.abs(D) ** 2
    mu = mg.khat[2]
    b, nb = O._bins(mg, edges)
    nm = np.maximum(np.bincount(b.ravel(), minlength=nb + 1)[:nb], 1)
    shell = lambda v: np.bincount(b.ravel(), weights=v.ravel(), minlength=nb + 1)[:nb] / nm
    for L in (2, 4, 6):
        want = O.norm_factor(2, L) * shell(0.5 * (1 - mu ** 2) * lpmv(2, L, mu) * p2)
        got = res.p[O.M_INDEX[("cross", L)]]
        np.testing.assert_allclose(got.real, want, rtol=1e-9, atol=1e-9 * p2.max())
        np.testing.assert_allclose(got.imag, 0, atol=1e-9 * p2.max())
    for l in (0, 2, 4):
        want = (2 * l + 1) * shell(0.25 * (1 - mu ** 2) ** 2 * lpmv(0, l, mu) * p2)
        np.testing.assert_allclose(res.p[O.M_INDEX[("plus", l)]].real, want, rtol=1e-9, atol=1e-9 * p2.max())
    for L in (4, 6, 8, 10, 12):
        want = O.norm_factor(4, L) * shell(0.25 * (1 - mu ** 2) ** 2 * lpmv(4, L, mu) * p2)
        got = res.p[O.M_INDEX[("minus", L)]]
        np.testing.assert_allclose(got.real, want, rtol=1e-9, atol=1e-9 * p2.max())
        np.testing.assert_allclose(got.imag, 0, atol=1e-9 * p2.max())
    # with many modes the shell averages approach the paper's printed 1/6, 2/15, -4/21, 2/35, 1/420
    hi = nb - 1
    ref = shell(p2)[hi]
    assert res.p[O.M_INDEX[("cross", 2)]].real[hi] / ref == pytest.approx(1 / 6, rel=0.05)
    assert res.p[O.M_INDEX[("plus", 0)]].real[hi] / ref == pytest.approx(2 / 15, rel=0.05)
    assert res.p[O.M_INDEX[("minus", 4)]].real[hi] / ref == pytest.approx(1 / 420, rel=0.05)


def test_lpp_approaches_gpp_with_observer_distance():
    """Case (a) -> case (c) as the observer recedes: |LPP - GPP| falls roughly like 1/d."""
    n, box = 12, 200.0
    pk = S.power_law_pk(1e4, 0.1, -1.5)
    dk = S.gaussian_field_k(n, box, pk, seed=5)
    pos, delta, tij = _grid_catalogues(n, box, dk)
    edges = np.linspace(0, np.pi * n / box, 5)
    errs = []
    for dist in (1e3, 1e4, 1e5):
        obs = (box / 2, box / 2, box / 2 - dist)
        common = dict(n=n, box=box, observer=obs, scheme=2, compensate=False, los_global=(0, 0, 1),
                      k_edges=edges, norm_override=1.0, subtract_shot=False,
                      moments=(("cross", 2), ("plus", 2), ("minus", 4)))
        a = O.multipoles(O.Plan(**common), pos, shapes_s6=tij, dens_pos=pos, dens_w=delta)
        c = O.multipoles(O.Plan(los_proj_global=True, los_est_global=True, **common), pos,
                         shapes_s6=tij, dens_pos=pos, dens_w=delta)
        i = O.M_INDEX[("cross", 2)]
        errs.append(np.max(np.abs(a.p[i] - c.p[i])) / np.max(np.abs(c.p[i])))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 5 and errs[0] / errs[1] > 5


def test_shot_noise_and_normalisation_periodic():
    """Pure shape noise, periodic box: P_+^(0) before subtraction scatters around the shot noise
    Sum w^2|gamma|^2/I with I = (Sum w)^2/V, so the subtracted monopole is consistent with zero."""
    n, box = 16, 300.0
    rng = np.random.default_rng(8)
    npart = 3000
    pos = rng.uniform(0, box, (3, npart))
    g12 = rng.standard_normal((2, npart)) * 0.3
    edges = np.linspace(0.05, np.pi * n / box, 4)
    plan = O.Plan(n=n, box=box, observer=(box / 2, box / 2, -2000), scheme=3, interlace=True,
                  k_edges=edges, moments=(("plus", 0),))
    r = O.multipoles(plan, pos, shapes_g12=g12)
    assert r.norm_auto == pytest.approx(npart ** 2 / box ** 3)
    assert r.shot_plus == pytest.approx(np.sum(g12 ** 2) / r.norm_auto)
    rel = r.p[O.M_INDEX[("plus", 0)]].real / r.shot_plus
    assert np.all(np.abs(rel) < 0.25)


# ------------------------------------------------------------------ window multipoles
def test_window_fft_equals_pair_count_on_nodes():
    """Randoms on grid nodes, CIC without deconvolution: the FFT window multipoles equal
    the brute-force endpoint pair sums exactly (Eq. windowQ_ell with d = x)."""
    n, box = 16, 160.0
    rng = np.random.default_rng(31)
    cnt = 150
    cells = rng.choice(n ** 3, cnt, replace=False)
    ix, iy, iz = np.unravel_index(cells, (n, n, n))
    h = box / n
    pos = np.stack([ix * h, iy * h, iz * h]).astype(np.float64)
    w = rng.uniform(0.5, 1.5, cnt)
    nbar = rng.uniform(0.5, 2.0, cnt)
    obs = (box / 2, box / 2, -400.0)
    edges = np.linspace(0.0, 6.5 * h, 7)
    fft = O.window_multipoles(n, box, (0, 0, 0), obs, pos, w, nbar, 0.7, edges, scheme=2, compensate=False)
    brute = O.window_pair_count(n, box, obs, pos, w, nbar, 0.7, edges)
    np.testing.assert_allclose(fft.q, brute, rtol=1e-10, atol=1e-12 * np.abs(brute).max())


def test_window_uniform_periodic_is_isotropic():
    """A uniform periodic window seen from far away (x ~ z for every random): Q_0 = 1 and
    Q_l(b) = (2l+1) <L_l(s_z)> over the lattice separations of shell b (a finite-sum identity;
    it tends to 0 for l > 0 in wide shells)."""
    from scipy.special import eval_legendre
    n, box = 24, 240.0
    rng = np.random.default_rng(32)
    cnt = 60000
    pos = rng.uniform(0, box, (3, cnt))
    nbar = np.full(cnt, cnt / box ** 3)
    edges = np.linspace(10.0, 80.0, 6)
    r = O.window_multipoles(n, box, (0, 0, 0), (box / 2, box / 2, -1e7), pos, None, nbar, 1.0, edges,
                            scheme=3, compensate=True)
    sx, sy, sz, h = O._separations(n, box)
    q2 = sx * sx + sy * sy + sz * sz
    b = np.searchsorted(edges, h * np.sqrt(q2), side="right") - 1
    mu = sz / np.sqrt(np.maximum(q2, 1e-300))
    for li, ell in enumerate((0, 2, 4, 6, 8)):
        want = np.array([(2 * ell + 1) * eval_legendre(ell, mu[(b == i) & (q2 > 0)]).mean() for i in range(5)])
        np.testing.assert_allclose(r.q[li], want, atol=0.03)
    np.testing.assert_allclose(r.q[0], 1.0, atol=0.02)
