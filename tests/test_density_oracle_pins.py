"""Pins of the oracle's density multipoles (Eq. lpp_dens_app, Eq. delta_ell):

* l = 0 is the density monopole slot of the tensor-moment oracle (same normalisation and
  shot noise, periodic and with randoms);
* with the global line of sight the LPP form reduces to the GPP form (Eq. gpp_dens):
  (2l+1) < L_l(khat . n) |delta(k)|^2 > with the Legendre polynomial from scipy, not from the
  Cartesian expansion;
* brute force on a tiny grid: for single wave vectors, the catalogue gridded with the
  per-galaxy weights w L_l(khat . xhat) of that wave vector (Legendre from scipy), then
  transformed and read at that k, equals delta^(l)(k) from the expansion.
A wrong multinomial count, a dropped monomial or a transposed k / x index in the expansion
fails the last two; a wrong factor (2l+1), normalisation or shot term fails the first two.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import lpp_oracle as O
from paper_2202_11839_gb300 import synthetic as S
from tests.parity_util import default_edges


def _cat(count, n_rand, seed, box=300.0):
    rng = np.random.default_rng(seed)
    pos = S.uniform_positions(count, box, (0, 0, 0), seed, 0, np.float64)
    w = rng.uniform(0.5, 1.5, count)
    out = dict(pos=pos, w=w)
    if n_rand:
        out["rpos"] = S.uniform_positions(n_rand, box, (0, 0, 0), seed, 6, np.float64)
        out["rw"] = rng.uniform(0.8, 1.2, n_rand)
        out["rnbar"] = rng.uniform(0.5, 2.0, n_rand)
    return out


def _plan(n=16, box=300.0, **kw):
    return O.Plan(n=n, box=box, observer=(150.0, 150.0, -700.0), scheme=kw.pop("scheme", 3),
                  interlace=kw.pop("interlace", True), k_edges=default_edges(n, box), **kw)


@pytest.mark.parametrize("n_rand", [0, 2000])
def test_monopole_is_the_density_slot(n_rand):
    c = _cat(1500, n_rand, 3)
    plan = _plan()
    d = O.density_multipoles(plan, c["pos"], c["w"], c.get("rpos"), c.get("rw"), c.get("rnbar"))
    # the tensor-moment oracle needs a shape catalogue: any shapes, the density slot ignores them
    shapes = np.zeros((6, c["pos"].shape[1]))
    r = O.multipoles(plan, c["pos"], c["w"], shapes, None, None, None, c.get("rpos"), c.get("rw"), c.get("rnbar"))
    np.testing.assert_allclose(d.p[0], r.p[O.M_INDEX[("dd", 0)]], rtol=1e-12, atol=0)
    assert d.norm == pytest.approx(r.norm_dd, rel=1e-14)
    assert d.shot == pytest.approx(r.shot_dd, rel=1e-14)


@pytest.mark.parametrize("nvec", [(0.0, 0.0, 1.0), (0.3, -0.5, 0.81)])
def test_global_line_of_sight_reduces_to_gpp(nvec):
    c = _cat(1200, 1500, 5)
    plan = _plan(los_est_global=True, los_global=nvec)
    d = O.density_multipoles(plan, c["pos"], c["w"], c["rpos"], c["rw"], c["rnbar"])
    mg = O.ModeGrid(plan.n, plan.box)
    ftd = O.FieldTransformer(c["pos"], plan.n, plan.box, plan.origin, plan.scheme, plan.interlace, plan.compensate, mg)
    ftr = O.FieldTransformer(c["rpos"], plan.n, plan.box, plan.origin, plan.scheme, plan.interlace, plan.compensate,
                             mg)
    alpha = c["w"].sum() / c["rw"].sum()
    delta = ftd.ft(c["w"].astype(complex)) - alpha * ftr.ft(c["rw"].astype(complex))
    nh = np.asarray(nvec) / np.linalg.norm(nvec)
    mu = mg.khat[0] * nh[0] + mg.khat[1] * nh[1] + mg.khat[2] * nh[2]
    b, nb = O._bins(mg, np.asarray(plan.k_edges))
    nm = np.maximum(d.n_modes, 1)
    for i, ell in enumerate(d.ells):
        want = (2 * ell + 1) * np.bincount(b.ravel(), weights=(eval_legendre(ell, mu) * np.abs(delta) ** 2).ravel(),
                                           minlength=nb + 1)[:nb] / nm
        np.testing.assert_allclose(d.raw[i].real, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
        assert np.abs(d.raw[i].imag).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("ell", [2, 4])
def test_brute_force_per_wave_vector(ell):
    n, box = 8, 200.0
    c = _cat(300, 0, 9, box)
    plan = O.Plan(n=n, box=box, observer=(100.0, 60.0, -150.0), scheme=2, interlace=True,
                  k_edges=default_edges(n, box))
    mg = O.ModeGrid(n, box)
    field = O.density_ell_field(plan, mg, c["pos"], c["w"], ell)
    xhat = O.line_of_sight(c["pos"], plan.observer)
    ft = O.FieldTransformer(c["pos"], n, box, plan.origin, plan.scheme, plan.interlace, plan.compensate, mg)
    rng = np.random.default_rng(1)
    for _ in range(12):
        ijk = tuple(int(v) for v in rng.integers(0, n, 3))
        if ijk == (0, 0, 0):
            continue
        kh = np.array([mg.khat[a][ijk] for a in range(3)])
        weights = c["w"] * eval_legendre(ell, xhat @ kh)
        want = ft.ft(weights.astype(complex))[ijk]
        assert abs(field[ijk] - want) <= 1e-11 * (np.abs(c["w"]).sum()), (ijk, field[ijk], want)
