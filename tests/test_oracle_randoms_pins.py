"""Pins of the randoms branch of the oracle's estimator (normalisation, alpha, shot noise).

With a randoms catalogue the density field is delta = data - alpha randoms, alpha = sum w_d /
sum w_r, the normalisation is I = alpha sum_r nbar w_r^2 and the density shot noise is
(sum w_d^2 + alpha^2 sum w_r^2) / I (the reading of the paper's silence on normalisation and
shot noise; only the plus monopole and the density monopole carry shot noise, Sec. 5).
These tests fix those formulas against facts that do not come from the oracle:

* closed form: uniform randoms with nbar = N_d / V give I = (sum w)^2 / V, the periodic
  normalisation, for unit and for constant weights;
* statistics of a Poisson catalogue: data and randoms drawn independently and uniformly on
  the grid nodes have E|delta(k)|^2 = sum w_d^2 + alpha^2 sum w_r^2 exactly at every k != 0
  (CIC on nodes without deconvolution is the exact DFT of the point set), so the subtracted
  P_dd^(0) and P_+^(0) scatter around zero with the known spread sqrt(2 / N_modes);
* a clustered catalogue (Poisson counts of lam (1 + delta_x) per node) recovers the power of
  the input field delta_x, V |DFT delta|^2 / n^6, through I.
Planting a dropped alpha in I, or a dropped alpha^2 in the shot noise, fails these tests.
"""
import math

import numpy as np
import pytest

from oracle import lpp_oracle as O

N, BOX = 32, 320.0
H = BOX / N


def _on_nodes(rng, cnt):
    return (rng.integers(0, N, (3, cnt)) * H).astype(np.float64)


def _plan(moments):
    return O.Plan(n=N, box=BOX, observer=(BOX / 2, BOX / 2, -2000.0), scheme=2, interlace=False, compensate=False,
                  k_edges=np.linspace(0.0, math.pi * N / BOX, 9), moments=moments)


@pytest.mark.parametrize("c", [1.0, 1.7])
def test_uniform_randoms_normalisation_is_the_periodic_one(c):
    rng = np.random.default_rng(40)
    nd, nr = 3000, 9000
    dp = rng.uniform(0, BOX, (3, nd))
    rp = rng.uniform(0, BOX, (3, nr))
    wd, wr = np.full(nd, c), np.full(nr, c)
    nbar = np.full(nr, nd / BOX ** 3)
    g12 = rng.standard_normal((2, nd))
    r = O.multipoles(_plan((("dd", 0),)), dp, wd, None, g12, None, None, rp, wr, nbar)
    assert r.alpha == pytest.approx(nd / nr, rel=1e-14)
    want = (c * nd) ** 2 / BOX ** 3
    for nm in ("norm_dd", "norm_auto", "norm_cross"):
        assert getattr(r, nm) == pytest.approx(want, rel=1e-12), nm
    # shot noise of the density: (N_d c^2 + alpha^2 N_r c^2) / I = V (1 + N_d/N_r) / N_d
    assert r.shot_dd == pytest.approx(BOX ** 3 * (1.0 + nd / nr) / nd, rel=1e-12)


def test_poisson_catalogue_with_randoms_is_pure_shot_noise():
    rng = np.random.default_rng(41)
    nd, nr = 20000, 40000
    dp, rp = _on_nodes(rng, nd), _on_nodes(rng, nr)
    wd, wr = rng.uniform(0.5, 1.5, nd), rng.uniform(0.5, 1.5, nr)
    nbar = np.full(nr, nd / BOX ** 3)
    g12 = rng.standard_normal((2, nd)) * 0.3
    r = O.multipoles(_plan((("dd", 0), ("plus", 0))), dp, wd, None, g12, None, None, rp, wr, nbar)
    for slot, shot in ((("dd", 0), r.shot_dd), (("plus", 0), r.shot_plus)):
        p = r.p[O.M_INDEX[slot]].real / shot
        # a mode and its mirror carry the same |delta|^2: N / 2 independent exponential variates
        tot = np.sum(p * r.n_modes) / np.sum(r.n_modes)
        assert abs(tot) < 4.0 * math.sqrt(2.0 / np.sum(r.n_modes)), (slot, tot)
        big = r.n_modes >= 1000
        assert np.all(np.abs(p[big]) < 5.0 * np.sqrt(2.0 / r.n_modes[big])), (slot, p)


def test_clustered_catalogue_with_randoms_recovers_the_input_power():
    rng = np.random.default_rng(43)
    lam = 12.0
    delta = rng.uniform(-0.6, 0.6, (N, N, N))
    counts = rng.poisson(lam * (1.0 + delta))
    idx = np.nonzero(counts)
    dp = (np.repeat(np.stack(idx), counts[idx], axis=1) * H).astype(np.float64)
    nd = dp.shape[1]
    rp = _on_nodes(rng, 2 * nd)
    nbar = np.full(rp.shape[1], nd / BOX ** 3)
    plan = _plan((("dd", 0),))
    r = O.multipoles(plan, dp, None, None, np.zeros((2, nd)), None, None, rp, None, nbar)
    mg = O.ModeGrid(N, BOX)
    b, nb = O._bins(mg, np.asarray(plan.k_edges))
    pw = np.abs(np.fft.fftn(delta)) ** 2 * BOX ** 3 / N ** 6
    want = np.bincount(b.ravel(), weights=pw.ravel(), minlength=nb + 1)[:nb] / np.maximum(r.n_modes, 1)
    got = r.p[O.M_INDEX[("dd", 0)]].real
    assert np.sum(got * r.n_modes) / np.sum(want * r.n_modes) == pytest.approx(1.0, abs=0.04)
    big = r.n_modes >= 1000
    np.testing.assert_allclose(got[big], want[big], rtol=0.15)
