"""Density multipoles P^(l)_dd, l = 2, 4 (Eq. lpp_dens_app) on the GPU against the FP64 oracle.

The oracle forms delta^(l)(k) = FT[w L_l(khat . xhat)] by expanding L_l into Cartesian
monomials of khat and xhat (one FFT per monomial); the CUDA path uses the addition theorem
(2l + 1 real harmonic fields of each catalogue).  The two must agree element by element:
1e-10 of the per-shell scale |P^(l)| + P^(0)_dd (before shot-noise subtraction) in FP64,
1e-5 in FP32.  Cases: periodic box, randoms (density = data - alpha randoms), a separate
density catalogue, the global line of sight of Eq. gpp_dens, CIC and TSC, interlaced and not
(two fields per grid), and a plan that also computes every tensor moment (its tensor slots
must still match the oracle: the density channels run in batches of their own).
"""
import numpy as np
import pytest

from oracle import lpp_oracle as O
from tests import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_11839_gb300 import lpp
    lpp.load_library()
    return lpp


def _cfg(n, box, **kw):
    c = dict(n=n, box=box, observer=(box / 2, box / 2, -700.0), scheme=3, interlace=True,
             k_edges=U.default_edges(n, box, kw.pop("nb", 8), kw.pop("frac", 1.0)), cross_b=False)
    c.update(kw)
    return c


def _check(L, gpu, dref, tol, label):
    np.testing.assert_array_equal(gpu.n_modes, dref.n_modes)
    assert abs(gpu.norm_dd - dref.norm) <= 1e-9 * abs(dref.norm), (label, gpu.norm_dd, dref.norm)
    mono = np.abs(dref.raw[0].real) / dref.norm
    for i, slot in ((1, L.LPP_MOM_DD2), (2, L.LPP_MOM_DD4)):
        sc = np.abs(dref.p[i]) + mono
        err = (np.abs(gpu.p[slot] - dref.p[i]) / np.where(sc > 0, sc, 1.0)).max()
        assert err < tol, (label, dref.ells[i], err)
    sc0 = np.abs(dref.p[0]) + mono
    err0 = (np.abs(gpu.p[L.LPP_MOM_DD0] - dref.p[0]) / np.where(sc0 > 0, sc0, 1.0)).max()
    assert err0 < tol, (label, 0, err0)


CASES = {
    "periodic_tsc_il": (_cfg(16, 300.0), dict(count=1500)),
    "randoms_tsc_il": (_cfg(16, 300.0), dict(count=1200, n_rand=3000)),
    "separate_density_randoms_cic": (_cfg(16, 300.0, scheme=2, interlace=False), dict(count=900, n_rand=2500,
                                                                                       separate_density=True)),
    "global_los_randoms": (_cfg(16, 300.0, los_est=1, los_global=(0.3, -0.2, 0.93)), dict(count=1000, n_rand=2000)),
    "pruned_n32_randoms_nonil": (_cfg(32, 400.0, interlace=False, frac=0.4, nb=5), dict(count=2500, n_rand=5000)),
    "zslab_n32_randoms": (_cfg(32, 300.0), dict(count=1500, n_rand=3000, zslab=(0.3, 0.45))),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_density_multipoles_fp64(L, name):
    cfg, ck = CASES[name]
    cfg = dict(cfg, gpu_moments=L.LPP_WANT_DENSITY | (1 << L.LPP_MOM_DD0))
    cat = U.make_case(name, cfg["n"], seed=13, box=cfg["box"], dtype=np.float64, **ck)
    gpu = U.run_gpu(cfg, cat, L.LPP_FP64)
    _check(L, gpu, U.run_oracle_density(cfg, cat), 1e-10, name)


@pytest.mark.parametrize("name", ["randoms_tsc_il", "pruned_n32_randoms_nonil"])
def test_density_multipoles_fp32(L, name):
    cfg, ck = CASES[name]
    cfg = dict(cfg, gpu_moments=L.LPP_WANT_DENSITY | (1 << L.LPP_MOM_DD0))
    cat = U.make_case(name, cfg["n"], seed=17, box=cfg["box"], dtype=np.float32, **dict(ck, count=4 * ck["count"]))
    gpu = U.run_gpu(cfg, cat, L.LPP_FP32)
    _check(L, gpu, U.run_oracle_density(cfg, cat), 1e-5, name)


@pytest.mark.parametrize("prec,tol,n", [(1, 1e-10, 16), (0, 1e-5, 32)])
def test_density_with_every_tensor_moment(L, prec, tol, n):
    """All twelve slots in one plan: the tensor slots against O.multipoles and the density
    slots against O.density_multipoles (FP32: n = 32, 8-grid batches of tensor channels
    followed by the 14 density channels)."""
    dt = np.float64 if prec else np.float32
    cfg = _cfg(n, 400.0, cross_b=True, gpu_moments=L.LPP_WANT_ALL | L.LPP_WANT_DENSITY)
    cat = U.make_case("all12", n, count=3000, seed=19, box=400.0, dtype=dt, n_rand=6000)
    gpu = U.run_gpu(cfg, cat, prec)
    U.assert_parity(gpu, U.run_oracle(cfg, cat), tol, "all twelve slots")
    _check(L, gpu, U.run_oracle_density(cfg, cat), tol, "all twelve slots")
