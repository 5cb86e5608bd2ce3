"""The timed survey configuration's kernels against the FP64 oracle at full grid size.

The benchmark's estimate runs on a 512^3 grid with TSC + interlacing in FP32, where every
even channel batch goes through the two-slot fused assignment + x-FFT kernel with
fixed-point (integer) tiles and per-tile range records, and its window multipoles run on the
same large grid.  These tests put a polar-cap survey catalogue (the benchmark's geometry and
shells, fewer galaxies so that the oracle finishes in minutes) through exactly those
kernels and compare every moment and shell with the oracle, element by element, at the FP32
tolerance 1e-5 of the per-bin scale |P| + sqrt(P_+^(0) P_dd^(0)).  The path counters of the
plan show that the two-slot fixed-point form did run.
"""
import numpy as np
import pytest

from oracle import lpp_oracle as O
from paper_2202_11839_gb300 import synthetic as S
from tests import parity_util as U

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
BOX = 4000.0
OBS = (BOX / 2, BOX / 2, 200.0)


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_11839_gb300 import lpp
    lpp.load_library()
    return lpp


@pytest.fixture(scope="module")
def survey():
    data, rand = S.survey_mock(6000, 40000, 64, BOX, S.bbks_pk(0.2, 0.8), 1.0, 0.25, 3, OBS)
    return data, rand


def test_survey_512_two_slot_fixed_point_matches_oracle(L, survey):
    """512^3, TSC + interlacing, FP32, the benchmark's 40 shells to k = 0.2: the cross L = 2
    moment with its B part (10 channel fields: batches of 8 and 2, both even, so both run two
    slots per CTA), the density and plus monopoles from the partner pass."""
    data, rand = survey
    cat = dict(pos=data.pos, shape=data.shape, rpos=rand.pos, rnbar=rand.nbar)
    cfg = dict(n=512, box=BOX, observer=OBS, scheme=3, interlace=True, k_edges=S.linear_edges(0.0, 0.2, 40),
               cross_b=True,
               gpu_moments=(1 << L.LPP_MOM_DD0) | (1 << L.LPP_MOM_CROSS2) | (1 << L.LPP_MOM_PLUS0),
               oracle_moments=(("dd", 0), ("cross", 2), ("plus", 0)))
    gpu = U.run_gpu(cfg, cat, L.LPP_FP32)
    ps = gpu.extra["path"]
    assert ps["two_slot_launches"] == 2, ps
    assert ps["two_slot_fixed_tiles"] > 0, ps
    ref = U.run_oracle(cfg, cat)
    err = U.assert_parity(gpu, ref, TOL32, "survey 512^3 two-slot")
    print("per-moment max relative error:", {f"{k}{l}": float(e) for (k, l), e in zip(O.MOMENTS, err)})


def test_survey_window_256_matches_oracle(L, survey):
    """Window multipoles Q_0, Q_2, Q_4 of the survey randoms on a 256^3 grid over the same box
    (the bench computes them on its 512^3 grid with the same kernels), 95 shells of 20 Mpc/h."""
    import torch
    data, rand = survey
    n = 256
    s_edges = np.linspace(0.0, 1900.0, 96)
    plan = L.Plan(n, BOX, np.linspace(0.0, 0.1, 3), observer=OBS, scheme=L.LPP_TSC, compensate=True,
                  precision=L.LPP_FP32, moments=1, max_shapes=data.count, max_randoms=rand.count)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plan.assign(L.LPP_SHAPES, t(data.pos))
    plan.assign(L.LPP_RANDOMS, t(rand.pos), None, t(rand.nbar))
    q, sm, npt, norm = plan.window_q(s_edges)
    plan.close()
    alpha = data.count / rand.count
    ref = O.window_multipoles(n, BOX, (0, 0, 0), OBS, rand.pos, None, rand.nbar, alpha, s_edges, scheme=3,
                              compensate=True, ells=(0, 2, 4))
    np.testing.assert_array_equal(npt, ref.n_points)
    np.testing.assert_allclose(sm, ref.s_mean, rtol=1e-12)
    assert abs(norm - ref.norm) <= 1e-6 * abs(ref.norm)
    scale = np.abs(ref.q[0])[None, :] + np.abs(ref.q)
    err = np.abs(q[:3] - ref.q) / np.where(scale > 0, scale, 1.0)
    assert err.max() < TOL32, err.max(axis=1)


def test_benchmark_workload_fp32_matches_fp64_path(L):
    """The benchmark's own workload (1.5M shapes, 15M randoms, 512^3, all ten slots): the FP32
    estimate against the FP64 path on the same catalogues, every slot within 1e-5 of the
    per-bin scale (the FP64 path itself matches the oracle to 1e-10 in the parity tests).  The
    lowest shells of the density monopole are the sensitive ones: there the density field
    data - alpha randoms nearly cancels, and any bias in its accumulation shows."""
    import torch
    wl = S.workload_survey()
    dev = torch.device("cuda", 0)
    common = dict(origin=wl.origin, observer=wl.observer, pole=wl.pole, scheme=L.LPP_TSC, interlace=True,
                  compensate=True, moments=L.LPP_WANT_ALL, max_shapes=wl.shapes.count, max_randoms=wl.randoms.count)
    est = {}
    for prec, dt in ((L.LPP_FP32, np.float32), (L.LPP_FP64, np.float64)):
        tt = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32), dtype=dt)).to(dev)
        plan = L.Plan(wl.n, wl.box, wl.k_edges, precision=prec, **common)
        plan.assign(L.LPP_SHAPES, tt(wl.shapes.pos), None, None, tt(wl.shapes.shape), L.LPP_SHAPE_TENSOR6)
        plan.assign(L.LPP_RANDOMS, tt(wl.randoms.pos), None, tt(wl.randoms.nbar))
        est[prec] = plan.multipoles()
        if prec == L.LPP_FP32:
            ps = plan.path_stats()
        assert plan.guard_intact()
        plan.close()
        del plan
        torch.cuda.empty_cache()
    a, b = est[L.LPP_FP32], est[L.LPP_FP64]
    assert ps["two_slot_launches"] > 0 and ps["two_slot_fixed_tiles"] > 0, ps
    pp = np.abs(b.raw[L.LPP_MOM_PLUS0].real) / b.norm_auto
    pd = np.abs(b.raw[L.LPP_MOM_DD0].real) / b.norm_dd
    sc = np.abs(b.p) + np.sqrt(pp * pd)[None, :]
    err = (np.abs(a.p - b.p) / np.where(sc > 0, sc, 1.0)).max(axis=1)[:10]
    assert err.max() < TOL32, {L.MOMENT_NAMES[i]: float(e) for i, e in enumerate(err)}
