"""CUDA path vs the FP64 oracle, element by element over every moment and shell.

Tolerances: relative to the per-bin scale |P| + sqrt(P_+^(0) P_dd^(0)); 1e-10 for the
FP64 path and 1e-5 for the FP32 bulk path (FP32 grids and products, FP64 shell sums).
"""
import math

import numpy as np
import pytest

from oracle import lpp_oracle as O
from tests import parity_util as U

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2202_11839_gb300 import lpp
    lpp.load_library()
    return lpp


def _cfg(n, box, **kw):
    c = dict(n=n, box=box, observer=(box / 2, box / 2, -800.0), scheme=2, interlace=False,
             k_edges=U.default_edges(n, box, kw.pop("nb", 8), kw.pop("frac", 1.0)))
    c.update(kw)
    return c


CASES64 = {
    "cic_periodic": (_cfg(16, 300.0), dict(count=1500)),
    "tsc_interlaced_randoms_density": (_cfg(16, 300.0, scheme=3, interlace=True),
                                       dict(count=1200, n_rand=3000, separate_density=True)),
    "gpp_global_los": (_cfg(16, 300.0, los_proj=1, los_est=1, los_global=(0.2, -0.1, 0.97)), dict(count=1000)),
    "inconsistent_los_case_b": (_cfg(16, 300.0, los_proj=0, los_est=1), dict(count=1000)),
    "pruned_k_range_n32": (_cfg(32, 400.0, scheme=3, interlace=True, frac=0.35, nb=5), dict(count=2500)),
    "no_compensation_gamma12": (_cfg(16, 250.0, compensate=False), dict(count=900, gamma12=True)),
    "tiny_grid_n8": (_cfg(8, 100.0, scheme=3, nb=3), dict(count=300)),
    "batch1_ragged": (_cfg(16, 300.0, batch=1, scheme=3, interlace=True), dict(count=700)),
    "batch3_noninterlaced": (_cfg(16, 300.0, batch=3), dict(count=700)),
    # most z planes empty: the fused pass stores nothing there and the y pass writes zeros
    "zslab_tsc_il_randoms_density_n32": (_cfg(32, 300.0, scheme=3, interlace=True),
                                         dict(count=1500, n_rand=3000, separate_density=True, zslab=(0.3, 0.45))),
    "zslab_cic_wrapping_n32": (_cfg(32, 300.0, scheme=2), dict(count=1200, zslab=(0.0, 0.08))),
    # confined in y and z: empty tiles and unreached pencils inside the reached planes
    "yz_box_tsc_il_randoms_n32": (_cfg(32, 300.0, scheme=3, interlace=True, frac=0.6),
                                  dict(count=1500, n_rand=4000, yslab=(0.55, 0.8), zslab=(0.2, 0.4))),
    # every tensor moment, the minus moments L = 10, 12 included (0x3000: slots 12 and 13)
    "minus_high_tsc_il_randoms_density": (_cfg(16, 300.0, scheme=3, interlace=True, gpu_moments=0x33FF,
                                               oracle_moments=tuple(O.MOMENTS)),
                                          dict(count=1200, n_rand=3000, separate_density=True)),
}


@pytest.mark.parametrize("name", sorted(CASES64))
def test_fp64_parity(L, name):
    cfg, ck = CASES64[name]
    cat = U.make_case(name, cfg["n"], seed=11, box=cfg["box"], dtype=np.float64, **ck)
    ref = U.run_oracle(cfg, cat)
    gpu = U.run_gpu(cfg, cat, L.LPP_FP64)
    U.assert_parity(gpu, ref, TOL64, name)


CASES32 = {
    "tsc_interlaced_n32": (_cfg(32, 500.0, scheme=3, interlace=True), dict(count=6000)),
    "cic_randoms_n32": (_cfg(32, 500.0, scheme=2, frac=0.5), dict(count=4000, n_rand=12000)),
    "gamma12_n64_pruned": (_cfg(64, 800.0, scheme=3, interlace=True, frac=0.4, nb=6), dict(count=5000, gamma12=True)),
    # one weight 1e4 times the others: coefficient maxima far above the typical value
    "outlier_weight_n32": (_cfg(32, 500.0, scheme=3, interlace=True), dict(count=6000, outlier=1.0e4)),
    "yz_box_randoms_n64": (_cfg(64, 800.0, scheme=3, interlace=True, frac=0.5),
                           dict(count=6000, n_rand=12000, yslab=(0.1, 0.35), zslab=(0.6, 0.75))),
    "zslab_randoms_n64": (_cfg(64, 800.0, scheme=3, interlace=True, frac=0.5), dict(count=6000, n_rand=12000,
                                                                                   zslab=(0.55, 0.7))),
    # the minus moments L = 10, 12 alone beside the two monopoles (slots 0, 4, 12, 13)
    "minus_high_only_n32": (_cfg(32, 500.0, scheme=3, interlace=True, gpu_moments=0x3011,
                                 oracle_moments=(("dd", 0), ("plus", 0), ("minus", 10), ("minus", 12))),
                            dict(count=6000)),
}


@pytest.mark.parametrize("name", sorted(CASES32))
def test_fp32_parity(L, name):
    cfg, ck = CASES32[name]
    cat = U.make_case(name, cfg["n"], seed=5, box=cfg["box"], dtype=np.float32, **ck)
    ref = U.run_oracle(cfg, cat)
    gpu = U.run_gpu(cfg, cat, L.LPP_FP32)
    U.assert_parity(gpu, ref, TOL32, name)


def test_host_inputs_match_device_inputs(L):
    cfg, ck = CASES32["tsc_interlaced_n32"]
    cat = U.make_case("h", cfg["n"], seed=9, box=cfg["box"], dtype=np.float32, **ck)
    a = U.run_gpu(cfg, cat, L.LPP_FP32, device_inputs=True)
    b = U.run_gpu(cfg, cat, L.LPP_FP32, device_inputs=False)
    ref = U.run_oracle(cfg, cat)
    sc = U.scale(ref)
    assert np.max(np.abs(U.oracle_rows(a.p) - U.oracle_rows(b.p)) / np.where(sc > 0, sc, 1)) < 1e-6


def test_repeat_runs_agree(L):
    """Atomic accumulation order varies between runs; results stay within the FP32 tolerance."""
    cfg, ck = CASES32["cic_randoms_n32"]
    cat = U.make_case("r", cfg["n"], seed=3, box=cfg["box"], dtype=np.float32, **ck)
    ref = U.run_oracle(cfg, cat)
    a = U.run_gpu(cfg, cat, L.LPP_FP32)
    b = U.run_gpu(cfg, cat, L.LPP_FP32)
    sc = U.scale(ref)
    assert np.max(np.abs(U.oracle_rows(a.p) - U.oracle_rows(b.p)) / np.where(sc > 0, sc, 1)) < 1e-6


def test_particle_outside_box_is_an_error(L):
    import torch
    cfg = _cfg(16, 100.0)
    cat = U.make_case("o", 16, count=50, seed=1, box=100.0, dtype=np.float64)
    cat["pos"][0, 3] = 100.5   # beyond origin + box
    with pytest.raises(L.LppError) as ei:
        U.run_gpu(cfg, cat, L.LPP_FP64)
    assert ei.value.status == L.LPP_ERR_DOMAIN


def test_upper_face_wraps_to_zero(L):
    """A particle exactly on origin + box is accepted and wraps onto node 0 (periodic)."""
    cfg = _cfg(16, 100.0)
    cat = U.make_case("f", 16, count=60, seed=2, box=100.0, dtype=np.float64)
    cat["pos"][:, 0] = (100.0, 50.0, 100.0)
    ref = U.run_oracle(cfg, cat)
    gpu = U.run_gpu(cfg, cat, L.LPP_FP64)
    U.assert_parity(gpu, ref, TOL64, "upper face")


def test_particle_on_frame_pole_is_an_error(L):
    cfg = _cfg(16, 100.0, observer=(50.0, 50.0, 50.0), pole=(0.0, 0.0, 1.0))
    cat = U.make_case("p", 16, count=40, seed=4, box=100.0, dtype=np.float64)
    cat["pos"][:, 7] = (50.0, 50.0, 80.0)   # straight above the observer, on the pole
    with pytest.raises(L.LppError) as ei:
        U.run_gpu(cfg, cat, L.LPP_FP64)
    assert ei.value.status == L.LPP_ERR_DOMAIN


def test_on_node_512_matches_direct_sum(L):
    """Full 512^3 grid (the timed configuration's size) with particles on nodes, CIC, no window
    deconvolution: the lowest shells equal the direct, unexpanded per-mode sums exactly
    (to FP32 rounding), which exercises every FFT pass, pruning and the combine at size."""
    n, box = 512, 4000.0
    rng = np.random.default_rng(12)
    cnt = 400
    cells = rng.integers(0, n, (3, cnt))
    h = box / n
    pos = (cells * h).astype(np.float32)
    shape = rng.standard_normal((6, cnt)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, cnt).astype(np.float32)
    edges = np.array([0.0, 0.004, 0.007, 0.01])
    obs = (2000.0, 2000.0, 200.0)
    cfg = dict(n=n, box=box, observer=obs, scheme=2, interlace=False, compensate=False, k_edges=edges,
               norm_override=1.0, subtract_shot=False, cross_b=True)
    gpu = U.run_gpu(cfg, dict(pos=pos, w=w, shape=shape), L.LPP_FP32)
    # direct sums over every mode of the three shells
    kf = 2 * math.pi / box
    m = int(edges[-1] / kf) + 1
    f = np.arange(-m, m + 1)
    fx, fy, fz = np.meshgrid(f, f, f, indexing="ij")
    q = (fx ** 2 + fy ** 2 + fz ** 2).ravel()
    kint = np.stack([fx.ravel(), fy.ravel(), fz.ravel()], 1)
    kmag = kf * np.sqrt(q)
    b = np.searchsorted(edges, kmag, side="right") - 1
    sel = (q > 0) & (b >= 0) & (b < len(edges) - 1)
    kint, b = kint[sel], b[sel]
    kvec = kint * kf
    khat = kint / np.linalg.norm(kint, axis=1)[:, None]
    p64 = pos.astype(np.float64)
    xh = O.line_of_sight(p64, obs)
    et, ep = O.sky_frame(xh, (-1, 0, 0))
    g = O.shear(shape.astype(np.float64), None, O.helicity_tensor(et, ep))
    w64 = w.astype(np.float64)
    D = O.direct_ft(kvec, p64, np.broadcast_to(w64, (len(kvec), cnt)))
    G = O.direct_ft(kvec, p64, np.broadcast_to(w64 * g, (len(kvec), cnt)))
    Gc = O.direct_ft(kvec, p64, np.broadcast_to(w64 * np.conj(g), (len(kvec), cnt)))
    nmodes = np.bincount(b, minlength=3)
    np.testing.assert_array_equal(gpu.n_modes, nmodes)
    partner = {"cross": np.conj(D), "plus": np.conj(G), "minus": np.conj(Gc)}
    for (kind, Lm) in [("cross", 2), ("cross", 4), ("plus", 2), ("minus", 4), ("minus", 8)]:
        F = O.direct_ft(kvec, p64, w64[None, :] * O.direct_kernel(kind, Lm, khat, xh, et, ep, g))
        fac = O.norm_factor({"cross": 2, "plus": 0, "minus": 4}[kind], Lm)
        val = F * partner[kind]
        want = fac * (np.bincount(b, weights=val.real, minlength=3) + 1j * np.bincount(b, weights=val.imag, minlength=3)) / nmodes
        got = gpu.p[O.M_INDEX[(kind, Lm)]]
        ref_scale = np.sqrt((np.bincount(b, weights=np.abs(G) ** 2, minlength=3) / nmodes) *
                            (np.bincount(b, weights=np.abs(D) ** 2, minlength=3) / nmodes))
        assert np.max(np.abs(got - want) / (np.abs(want) + ref_scale)) < TOL32, (kind, Lm)


def test_on_node_1024_matches_direct_sum(L):
    """The largest grid the library takes, 1024^3 (its own pass shapes: 8-pencil y/z tiles, a
    1024-point x transform of 2 x 8 x 8 x 8 in the fused kernel), particles on nodes, CIC, no
    deconvolution: the lowest shells equal the direct per-mode sums to FP32 rounding."""
    n, box = 1024, 8000.0
    rng = np.random.default_rng(13)
    cnt = 300
    cells = rng.integers(0, n, (3, cnt))
    h = box / n
    pos = (cells * h).astype(np.float32)
    shape = rng.standard_normal((6, cnt)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, cnt).astype(np.float32)
    edges = np.array([0.0, 0.002, 0.0035, 0.005])
    obs = (4000.0, 4000.0, -500.0)
    moments = (1 << L.LPP_MOM_DD0) | (1 << L.LPP_MOM_CROSS2) | (1 << L.LPP_MOM_PLUS2) | (1 << L.LPP_MOM_MINUS4)
    cfg = dict(n=n, box=box, observer=obs, scheme=2, interlace=False, compensate=False, k_edges=edges,
               norm_override=1.0, subtract_shot=False, cross_b=True, gpu_moments=moments, batch=2)
    gpu = U.run_gpu(cfg, dict(pos=pos, w=w, shape=shape), L.LPP_FP32)
    kf = 2 * math.pi / box
    m = int(edges[-1] / kf) + 1
    f = np.arange(-m, m + 1)
    fx, fy, fz = np.meshgrid(f, f, f, indexing="ij")
    q = (fx ** 2 + fy ** 2 + fz ** 2).ravel()
    kint = np.stack([fx.ravel(), fy.ravel(), fz.ravel()], 1)
    kmag = kf * np.sqrt(q)
    b = np.searchsorted(edges, kmag, side="right") - 1
    sel = (q > 0) & (b >= 0) & (b < len(edges) - 1)
    kint, b = kint[sel], b[sel]
    kvec = kint * kf
    khat = kint / np.linalg.norm(kint, axis=1)[:, None]
    p64 = pos.astype(np.float64)
    xh = O.line_of_sight(p64, obs)
    et, ep = O.sky_frame(xh, (-1, 0, 0))
    g = O.shear(shape.astype(np.float64), None, O.helicity_tensor(et, ep))
    w64 = w.astype(np.float64)
    D = O.direct_ft(kvec, p64, np.broadcast_to(w64, (len(kvec), cnt)))
    G = O.direct_ft(kvec, p64, np.broadcast_to(w64 * g, (len(kvec), cnt)))
    Gc = O.direct_ft(kvec, p64, np.broadcast_to(w64 * np.conj(g), (len(kvec), cnt)))
    nmodes = np.bincount(b, minlength=3)
    np.testing.assert_array_equal(gpu.n_modes, nmodes)
    shell = lambda v: (np.bincount(b, weights=v.real, minlength=3) + 1j * np.bincount(b, weights=v.imag, minlength=3)) / nmodes
    ref_scale = np.sqrt(shell(np.abs(G) ** 2).real * shell(np.abs(D) ** 2).real)
    want_dd = shell(np.abs(D) ** 2)
    assert np.max(np.abs(gpu.p[L.LPP_MOM_DD0] - want_dd) / np.abs(want_dd)) < TOL32
    partner = {"cross": np.conj(D), "plus": np.conj(G), "minus": np.conj(Gc)}
    for (kind, Lm) in [("cross", 2), ("plus", 2), ("minus", 4)]:
        F = O.direct_ft(kvec, p64, w64[None, :] * O.direct_kernel(kind, Lm, khat, xh, et, ep, g))
        fac = O.norm_factor({"cross": 2, "plus": 0, "minus": 4}[kind], Lm)
        want = fac * shell(F * partner[kind])
        got = gpu.p[L.MOMENT_NAMES.index(f"{kind}{Lm}")]
        assert np.max(np.abs(got - want) / (np.abs(want) + ref_scale)) < TOL32, (kind, Lm)


def test_empty_shape_catalogue(L):
    """No shape galaxies (count 0) beside a density catalogue and randoms: every tensor slot
    is exactly zero (their normalisation has no weight), nothing is NaN, and the density
    monopole equals the one of the same density and randoms with shapes present."""
    cfg, ck = CASES64["tsc_interlaced_randoms_density"]
    cat = U.make_case("empty", cfg["n"], seed=4, box=cfg["box"], dtype=np.float64, **ck)
    full = U.run_gpu(cfg, cat, L.LPP_FP64)
    empty = dict(cat, pos=cat["pos"][:, :0].copy(), w=cat["w"][:0].copy(), shape=cat["shape"][:, :0].copy())
    import torch
    plan = L.Plan(cfg["n"], cfg["box"], cfg["k_edges"], observer=cfg["observer"], scheme=cfg["scheme"],
                  interlace=cfg["interlace"], precision=L.LPP_FP64, moments=L.LPP_WANT_ALL | L.LPP_WANT_CROSS_B,
                  max_shapes=cat["pos"].shape[1], max_density=cat["dpos"].shape[1], max_randoms=cat["rpos"].shape[1])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plan.assign(L.LPP_SHAPES, t(empty["pos"]), t(empty["w"]), None, t(empty["shape"]), L.LPP_SHAPE_TENSOR6)
    plan.assign(L.LPP_DENSITY, t(cat["dpos"]), t(cat["dw"]))
    plan.assign(L.LPP_RANDOMS, t(cat["rpos"]), t(cat["rw"]), t(cat["rnbar"]))
    est = plan.multipoles()
    plan.close()
    assert np.all(np.isfinite(est.p)) and np.all(np.isfinite(est.raw))
    for s in range(1, 10):
        assert np.all(est.p[s] == 0), L.MOMENT_NAMES[s]
    np.testing.assert_allclose(est.p[L.LPP_MOM_DD0], full.p[L.LPP_MOM_DD0], rtol=1e-12, atol=0)


@pytest.mark.parametrize("cross_b", [True, False])
def test_fp32_interlaced_256_matches_fp64(L, cross_b):
    """256^3, TSC + interlacing, catalogue confined in y and z: the FP32 path (two slots per
    CTA, fixed-point tiles, skipped planes, pencils and columns) against the FP64 path (one
    slot per CTA, float atomics), which matches the oracle to 1e-10 on the small grids above;
    1e-5 of the per-bin scale |P| + sqrt(P_+^(0) P_dd^(0)).  With the B-mode cross parts
    there are 160 channels (20 batches of 8); without, 133, so the last batch has 5 grids and
    runs the one-slot kernel on the dynamic (slot, tile) schedule."""
    n, box = 256, 1000.0
    cat = U.make_case("box256", n, count=120_000, seed=21, box=box, dtype=np.float64, yslab=(0.2, 0.6),
                      zslab=(0.35, 0.7))
    cfg = _cfg(n, box, scheme=3, interlace=True, frac=0.5, nb=12, cross_b=cross_b)
    g64 = U.run_gpu(cfg, cat, L.LPP_FP64)
    c32 = {k: v.astype(np.float32) for k, v in cat.items()}
    g32 = U.run_gpu(cfg, c32, L.LPP_FP32)
    pp = np.abs(g64.raw[O.M_INDEX[("plus", 0)]].real) / g64.norm_auto
    pd = np.abs(g64.raw[O.M_INDEX[("dd", 0)]].real) / g64.norm_dd
    sc = np.abs(g64.p) + np.sqrt(pp * pd)[None, :]
    err = np.abs(g32.p - g64.p) / np.where(sc > 0, sc, 1.0)
    np.testing.assert_array_equal(g32.n_modes, g64.n_modes)
    assert err.max() < TOL32, {L.MOMENT_NAMES[i]: float(e) for i, e in enumerate(err.max(axis=1))}


@pytest.mark.slow
def test_periodic_fp64_workload_full_size(L):
    """The FP64 periodic workload at full size: 64^3 CIC, 50k galaxies, 20 bins to k_Ny."""
    from paper_2202_11839_gb300 import synthetic as S
    wl = S.workload_periodic_fp64()
    cat = dict(pos=wl.shapes.pos, shape=wl.shapes.shape)
    cfg = dict(n=wl.n, box=wl.box, observer=wl.observer, pole=wl.pole, scheme=wl.scheme,
               interlace=wl.interlace, k_edges=wl.k_edges, cross_b=False)
    ref = U.run_oracle(cfg, cat)
    gpu = U.run_gpu(cfg, cat, L.LPP_FP64)
    U.assert_parity(gpu, ref, TOL64, wl.name)


def test_one_slot_fused_pass_matches_two_slot(L):
    """fused_slots = 1 (the autotuner's alternative) against the library's two-slot choice at
    256^3, TSC + interlacing, FP32: the same estimate within the FP32 tolerance, and the path
    counters show which form ran."""
    n, box = 256, 1000.0
    cat = U.make_case("slots256", n, count=60_000, seed=23, box=box, dtype=np.float32, yslab=(0.2, 0.6),
                      zslab=(0.35, 0.7), n_rand=100_000)
    cfg = _cfg(n, box, scheme=3, interlace=True, frac=0.5, nb=12, cross_b=True)
    two = U.run_gpu(cfg, cat, L.LPP_FP32)
    one = U.run_gpu(dict(cfg, fused_slots=1), cat, L.LPP_FP32)
    assert two.extra["path"]["two_slot_launches"] > 0
    assert one.extra["path"]["two_slot_launches"] == 0
    pp = np.abs(two.raw[O.M_INDEX[("plus", 0)]].real) / two.norm_auto
    pd = np.abs(two.raw[O.M_INDEX[("dd", 0)]].real) / two.norm_dd
    sc = np.abs(two.p) + np.sqrt(pp * pd)[None, :]
    assert (np.abs(one.p - two.p) / np.where(sc > 0, sc, 1.0)).max() < TOL32
