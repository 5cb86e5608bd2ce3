"""Shared helpers for parity tests: run one catalogue set through the CUDA path and the oracle."""
from __future__ import annotations

import math

import numpy as np

from oracle import lpp_oracle as O
from paper_2202_11839_gb300 import synthetic as S

ALL_MOMENTS = tuple(O.DEFAULT_MOMENTS)


def oracle_rows(p: np.ndarray) -> np.ndarray:
    """The rows of a GPU estimate (the library's slot order) that the oracle's moments
    (O.MOMENTS, in its own order) correspond to."""
    from paper_2202_11839_gb300 import lpp as L
    return p[[L.MOMENT_NAMES.index(f"{k}{ell}") for (k, ell) in O.MOMENTS]]


def make_case(kind: str, n: int, count: int, seed: int, box: float = 300.0, n_rand: int = 0,
              dtype=np.float64, separate_density: bool = False, gamma12: bool = False, zslab=None,
              outlier: float = 0.0, yslab=None):
    """Small synthetic catalogues: uniform positions, random tensors (or gamma_1,2), optional
    randoms; with zslab = (a, b) every catalogue is confined to a <= z / box < b (so most z
    planes of the grid receive nothing)."""
    rng = np.random.default_rng(seed)
    lo = 0.0

    def squeeze(p):
        # zslab / yslab = (a, b): confine that coordinate to a <= c / box < b
        for ax, sl in ((2, zslab), (1, yslab)):
            if sl is not None:
                p = p.copy()
                p[ax] = (sl[0] * box + (p[ax] / box) * (sl[1] - sl[0]) * box).astype(p.dtype)
        return p
    pos = squeeze(S.uniform_positions(count, box, (lo, lo, lo), seed, 0, dtype))
    shape = rng.standard_normal((2 if gamma12 else 6, count)).astype(dtype)
    w = rng.uniform(0.5, 1.5, count).astype(dtype)
    if outlier:
        w[count // 3] *= dtype(outlier)   # one galaxy far heavier than the rest
    out = dict(pos=pos, w=w, shape=shape)
    if separate_density:
        out["dpos"] = squeeze(S.uniform_positions(count // 2 + 7, box, (lo, lo, lo), seed, 5, dtype))
        out["dw"] = rng.uniform(0.5, 1.5, out["dpos"].shape[1]).astype(dtype)
    if n_rand:
        out["rpos"] = squeeze(S.uniform_positions(n_rand, box, (lo, lo, lo), seed, 6, dtype))
        out["rw"] = rng.uniform(0.8, 1.2, n_rand).astype(dtype)
        out["rnbar"] = rng.uniform(0.5, 2.0, n_rand).astype(dtype)
    return out


def run_oracle(cfg: dict, cat: dict) -> O.Result:
    plan = O.Plan(n=cfg["n"], box=cfg["box"], origin=cfg.get("origin", (0, 0, 0)), observer=cfg["observer"],
                  pole=cfg.get("pole", (-1, 0, 0)), scheme=cfg["scheme"], interlace=cfg["interlace"],
                  compensate=cfg.get("compensate", True),
                  los_proj_global=cfg.get("los_proj", 0) == 1, los_est_global=cfg.get("los_est", 0) == 1,
                  los_global=cfg.get("los_global", (0, 0, 1)), cross_b=cfg.get("cross_b", True),
                  k_edges=cfg["k_edges"], norm_override=cfg.get("norm_override", 0.0),
                  subtract_shot=cfg.get("subtract_shot", True), moments=cfg.get("oracle_moments", ALL_MOMENTS))
    g12 = cat["shape"] if cat["shape"].shape[0] == 2 else None
    s6 = cat["shape"] if cat["shape"].shape[0] == 6 else None
    return O.multipoles(plan, cat["pos"], cat.get("w"), s6, g12, cat.get("dpos"), cat.get("dw"),
                        cat.get("rpos"), cat.get("rw"), cat.get("rnbar"))


def run_oracle_density(cfg: dict, cat: dict) -> O.DensityResult:
    """Density multipoles l = 0, 2, 4 of the oracle (Eq. lpp_dens_app) for the catalogue set:
    the density catalogue (else the shape galaxies) minus alpha randoms."""
    plan = O.Plan(n=cfg["n"], box=cfg["box"], origin=cfg.get("origin", (0, 0, 0)), observer=cfg["observer"],
                  scheme=cfg["scheme"], interlace=cfg["interlace"], compensate=cfg.get("compensate", True),
                  los_est_global=cfg.get("los_est", 0) == 1, los_global=cfg.get("los_global", (0, 0, 1)),
                  k_edges=cfg["k_edges"], norm_override=cfg.get("norm_override", 0.0),
                  subtract_shot=cfg.get("subtract_shot", True))
    dpos, dw = (cat["dpos"], cat.get("dw")) if "dpos" in cat else (cat["pos"], cat.get("w"))
    return O.density_multipoles(plan, dpos, dw, cat.get("rpos"), cat.get("rw"), cat.get("rnbar"))


def run_gpu(cfg: dict, cat: dict, precision: int, device_inputs: bool = True):
    import torch

    from paper_2202_11839_gb300 import lpp as L
    dt = np.float64 if precision == L.LPP_FP64 else np.float32
    moments = cfg.get("gpu_moments", L.LPP_WANT_ALL) | (L.LPP_WANT_CROSS_B if cfg.get("cross_b", True) else 0)
    plan = L.Plan(cfg["n"], cfg["box"], cfg["k_edges"], origin=cfg.get("origin", (0, 0, 0)),
                  observer=cfg["observer"], pole=cfg.get("pole", (-1, 0, 0)), scheme=cfg["scheme"],
                  interlace=cfg["interlace"], compensate=cfg.get("compensate", True), precision=precision,
                  los_proj=cfg.get("los_proj", 0), los_est=cfg.get("los_est", 0),
                  los_global=cfg.get("los_global", (0, 0, 1)), moments=moments,
                  norm_override=cfg.get("norm_override", 0.0), subtract_shot=cfg.get("subtract_shot", True),
                  max_shapes=cat["pos"].shape[1], max_density=cat["dpos"].shape[1] if "dpos" in cat else 0,
                  max_randoms=cat["rpos"].shape[1] if "rpos" in cat else 0, host_inputs=not device_inputs,
                  batch=cfg.get("batch", 0), fused_slots=cfg.get("fused_slots", 0))

    def conv(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        return torch.from_numpy(a).cuda() if device_inputs else a

    kind = L.LPP_SHAPE_GAMMA12 if cat["shape"].shape[0] == 2 else L.LPP_SHAPE_TENSOR6
    plan.assign(L.LPP_SHAPES, conv(cat["pos"]), conv(cat.get("w")), None, conv(cat["shape"]), kind)
    if "dpos" in cat:
        plan.assign(L.LPP_DENSITY, conv(cat["dpos"]), conv(cat.get("dw")))
    if "rpos" in cat:
        plan.assign(L.LPP_RANDOMS, conv(cat["rpos"]), conv(cat.get("rw")), conv(cat.get("rnbar")))
    est = plan.multipoles()
    est.extra["path"] = plan.path_stats()
    assert plan.guard_intact(), "a kernel wrote outside the plan workspace"
    plan.close()
    return est


def scale(ref: O.Result) -> np.ndarray:
    """Per-bin error scale |P| + sqrt(P_+^(0) P_dd^(0)) (both before shot-noise subtraction)."""
    pp = np.abs(ref.raw[O.M_INDEX[("plus", 0)]].real) / max(ref.norm_auto, 1e-300)
    pd = np.abs(ref.raw[O.M_INDEX[("dd", 0)]].real) / max(ref.norm_dd, 1e-300)
    return np.abs(ref.p) + np.sqrt(pp * pd)[None, :]


def max_rel_err(gpu, ref: O.Result) -> np.ndarray:
    """max over bins of |gpu - oracle| / scale, per moment slot (real and imaginary parts)."""
    sc = scale(ref)
    sc = np.where(sc > 0, sc, 1.0)
    d = np.abs(oracle_rows(gpu.p) - ref.p) / sc
    return d.max(axis=1)


def assert_parity(gpu, ref: O.Result, tol: float, label: str = ""):
    np.testing.assert_array_equal(gpu.n_modes, ref.n_modes)
    np.testing.assert_allclose(gpu.k_mean, ref.k_mean, rtol=1e-13, atol=0)
    # scalar sums: per-particle shears are formed in the path's precision
    stol = min(1e-9, tol * 0.1) if tol < 1e-8 else tol * 0.1
    for nm in ("norm_auto", "norm_cross", "norm_dd", "shot_plus", "shot_dd", "alpha"):
        a, b = getattr(gpu, nm), getattr(ref, nm)
        assert abs(a - b) <= stol * max(abs(b), 1e-300) + 1e-300, (label, nm, a, b)
    err = max_rel_err(gpu, ref)
    bad = {O.MOMENTS[i]: float(e) for i, e in enumerate(err) if not e <= tol}
    assert not bad, f"{label}: per-moment max relative error above {tol}: {bad}"
    return err


def default_edges(n: int, box: float, nb: int = 8, frac: float = 1.0):
    kny = math.pi * n / box
    return np.linspace(0.0, kny * frac, nb + 1)
