"""The LPP-versus-GPP comparison of Sec. 4.2 on the polar-cap survey geometry.

Three treatments of the line of sight (LOS) on the same realisations of a tidal field
(Sec. 4.2 and its figure of the three set-ups):

* case (a): the shape field is the tidal tensor projected with each galaxy's own LOS
  (gamma = e_ij(xhat) T_ij) and measured with the LPP estimator (local LOS);
* case (b): the same projection, measured with the GPP estimator along one global LOS n,
  the direction of the survey's midpoint (Eq. gpp_estimator_cross): an inconsistent
  treatment;
* case (c): the distant-observer set-up, projection and estimator both along n.

Every estimate runs in the library (plan flags los_proj / los_est).  This module only draws
the inputs: a Gaussian density field with a BBKS spectrum on a grid, its tidal tensor
T_ij = (k_i k_j / k^2 - delta_ij / 3) delta, and uniform positions in the survey region
where the shapes s_ij = T_ij and the density weights delta are read (nearest grid point).
The fields are drawn with torch on the device, seeded; they are inputs, not the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import lpp as L
from . import synthetic as S


@dataclass
class LosStudy:
    n: int = 256                   # estimator grid
    n_field: int = 256             # grid of the simulated fields
    box: float = 4000.0
    observer: tuple = (2000.0, 2000.0, 200.0)
    r_lo: float = 1000.0
    r_hi: float = 1800.0
    theta_max: float = math.radians(60.0)
    count: int = 4_000_000         # points sampling the survey region
    k_edges: np.ndarray = None

    def __post_init__(self):
        if self.k_edges is None:
            self.k_edges = np.linspace(0.0, 0.2, 21)

    @property
    def los_global(self):
        """Direction of the survey's midpoint (the cap axis, +z) seen from the observer."""
        return (0.0, 0.0, 1.0)


def _fields(study: LosStudy, seed: int, device):
    """delta(x) and T_ij(x) on the study's field grid (torch, FP32 on the device)."""
    import torch
    n, box = study.n_field, study.box
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    white = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float64)
    dk = torch.fft.fftn(white)
    f = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64) * (2.0 * math.pi / box)
    kx, ky, kz = torch.meshgrid(f, f, f, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    kk = torch.sqrt(k2)
    pk = S.bbks_pk(0.2, 0.8)
    amp = torch.from_numpy(np.sqrt(pk(kk.cpu().numpy()) * box ** 3 / n ** 3)).to(device)
    dk = dk * amp
    nyq = torch.abs(torch.fft.fftfreq(n, d=1.0 / n, device=device)) >= n // 2
    dk[nyq, :, :] = 0
    dk[:, nyq, :] = 0
    dk[:, :, nyq] = 0
    dk[0, 0, 0] = 0
    scale = n ** 3 / box ** 3
    delta = torch.real(torch.fft.ifftn(dk)) * scale
    k2s = torch.where(k2 > 0, k2, torch.ones_like(k2))
    ks = (kx, ky, kz)
    tij = []
    for (i, j) in S.TENSOR_ORDER:
        t = ks[i] * ks[j] / k2s
        if i == j:
            t = t - 1.0 / 3.0
        tij.append(torch.real(torch.fft.ifftn(t * dk)) * scale)
    return delta.float(), torch.stack(tij).float()


def _positions(study: LosStudy, seed: int):
    """Points uniform in volume in the cap-and-shell survey region, (3, count) FP64."""
    rng = S._rng(seed, 21)
    u = rng.random((3, study.count))
    r = np.cbrt(study.r_lo ** 3 + u[0] * (study.r_hi ** 3 - study.r_lo ** 3))
    mu = 1.0 - u[1] * (1.0 - math.cos(study.theta_max))
    ph = 2.0 * math.pi * u[2]
    st = np.sqrt(1.0 - mu * mu)
    return np.stack([study.observer[0] + r * st * np.cos(ph), study.observer[1] + r * st * np.sin(ph),
                     study.observer[2] + r * mu])


def run(study: LosStudy, seeds, device=None, moments=None):
    """Mean over the realisations `seeds` of the normalised multipoles of the three cases:
    {"a": p, "b": p, "c": p}, each (LPP_N_MOMENTS, n_bins) complex, plus the per-realisation
    estimates.  The density is the sampled field delta(x) itself (weights delta at the points),
    as in the paper's grid-field set-up, and every case uses the same fixed normalisation
    I = nbar^2 V_survey (the comparison is between cases, on the same realisations)."""
    import torch
    device = torch.device(device or "cuda")
    moments = moments if moments is not None else ((1 << L.LPP_MOM_DD0) | (1 << L.LPP_MOM_CROSS2) |
                                                    (1 << L.LPP_MOM_PLUS0) | (1 << L.LPP_MOM_PLUS2))
    vol = 2.0 * math.pi * (1.0 - math.cos(study.theta_max)) * (study.r_hi ** 3 - study.r_lo ** 3) / 3.0
    nbar = study.count / vol
    norm = nbar * nbar * vol
    cases = {"a": (L.LPP_LOS_LOCAL, L.LPP_LOS_LOCAL), "b": (L.LPP_LOS_LOCAL, L.LPP_LOS_GLOBAL),
             "c": (L.LPP_LOS_GLOBAL, L.LPP_LOS_GLOBAL)}
    plans = {c: L.Plan(study.n, study.box, study.k_edges, observer=study.observer, scheme=L.LPP_TSC,
                       interlace=True, precision=L.LPP_FP32, los_proj=lp, los_est=le,
                       los_global=study.los_global, moments=moments, norm_override=norm, subtract_shot=False,
                       max_shapes=study.count, max_density=study.count, device=device)
             for c, (lp, le) in cases.items()}
    per = {c: [] for c in cases}
    h = study.box / study.n_field
    for seed in seeds:
        delta, tij = _fields(study, seed, device)
        pos = torch.from_numpy(_positions(study, seed)).to(device)
        idx = torch.remainder(torch.floor(pos / h + 0.5).long(), study.n_field)
        d_at = delta[idx[0], idx[1], idx[2]].contiguous()
        s_at = tij[:, idx[0], idx[1], idx[2]].contiguous()
        posf = pos.float().contiguous()
        for c, plan in plans.items():
            plan.assign(L.LPP_SHAPES, posf, None, None, s_at, L.LPP_SHAPE_TENSOR6)
            plan.assign(L.LPP_DENSITY, posf, d_at)
            per[c].append(plan.multipoles().p)
    for plan in plans.values():
        plan.close()
    mean = {c: np.mean(np.stack(v), axis=0) for c, v in per.items()}
    return mean, per
