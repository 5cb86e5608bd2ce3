"""Batched mocks: many periodic tidal-field catalogues of uneven size on mixed grids through
the native batch executor (lpp_batch_*), one CUDA graph launch per batch.

The mocks follow the periodic-box recipe of the estimator's validation (Sec. 4.1): a
Gaussian density field with a BBKS spectrum (Gamma = 0.2, sigma_8 = 0.8) in a periodic box
of side 2000 Mpc/h, galaxies Poisson-sampled from 1 + delta (clipped at 0), shapes equal to
the tidal tensor times -A (A = 1) plus isotropic shape noise (sigma = 0.25), observer 4000
Mpc/h below the box centre, TSC with interlacing.  The Gaussian fields (and their tidal
tensors) are drawn on the host for a few base seeds; each mock then draws its own galaxy
count, Poisson sample, positions within cells and shape noise from its own seed on the
device (torch's counter-based generator), so 64 mocks are ready in seconds.

The grids per pass of each plan (its `batch`) and the fused pass's channel fields per CTA
(`fused_slots`) are chosen by `autotune`: every combination is timed on a sample mock with the
library's own kernel timers.  (The fused kernel's tile shape, 4 x 4 pencils, is fixed at
compile time.)
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import lpp as L
from . import synthetic as S

BOX = 2000.0
OBSERVER = (BOX / 2, BOX / 2, BOX / 2 - 4000.0)
K_EDGES = {256: S.linear_edges(0.0, 0.4, 40), 512: S.linear_edges(0.0, 0.4, 40)}


@dataclass
class Mock:
    seed: int
    n: int                      # grid side of its plan
    count: int
    pos: object                 # torch CUDA float32 (3, count)
    shape: object               # torch CUDA float32 (6, count)


@dataclass
class BaseField:
    lam: object                 # torch CUDA float32 (n_field^3,): mean count per cell / total
    tij: object                 # torch CUDA float32 (6, n_field^3)
    n_field: int


def base_field(seed: int, n_field: int, device, pk=None) -> BaseField:
    import torch
    pk = pk or S.bbks_pk(0.2, 0.8)
    dk = S.gaussian_field_k(n_field, BOX, pk, seed, 1)
    lam = np.maximum(0.0, 1.0 + S.real_space(dk, BOX)).ravel()
    lam /= lam.sum()
    tij = S.tidal_tensor_grids(dk, BOX).reshape(6, -1)
    return BaseField(torch.from_numpy(lam.astype(np.float32)).to(device),
                     torch.from_numpy(tij.astype(np.float32)).to(device), n_field)


def sample_mock(bf: BaseField, count: int, seed: int, n: int, amp_a: float = 1.0, sigma_noise: float = 0.25) -> Mock:
    """Poisson sample of count * lam per cell, uniform within cells, in random order; shapes
    -A T_ij at the cell plus isotropic traceless Gaussian noise (variance 2 sigma^2 on each of
    the five orthonormal traceless components)."""
    import torch
    dev = bf.lam.device
    g = torch.Generator(device=dev)
    g.manual_seed(1_000_003 * seed + 17)
    counts = torch.poisson(bf.lam * float(count), generator=g).to(torch.int64)
    cells = torch.repeat_interleave(torch.arange(bf.lam.numel(), device=dev), counts)
    cells = cells[torch.randperm(cells.numel(), generator=g, device=dev)]
    nf = bf.n_field
    ix, iy, iz = cells // (nf * nf), (cells // nf) % nf, cells % nf
    h = BOX / nf
    jit = torch.rand((3, cells.numel()), generator=g, device=dev, dtype=torch.float64)
    pos = torch.stack([(ix + jit[0]) * h, (iy + jit[1]) * h, (iz + jit[2]) * h]).to(torch.float32)
    pos.clamp_(max=float(np.nextafter(np.float32(BOX), np.float32(0))))
    shape = -amp_a * bf.tij[:, cells]
    z = torch.randn((5, cells.numel()), generator=g, device=dev, dtype=torch.float32) * (math.sqrt(2.0) * sigma_noise)
    r2, r6 = math.sqrt(2.0), math.sqrt(6.0)
    # TENSOR_ORDER xx, yy, zz, xy, xz, yz
    shape[0] += z[0] / r2 + z[1] / r6
    shape[1] += -z[0] / r2 + z[1] / r6
    shape[2] += -2.0 * z[1] / r6
    shape[3] += z[2] / r2
    shape[4] += z[3] / r2
    shape[5] += z[4] / r2
    return Mock(seed, n, int(cells.numel()), pos.contiguous(), shape.contiguous())


def make_mocks(n_mocks: int = 64, counts=(500_000, 4_000_000), grids=(256, 512), n_base: int = 4,
               n_field: int = 128, device="cuda", seed0: int = 1):
    """n_mocks mocks with seeds seed0.. and counts uniform in `counts`; mock j uses grid
    grids[j % len(grids)] and base field j % n_base."""
    rng = np.random.default_rng(seed0)
    want = rng.integers(counts[0], counts[1] + 1, n_mocks)
    bases = [base_field(seed0 + b, n_field, device) for b in range(n_base)]
    return [sample_mock(bases[j % n_base], int(want[j]), seed0 + j, grids[j % len(grids)]) for j in range(n_mocks)]


def k_edges(n: int):
    """40 linear shells to k = 0.4 h/Mpc on the production grids, 20 to 0.8 k_Nyquist otherwise."""
    return K_EDGES[n] if n in K_EDGES else S.linear_edges(0.0, 0.8 * math.pi * n / BOX, 20)


def plan_for(n: int, max_shapes: int, batch: int, precision=L.LPP_FP32, device=None, stream=None,
             fused_slots: int = 0) -> L.Plan:
    return L.Plan(n, BOX, k_edges(n), observer=OBSERVER, scheme=L.LPP_TSC,
                  interlace=True, precision=precision, max_shapes=max_shapes, batch=batch, device=device,
                  stream=stream, fused_slots=fused_slots)


@dataclass
class Tuning:
    n: int
    batch: int
    fused_slots: int = 0
    ms: dict = field(default_factory=dict)      # "grids/slots" -> ms per estimate


def _cache_key(mock: Mock, candidates, slot_modes) -> str:
    """The tuning's identity: the grid, the sample's size to two significant digits, the
    searched shapes and the device."""
    import torch
    dev = torch.cuda.get_device_name(mock.pos.device) if torch.cuda.is_available() else "cpu"
    count = float(f"{mock.count:.2g}")
    return json.dumps([mock.n, count, list(candidates), list(slot_modes), dev])


def autotune(mock: Mock, candidates=(4, 6, 8, 16), slot_modes=(0, 1), repeats: int = 2,
             cache: str | None = None, tuner=None) -> Tuning:
    """Plan shape for the mock's grid size: grids per pass x the fused pass's channel fields per
    CTA (library choice, or always one), the combination with the shortest estimate, timed by
    the library's own kernel timers on the sample mock.  cache (default: the LPP_AUTOTUNE_CACHE
    environment variable) names a JSON file of earlier tunings: a tuning found there for the
    same key (_cache_key) is returned without timing, a new one is added to it.  tuner: the
    timing function (default _tune)."""
    cache = cache if cache is not None else os.environ.get("LPP_AUTOTUNE_CACHE") or None
    tuner = tuner or _tune
    if cache is None:
        return tuner(mock, candidates, slot_modes, repeats)
    key = _cache_key(mock, candidates, slot_modes)
    table = {}
    if os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        t = table[key]
        return Tuning(mock.n, int(t["batch"]), int(t["fused_slots"]), dict(t.get("ms", {})))
    res = tuner(mock, candidates, slot_modes, repeats)
    table[key] = {"batch": res.batch, "fused_slots": res.fused_slots, "ms": res.ms}
    tmp = cache + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1)
    os.replace(tmp, cache)
    return res


def _tune(mock: Mock, candidates, slot_modes, repeats: int) -> Tuning:
    import torch
    res = Tuning(mock.n, candidates[0])
    best = None
    for c in candidates:
        for fs in slot_modes:
            try:
                plan = plan_for(mock.n, mock.count, c, device=mock.pos.device, fused_slots=fs)
            except (L.LppError, torch.OutOfMemoryError):
                continue
            plan.assign(L.LPP_SHAPES, mock.pos, None, None, mock.shape, L.LPP_SHAPE_TENSOR6)
            plan.multipoles()
            plan.set_timing(True)
            ms = []
            for _ in range(repeats):
                plan.multipoles()
                ms.append(sum(v["ms"] for v in plan.kernel_stats().values()))
            plan.set_timing(False)
            res.ms[f"{c}/{fs}"] = min(ms)
            if best is None or min(ms) < best:
                best, res.batch, res.fused_slots = min(ms), c, fs
            del plan
            torch.cuda.empty_cache()
    return res


class BatchRun:
    """Plans (slots_per_grid per grid size, tuned batch) and the captured batch of mocks."""

    def __init__(self, mocks, tuning: dict, slots_per_grid: dict | None = None, use_graph: bool = True):
        slots_per_grid = slots_per_grid or {}
        self.mocks = mocks
        self.plans, self.plan_of = [], []
        by_grid = {}
        for m in mocks:
            by_grid.setdefault(m.n, []).append(m)
        slot_index = {}
        for n, ms in sorted(by_grid.items()):
            k = max(1, int(slots_per_grid.get(n, 1)))
            cap = max(m.count for m in ms)
            slot_index[n] = []
            for _ in range(k):
                slot_index[n].append(len(self.plans))
                t = tuning.get(n)
                self.plans.append(plan_for(n, cap, t.batch if t else 8, device=ms[0].pos.device,
                                           fused_slots=t.fused_slots if t else 0))
        seen = {n: 0 for n in by_grid}
        # mocks of a grid size go round-robin over its slots
        for m in mocks:
            sl = slot_index[m.n]
            self.plan_of.append(sl[seen[m.n] % len(sl)])
            seen[m.n] += 1
        shapes = [self.plans[self.plan_of[j]].particles(L.LPP_SHAPES, m.pos, None, None, m.shape,
                                                        L.LPP_SHAPE_TENSOR6) for j, m in enumerate(mocks)]
        self.batch = L.Batch(self.plans, self.plan_of, shapes, None, use_graph=use_graph,
                             keep=[(m.pos, m.shape) for m in mocks])

    def run(self, stream=None):
        self.batch.launch(stream)
        return self.batch.results()

    def close(self):
        self.batch.close()
        self.plans.clear()


# ------------------------------------------------------------------ persisted results
def _result_name(mock: Mock) -> str:
    return f"mock_{mock.seed}_n{mock.n}_c{mock.count}.npz"


def save_estimate(path: str, est: L.Estimate):
    """One mock's estimate (FP64 rows, shells and normalisations) to an .npz file, written to
    a temporary name and moved into place, so a file that exists is complete."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, p=est.p, raw=est.raw, k_mean=est.k_mean, n_modes=est.n_modes,
             scalars=np.array([est.norm_auto, est.norm_cross, est.norm_dd, est.shot_plus, est.shot_dd, est.alpha]))
    os.replace(tmp, path)


def load_estimate(path: str) -> L.Estimate:
    with np.load(path) as z:
        sc = z["scalars"]
        return L.Estimate(z["p"], z["raw"], z["k_mean"], z["n_modes"], *[float(v) for v in sc])


def run_resumable(mocks, tuning: dict, out_dir: str, chunk: int = 16, slots_per_grid: dict | None = None,
                  use_graph: bool = True, runner=None):
    """The estimates of every mock (in the order of mocks), persisted per mock in out_dir as they
    complete: mocks whose result file exists are read back instead of run (a rerun after an
    interruption skips the finished seeds); the others run in batches of `chunk` mocks (one
    lpp_batch launch each), and each batch's results are written before the next starts, so an
    interruption loses at most one batch.  runner(mocks) -> estimates replaces the batch
    executor (default: BatchRun with the tuning)."""
    os.makedirs(out_dir, exist_ok=True)

    def default_runner(ms):
        run = BatchRun(ms, tuning, slots_per_grid, use_graph=use_graph)
        try:
            return run.run()
        finally:
            run.close()

    runner = runner or default_runner
    paths = [os.path.join(out_dir, _result_name(m)) for m in mocks]
    todo = [j for j, p in enumerate(paths) if not os.path.exists(p)]
    for c0 in range(0, len(todo), max(1, chunk)):
        part = todo[c0:c0 + max(1, chunk)]
        ests = runner([mocks[j] for j in part])
        for j, est in zip(part, ests):
            save_estimate(paths[j], est)
    return [load_estimate(p) for p in paths]
