"""Benchmark of the LPP projected-tensor multipole estimator on GB300.

One step = one complete estimate (sky frames, shears and harmonic weights; CIC/TSC
assignment with interlacing; 3D FFTs; k-space contraction; FP64 shell sums;
normalisation and shot noise) of the polar-cap survey workload: 512^3 grid, L = 4000
Mpc/h, 1.5M shape galaxies, 15M randoms, TSC + interlacing, FP32 grids / FP64 sums,
all ten moment slots (cross L=2,4,6; plus l=0,2,4; minus L=4,6,8; density monopole).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lpp|reference]

Prints one JSON line (rank 0).  Under torchrun each rank times an independent mock
(seed + rank) of the same size: the path shards by catalogue with no exchange.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LPP tensor-multipole estimates/sec at 512^3; templates/sec surrogate vs plain"
# instruction issue peak of the GB300: 152 SMs x 4 warp schedulers x 1 warp instruction per
# cycle x 2070 MHz (the maximum SM clock)
ISSUE_PEAK_WARP_INSTR_S = 152 * 4 * 1.0 * 2070e6
UNIT = "estimates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lpp", choices=["lpp", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--data", type=int, default=1_500_000)
    ap.add_argument("--randoms", type=int, default=15_000_000)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--moment-mask", type=int, default=-1,
                    help="bit mask of moment slots (default: all ten); smaller cases for profiling")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP32-vs-FP64 error of the timed estimate")
    ap.add_argument("--shard", action="store_true",
                    help="time one estimate split by moment slot over the ranks (strong scaling)")
    ap.add_argument("--batch-mocks", type=int, default=64)
    return ap.parse_args()


def replica_throughput(elapsed, steps: int, world: int, pg=None, device=None):
    """Whole-job throughput of `world` independent replicas that each ran `steps` steps in
    `elapsed` (any time unit): the slowest rank's time (max over ranks through `pg`) bounds
    the job, and every rank's steps count.  Returns (units per elapsed unit, max elapsed)."""
    if pg is not None and world > 1:
        import torch
        t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed = float(t.item())
    return world * steps / elapsed, elapsed


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, seed):
    from paper_2202_11839_gb300 import synthetic as S
    return S.workload_survey(n_data=args.data, n_rand=args.randoms, n=args.n, seed=seed)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region; the raw
    CSV goes to $LPP_CLOCKS_DIR (default: the system temporary directory)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("LPP_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"lpp_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle timing
def _oracle_slot_task(task):
    """One moment slot of the oracle's estimate (a pool task): returns its seconds."""
    cfg, cat, moments = task
    from oracle import lpp_oracle as O
    plan = O.Plan(n=cfg["n"], box=cfg["box"], origin=cfg["origin"], observer=cfg["observer"], pole=cfg["pole"],
                  scheme=3, interlace=True, k_edges=cfg["k_edges"], cross_b=True, moments=moments)
    t0 = time.perf_counter()
    O.multipoles(plan, cat["pos"], None, cat["shape"], None, None, None, cat["rpos"], None, cat["rnbar"])
    return time.perf_counter() - t0


class OracleTimer:
    """The FP64 oracle as it stands, timed on the host cores on a bounded sample of the workload.

    Sample: one complete oracle estimate (all ten moment slots, cross E and B parts, TSC +
    interlacing, the randoms) on an ns^3 grid over the same box, with the first
    count (ns/n)^3 shape galaxies and randoms (the same particles per cell).  The oracle's
    cost is dominated by its field transforms, so the time is scaled to the n^3 grid by
    (n/ns)^3 log(n^3)/log(ns^3) (an extrapolation, stated in the sample text).  With
    workers > 1 the ten slots run as separate processes of a spawn pool (each recomputes the
    partner fields, as the oracle does for one slot) and the wall time of the whole set is
    taken; the pool is created before any GPU work and warmed before timing."""

    def __init__(self, wl, ns: int = 64, workers: int = 1):
        import multiprocessing as mp
        self.wl, self.ns = wl, ns
        ratio = (wl.n / ns) ** 3
        shp, rnd = wl.shapes, wl.randoms
        m, mr = max(1, int(shp.count / ratio)), max(1, int(rnd.count / ratio)) if rnd is not None else 0
        self.counts = (m, mr)
        self.cat = dict(pos=shp.pos[:, :m].astype(np.float64), shape=shp.shape[:, :m].astype(np.float64),
                        rpos=rnd.pos[:, :mr].astype(np.float64), rnbar=rnd.nbar[:mr].astype(np.float64))
        self.cfg = dict(n=ns, box=wl.box, origin=wl.origin, observer=wl.observer, pole=wl.pole,
                        k_edges=np.asarray(wl.k_edges))
        self.scale = ratio * math.log(wl.n ** 3) / math.log(ns ** 3)
        self.workers = max(1, min(workers, 10))
        self.pool = None
        if self.workers > 1:
            self.pool = mp.get_context("spawn").Pool(self.workers)
            self.pool.map(abs, range(self.workers))   # start the workers before timing

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def sample(self):
        """One timed sample: (estimates/s scaled to the workload, wall seconds, description)."""
        from oracle import lpp_oracle as O
        t0 = time.perf_counter()
        if self.pool is None:
            _oracle_slot_task((self.cfg, self.cat, tuple(O.DEFAULT_MOMENTS)))
        else:
            self.pool.map(_oracle_slot_task, [(self.cfg, self.cat, (mom,)) for mom in O.DEFAULT_MOMENTS], chunksize=1)
        wall = time.perf_counter() - t0
        wl = self.wl
        desc = (f"one complete oracle estimate (ten slots, cross E+B, TSC+interlacing) on a {self.ns}^3 grid over "
                f"the same box with {self.counts[0]} of {wl.shapes.count} shape galaxies and {self.counts[1]} of "
                f"{wl.randoms.count} randoms ({wall:.2f} s wall on {self.workers} process"
                f"{'es, one per moment slot' if self.workers > 1 else ''}), extrapolated to {wl.n}^3 by "
                f"(n/ns)^3 log(n^3)/log(ns^3) = {self.scale:.0f} (numpy/pocketfft, one thread per process)")
        return 1.0 / (wall * self.scale), wall, desc


def cpu_baseline_leg(wl, steps: int = 1):
    """The oracle on all host cores (nproc, moment-parallel) and on one core."""
    nproc = os.cpu_count() or 1
    out = {}
    for key, workers in (("all", nproc), ("one", 1)):
        tmr = OracleTimer(wl, workers=workers)
        vals, desc = [], ""
        for _ in range(steps):
            v, _, desc = tmr.sample()
            vals.append(v)
        tmr.close()
        out[key] = {"value": statistics.median(vals), "cores": tmr.workers, "sample": desc}
    a, o = out["all"], out["one"]
    return {"value": a["value"], "unit": UNIT, "cores": a["cores"], "nproc": nproc, "kind": "oracle",
            "sample": a["sample"], "single_core": {"value": o["value"], "unit": UNIT, "cores": 1,
                                                   "sample": o["sample"]}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args, seed=0)
    nproc = os.cpu_count() or 1
    tmr = OracleTimer(wl, workers=nproc)
    vals, desc = [], ""
    for i in range(args.warmup + args.steps):
        v, w, desc = tmr.sample()
        if i >= args.warmup:
            vals.append(v)
    tmr.close()
    v = statistics.median(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "box": wl.box, "shape_galaxies": wl.shapes.count,
                   "randoms": wl.randoms.count if wl.randoms is not None else 0, "scheme": "tsc", "interlace": True},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": tmr.workers, "nproc": nproc, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------- GPU arm
def padded_window(wl, d_pos, d_rpos, d_rnbar, dev, s_edges):
    """Q_l(s) of the survey's randoms on a grid of twice the box, shifted by half a box, so that
    no separation up to the last shell wraps around (the estimate's own grid is periodic with
    the survey's box, shorter than its extent plus 3800 Mpc/h): 512^3 over 8000 Mpc/h
    (h = 15.6 Mpc/h).  The data catalogue is assigned for alpha (the normalisation I)."""
    from paper_2202_11839_gb300 import lpp as L
    origin = tuple(o - wl.box / 2 for o in wl.origin)
    wp = L.Plan(wl.n, 2 * wl.box, np.linspace(0.0, 0.01, 2), origin=origin, observer=wl.observer, pole=wl.pole,
                scheme=L.LPP_TSC, interlace=False, compensate=True, precision=L.LPP_FP32,
                moments=1 << L.LPP_MOM_DD0, max_density=int(d_pos.shape[1]), max_randoms=int(d_rpos.shape[1]),
                device=dev)
    wp.assign(L.LPP_DENSITY, d_pos)
    wp.assign(L.LPP_RANDOMS, d_rpos, None, d_rnbar)
    out = wp.window_q(s_edges)
    wp.close()
    return out


def template_leg(plan, est, wl, dev, d_pos, d_rpos, d_rnbar):
    """Window-convolved templates for the survey: Q_l(s) from its randoms (on a padded grid),
    then templates/s of the FFTLog path and of the trained surrogate (20k Latin-hypercube
    training templates), and the surrogate's error on 2k held-out parameter sets in Gaussian
    error bars."""
    import torch

    from paper_2202_11839_gb300 import lpp as L
    from paper_2202_11839_gb300 import surrogate as SG
    from paper_2202_11839_gb300 import synthetic as S
    s_edges = np.linspace(0.0, 3800.0, 191)
    q, s_mean, npts, _ = padded_window(wl, d_pos, d_rpos, d_rnbar, dev, s_edges)
    torch.cuda.empty_cache()
    keep = npts > 0
    tm = L.Template(q[:, keep], s_mean[keep], wl.k_edges, shot_plus=est.shot_plus, stream=plan.stream, device=dev)
    em = SG.Emulator(tm, SG.survey_volume(), est.shot_dd)
    em.train()
    rep = em.evaluate(em.cfg.n_test, seed=77)
    net = em.inference_net(8192)
    th = torch.from_numpy(S.latin_hypercube(8192, seed=78)).to(dev)
    rates = {}
    for name, fn in (("plain", em.plain), ("surrogate", net.predict)):
        for _ in range(3):
            fn(th)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(plan.stream)
        for _ in range(5):
            fn(th)
        e1.record(plan.stream)
        torch.cuda.synchronize()
        rates[name] = 5 * 8192 / (e0.elapsed_time(e1) / 1000.0)
    out = {"unit": "templates/s", "plain": rates["plain"], "surrogate": rates["surrogate"],
           "speedup": rates["surrogate"] / rates["plain"], "batch": 8192,
           "error_sigma": {"rms": rep.rms_sigma, "p99": rep.p99_sigma, "max": rep.max_sigma},
           "baseline_only_sigma": {"rms": rep.baseline_rms_sigma, "max": rep.baseline_max_sigma},
           "n_train": em.cfg.n_train, "n_test": em.cfg.n_test, "train_s": rep.train_seconds,
           "data_s": rep.data_seconds, "outputs": "gE_0,2 EE_0,2,4 BB_0,2,4 x 40 shells",
           "window": "Q_l(s) of the survey randoms, 512^3 over a padded 8000 Mpc/h box (no wrap-around)",
           "dtype": "bf16 network, f64 FFTLog"}
    net.close()
    em.net.close()
    tm.close()
    return out


def batch_leg(args, dev, steps: int):
    """64 periodic tidal mocks of 0.5M-4M galaxies on mixed 256^3 / 512^3 grids in one CUDA
    graph launch per step; estimates/s and the FP32 path's per-multipole error against the
    FP64 path (which matches the FP64 oracle to 1e-10 in the tests) for one mock per grid."""
    import torch

    from paper_2202_11839_gb300 import batch as B
    from paper_2202_11839_gb300 import lpp as L
    t0 = time.perf_counter()
    mocks = B.make_mocks(args.batch_mocks, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    grids = sorted({m.n for m in mocks})
    tuning = {n: B.autotune(max((m for m in mocks if m.n == n), key=lambda m: m.count)) for n in grids}
    torch.cuda.empty_cache()
    slots = {n: (2 if n < 512 else 1) for n in grids}
    run = B.BatchRun(mocks, tuning, slots_per_grid=slots, use_graph=True)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        run.run(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run.batch.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res = run.batch.results()
    # FP64 check of one mock per grid size
    errs = {}
    for n in grids:
        j = next(i for i, m in enumerate(mocks) if m.n == n)
        m = mocks[j]
        p64 = B.plan_for(n, m.count, 8, precision=L.LPP_FP64, device=dev)
        p64.assign(L.LPP_SHAPES, m.pos.double().contiguous(), None, None, m.shape.double().contiguous(),
                   L.LPP_SHAPE_TENSOR6)
        ref = p64.multipoles()
        del p64
        torch.cuda.empty_cache()
        e = slot_errors(res[j].p, ref)
        errs[f"{n}^3"] = {f"{k}{l}": float(v) for (k, l), v in zip(MOMENT_NAMES[:10], e)}
    counts = [m.count for m in mocks]
    out = {"value": len(mocks) * steps / (ms / 1000.0), "unit": "estimates/s", "mocks": len(mocks),
           "grids": {f"{n}^3": sum(1 for m in mocks if m.n == n) for n in grids},
           "galaxies": {"min": int(min(counts)), "max": int(max(counts)), "total": int(sum(counts))},
           "ms_per_batch": ms / steps, "steps": steps, "graph": True,
           "plans": {f"{n}^3": {"slots": slots[n], "grids_per_pass": tuning[n].batch,
                                "fused_slots": tuning[n].fused_slots,
                                "autotune_ms (grids/fused_slots)": {str(k): round(v, 2) for k, v in tuning[n].ms.items()}}
                     for n in grids},
           "error_vs_fp64": errs, "mock_generation_s": gen_s}
    run.close()
    del mocks
    torch.cuda.empty_cache()
    return out


MOMENT_NAMES = [("dd", 0), ("cross", 2), ("cross", 4), ("cross", 6), ("plus", 0), ("plus", 2), ("plus", 4),
                ("minus", 4), ("minus", 6), ("minus", 8), ("dd", 2), ("dd", 4)]


def slot_errors(p, ref):
    """Per moment slot: max over shells of |p - ref.p| / (|ref.p| + sqrt(P_+^(0) P_dd^(0))), the
    monopoles taken before shot-noise subtraction (the error scale of the parity tests)."""
    pp = np.abs(ref.raw[4].real) / max(ref.norm_auto, 1e-300)
    pd = np.abs(ref.raw[0].real) / max(ref.norm_dd, 1e-300)
    sc = np.abs(ref.p) + np.sqrt(pp * pd)[None, :]
    sc = np.where(sc > 0, sc, 1.0)
    return (np.abs(p - ref.p) / sc).max(axis=1)


def precision_leg(wl, est, common, dev):
    """The timed FP32 estimate against the FP64 path on the same catalogues (positions, shapes
    and n-bar of the FP32 run, widened): per moment slot, the largest error over the shells
    in units of the parity tests' scale.  The FP64 path matches the FP64 oracle to 1e-10 in
    the tests, and the FP32 path of this grid and configuration is compared with the oracle
    directly at 512^3 (tests/test_gpu_survey_fullsize.py)."""
    import torch

    from paper_2202_11839_gb300 import lpp as L
    shp, rnd = wl.shapes, wl.randoms
    td = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32), dtype=np.float64)).to(dev)
    c64 = dict(common, precision=L.LPP_FP64, batch=0)
    t0 = time.perf_counter()
    p64 = L.Plan(wl.n, wl.box, wl.k_edges, **c64)
    pos, shape, rpos, rnbar = td(shp.pos), td(shp.shape), td(rnd.pos), td(rnd.nbar)
    p64.assign(L.LPP_SHAPES, pos, None, None, shape, L.LPP_SHAPE_TENSOR6)
    p64.assign(L.LPP_RANDOMS, rpos, None, rnbar)
    ref = p64.multipoles()
    p64.close()
    del p64, pos, shape, rpos, rnbar
    torch.cuda.empty_cache()
    e = slot_errors(est.p, ref)
    return {"error_vs_fp64": {f"{k}{l}": float(v) for (k, l), v in zip(MOMENT_NAMES, e)
                              if common["moments"] & (1 << MOMENT_NAMES.index((k, l)))},
            "scale": "|P_fp64| + sqrt(P_+^(0) P_dd^(0)) per shell, max over the shells",
            "fp64_estimate_s": time.perf_counter() - t0}


def run_lpp(args):
    import torch

    from paper_2202_11839_gb300 import lpp as L
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    L.load_library()
    wl = workload(args, seed=rank)
    shp, rnd = wl.shapes, wl.randoms
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    d_pos, d_shape, d_rpos, d_rnbar = tt(shp.pos), tt(shp.shape), tt(rnd.pos), tt(rnd.nbar)
    moments = L.LPP_WANT_ALL if args.moment_mask < 0 else args.moment_mask
    common = dict(origin=wl.origin, observer=wl.observer, pole=wl.pole, scheme=L.LPP_TSC, interlace=True,
                  compensate=True, precision=L.LPP_FP32, moments=moments, max_shapes=shp.count,
                  max_randoms=rnd.count, batch=args.batch)
    plan = L.Plan(wl.n, wl.box, wl.k_edges, **common)
    plan.assign(L.LPP_SHAPES, d_pos, None, None, d_shape, L.LPP_SHAPE_TENSOR6)
    plan.assign(L.LPP_RANDOMS, d_rpos, None, d_rnbar)
    stream = plan.stream
    for _ in range(args.warmup):
        est = plan.multipoles()
    assert np.all(np.isfinite(est.p)), "non-finite estimate"
    plan.set_timing(True)
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = {k: {"ms": 0.0, "launches": 0, "bytes": 0.0} for k in L.KERNEL_KINDS}
    launches = 0
    for _ in range(args.steps):
        est = plan.multipoles()
        launches += plan.launch_count()
        for k, v in plan.kernel_stats().items():
            for f in ("ms", "launches", "bytes"):
                stats[k][f] += v[f]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    value, ms = replica_throughput(ms / 1000.0, args.steps, world, pg, dev)
    ms *= 1000.0
    plan.set_timing(False)
    n_fields = plan.field_count()

    # dominant kernel and its roofline
    hbm, peak_src = measured_peaks()
    dom = max((k for k in stats if k != "other"), key=lambda k: stats[k]["ms"])
    d = stats[dom]
    avg_s = d["ms"] / max(d["launches"], 1) / 1000.0
    bytes_per_launch = d["bytes"] / max(d["launches"], 1)
    achieved = bytes_per_launch / avg_s / 1e9 if avg_s > 0 else 0.0
    kern = {k: {"ms_per_step": round(v["ms"] / args.steps, 3), "launches_per_step": v["launches"] // args.steps,
                "gbs": round(v["bytes"] / (v["ms"] / 1000.0) / 1e9, 1) if v["ms"] > 0 else None}
            for k, v in stats.items()}

    templates = None
    if rank == 0 and not args.no_surrogate:
        templates = template_leg(plan, est, wl, dev, d_pos, d_rpos, d_rnbar)
    precision = None
    if rank == 0 and not args.no_fp64:
        precision = precision_leg(wl, est, common, dev)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        del plan
        torch.cuda.empty_cache()
        hplan = L.Plan(wl.n, wl.box, wl.k_edges, host_inputs=True, **common)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory().numpy()
        h_pos, h_shape, h_rpos, h_rnbar = pin(shp.pos), pin(shp.shape), pin(rnd.pos), pin(rnd.nbar)
        h2d = (h_pos.nbytes + h_shape.nbytes + h_rpos.nbytes + h_rnbar.nbytes)
        # FP64 shell sums of every channel and the two partner monopoles, the sums and the error flag
        d2h = (n_fields - 1) * (len(wl.k_edges) - 1) * 2 * 8 + 8 * 8 + 4
        for _ in range(1):
            hplan.assign(L.LPP_SHAPES, h_pos, None, None, h_shape, L.LPP_SHAPE_TENSOR6)
            hplan.assign(L.LPP_RANDOMS, h_rpos, None, h_rnbar)
            hplan.multipoles()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hplan.assign(L.LPP_SHAPES, h_pos, None, None, h_shape, L.LPP_SHAPE_TENSOR6)
            hplan.assign(L.LPP_RANDOMS, h_rpos, None, h_rnbar)
            hplan.multipoles()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        ev, te = replica_throughput(te, args.steps, world, pg, dev)
        e2e = {"value": ev, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        del hplan

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    batched = None
    if not args.no_batch:
        batched = batch_leg(args, dev, max(1, min(args.steps, 3)))
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline_leg(wl)
    # measured DRAM bytes per launch of the dominant kernel kind (profiles/traffic.json), for the
    # default full-size configuration only (the figures were taken for it)
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    default_cfg = (args.n == 512 and args.data == 1_500_000 and args.randoms == 15_000_000 and args.batch == 0
                   and args.moment_mask < 0)
    tr = {}
    if default_cfg and os.path.exists(prof):
        with open(prof) as f:
            tr = json.load(f)
        if tr.get("workload") == wl.name:
            traffic = tr.get("kernels", {}).get(dom, {}).get("bytes_per_launch")
    # the same roofline figures for every kernel kind (the two largest, the fused assignment
    # and the passes, take nearly equal time, so the dominant one can change between runs)
    kinds_roof = {}
    for k, v in stats.items():
        if k == "other" or v["launches"] == 0 or v["ms"] <= 0:
            continue
        t_s = v["ms"] / v["launches"] / 1000.0
        b_l = v["bytes"] / v["launches"]
        tk = None
        if tr.get("workload") == wl.name:
            tk = tr.get("kernels", {}).get(k, {}).get("bytes_per_launch")
        kinds_roof[k] = {"achieved": round(b_l / t_s / 1e9, 1), "frac": round(b_l / t_s / 1e9 / hbm, 4),
                         "bytes_per_launch": b_l, "avg_launch_ms": round(t_s * 1000.0, 4), "traffic": tk}
        # issue-rate roofline of the instruction-bound kinds: warp instructions per launch (ncu,
        # profiles/traffic.json) over the launch's event time, against 152 SMs x 4 schedulers x
        # one warp instruction per cycle at the maximum SM clock
        wi = tr.get("kernels", {}).get(k, {}).get("warp_instructions_per_launch") if tr.get("workload") == wl.name else None
        if wi:
            peak_issue = ISSUE_PEAK_WARP_INSTR_S
            kinds_roof[k]["issue"] = {"achieved": round(wi / t_s / 1e12, 4), "peak": round(peak_issue / 1e12, 4),
                                      "unit": "T warp-instr/s", "frac": round(wi / t_s / peak_issue, 4),
                                      "warp_instructions_per_launch": wi}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n, "box": wl.box, "shape_galaxies": shp.count,
                   "randoms": rnd.count, "scheme": "tsc", "interlace": True, "fields": n_fields,
                   "k_bins": len(wl.k_edges) - 1, "k_max": float(wl.k_edges[-1]),
                   "l2": "inputs larger than L2 (each grid 1 GiB)", "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_src, "traffic": traffic,
                     "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_s * 1000.0,
                     "kinds": kinds_roof},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "kernels": kern,
        "templates": templates,
        "precision": precision,
        "batched": batched,
    }
    print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


def run_shard(args):
    """One estimate of the survey workload split by moment slot over the ranks (every rank
    recomputes the partner fields, computes its slots' channels, then one sum all-reduce of
    the FP64 rows and one max all-reduce of the shell data over NCCL): strong scaling, one
    estimate per step for the whole job."""
    import torch

    from paper_2202_11839_gb300 import lpp as L
    from paper_2202_11839_gb300 import shard as SH
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    L.load_library()
    wl = workload(args, seed=0)
    shp, rnd = wl.shapes, wl.randoms
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    d_pos, d_shape, d_rpos, d_rnbar = tt(shp.pos), tt(shp.shape), tt(rnd.pos), tt(rnd.nbar)
    moments = L.LPP_WANT_ALL if args.moment_mask < 0 else args.moment_mask
    mask = SH.partition(moments, world)[rank]
    plan = None
    if mask:
        plan = L.Plan(wl.n, wl.box, wl.k_edges, origin=wl.origin, observer=wl.observer, pole=wl.pole,
                      scheme=L.LPP_TSC, interlace=True, precision=L.LPP_FP32, moments=mask, max_shapes=shp.count,
                      max_randoms=rnd.count, batch=args.batch)
        plan.assign(L.LPP_SHAPES, d_pos, None, None, d_shape, L.LPP_SHAPE_TENSOR6)
        plan.assign(L.LPP_RANDOMS, d_rpos, None, d_rnbar)

    def step():
        est = plan.multipoles() if plan is not None else None
        return SH.gather(est, mask, pg, dev)

    for _ in range(args.warmup):
        out = step()
    assert np.all(np.isfinite(out.p)), "non-finite estimate"
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = step()
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    clk = clocks.stop()
    if pg:
        t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed = float(t.item())
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": args.steps / elapsed, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "shape_galaxies": shp.count, "randoms": rnd.count,
                       "parallelism": f"moment-slot shards x{world}", "masks": SH.partition(moments, world),
                       "l2": "inputs larger than L2 (each grid 1 GiB)"},
            "timing": "host wall clock around the steps, a device synchronisation on both sides (the gather "
                      "copies the rows to the host every step)",
            "clocks": clk}), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_shard(args)
    else:
        run_lpp(args)


if __name__ == "__main__":
    main()
