"""Host logic of the JSON plan configurations, the autotuner's cache and the resumable batch
results (no GPU: fake tuners and runners stand in for the timed plans and the batch)."""
import json
import math
import os

import numpy as np
import pytest


def _mods():
    from paper_2202_11839_gb300 import batch as B
    from paper_2202_11839_gb300 import config as CF
    from paper_2202_11839_gb300 import lpp as L
    return L, CF, B


@pytest.mark.parametrize("name,ctor", [("survey_cap_L4000_N512_tsc_il", "workload_survey"),
                                       ("periodic_L2000_N256_tsc_il", "workload_periodic_tsc"),
                                       ("periodic_L500_N64_cic_fp64", "workload_periodic_fp64")])
def test_configs_describe_the_workloads(name, ctor):
    """Each configuration under configs/ gives the plan its synthetic workload is measured
    with: grid, box, origin, observer, pole, scheme, interlacing and the shells exactly."""
    L, CF, B = _mods()
    from paper_2202_11839_gb300 import synthetic as S
    import inspect
    wl_fn = getattr(S, ctor)
    cfg = CF.load(name)
    n, box, e, kw = CF.plan_args(cfg)
    # the workload's plan geometry without generating its catalogues: the defaults of its
    # constructor and the fixed fields of the Workload it returns
    src = inspect.getsource(wl_fn)
    assert f'"{name}"' in src
    sig = inspect.signature(wl_fn).parameters
    assert n == sig["n"].default and box == sig["box"].default
    assert kw["scheme"] == (L.LPP_TSC if "tsc" in name else L.LPP_CIC)
    assert kw["interlace"] == ("_il" in name)
    assert kw["moments"] == L.LPP_WANT_ALL
    if ctor == "workload_survey":
        assert kw["observer"] == (box / 2, box / 2, 200.0)
        np.testing.assert_array_equal(e, S.linear_edges(0.0, 0.2, 40))
    elif ctor == "workload_periodic_tsc":
        assert kw["observer"] == (box / 2, box / 2, box / 2 - 4000.0)
        np.testing.assert_array_equal(e, S.linear_edges(0.0, 0.4, 40))
    else:
        np.testing.assert_allclose(e, S.linear_edges(0.0, math.pi * n / box, 20), rtol=1e-15, atol=0)
        assert kw["precision"] == L.LPP_FP64


def test_config_fields_and_errors():
    L, CF, B = _mods()
    assert CF.moment_mask(["dd0", "cross2", "cross_b"]) == 0b11 | L.LPP_WANT_CROSS_B
    assert CF.moment_mask("all") == L.LPP_WANT_ALL
    assert CF.moment_mask(["minus10", "minus12"]) == L.LPP_WANT_MINUS_HIGH
    with pytest.raises(ValueError):
        CF.moment_mask(["quadrupole"])
    with pytest.raises(ValueError):
        CF.plan_args({"n": 64, "box": 100.0, "k_edges": [0, 1], "grid": 3})
    with pytest.raises(ValueError):
        CF.plan_args({"n": 64, "box": 100.0, "k_edges": [0.2, 0.1]})
    n, box, e, kw = CF.plan_args({"n": 32, "box": 100.0, "k_edges": {"lo": 0.0, "hi": 1.0, "n": 4},
                                  "los_est": "global", "los_global": [0, 0, 1], "batch": 3})
    assert (n, box, kw["los_est"], kw["batch"]) == (32, 100.0, L.LPP_LOS_GLOBAL, 3)
    np.testing.assert_array_equal(e, [0.0, 0.25, 0.5, 0.75, 1.0])


class _FakeMock:
    def __init__(self, seed, n, count):
        import torch
        self.seed, self.n, self.count = seed, n, count
        self.pos = torch.zeros(3, 1)
        self.shape = torch.zeros(6, 1)


def test_autotune_cache(tmp_path):
    """A tuning is timed once per key and read back from the cache file afterwards; another
    grid size or sample size is a new key."""
    L, CF, B = _mods()
    calls = []

    def tuner(mock, candidates, slot_modes, repeats):
        calls.append(mock.n)
        return B.Tuning(mock.n, 6, 1, {"6/1": 1.5})

    cache = str(tmp_path / "tune.json")
    a = B.autotune(_FakeMock(1, 256, 1_000_000), cache=cache, tuner=tuner)
    b = B.autotune(_FakeMock(2, 256, 1_010_000), cache=cache, tuner=tuner)   # same key (2 digits)
    c = B.autotune(_FakeMock(3, 512, 1_000_000), cache=cache, tuner=tuner)
    assert calls == [256, 512]
    assert (a.batch, a.fused_slots) == (b.batch, b.fused_slots) == (6, 1) and c.n == 512
    with open(cache) as f:
        assert len(json.load(f)) == 2
    os.environ.pop("LPP_AUTOTUNE_CACHE", None)
    B.autotune(_FakeMock(4, 256, 1_000_000), tuner=tuner)                    # no cache: times again
    assert calls == [256, 512, 256]


def test_resumable_batch_skips_finished_mocks(tmp_path):
    """run_resumable writes each mock's estimate as its batch completes; a rerun reads them
    back and runs nothing, and after one result file is lost only that mock runs again."""
    L, CF, B = _mods()
    ran = []

    def runner(ms):
        ran.append([m.seed for m in ms])
        out = []
        for m in ms:
            p = np.full((L.LPP_N_MOMENTS, 3), m.seed + 0.5j)
            out.append(L.Estimate(p, 2 * p, np.arange(3.0), np.array([5, 6, 7]), 1.0 * m.seed, 2.0, 3.0, 4.0, 5.0,
                                  0.1 * m.seed))
        return out

    mocks = [_FakeMock(s, 256 if s % 2 else 512, 1000 + s) for s in range(1, 8)]
    out = str(tmp_path / "res")
    first = B.run_resumable(mocks, {}, out, chunk=3, runner=runner)
    assert ran == [[1, 2, 3], [4, 5, 6], [7]]
    second = B.run_resumable(mocks, {}, out, chunk=3, runner=runner)
    assert ran == [[1, 2, 3], [4, 5, 6], [7]]
    for a, b, m in zip(first, second, mocks):
        np.testing.assert_array_equal(a.p, b.p)
        assert a.norm_auto == m.seed and a.alpha == pytest.approx(0.1 * m.seed)
        np.testing.assert_array_equal(a.n_modes, [5, 6, 7])
    os.remove(os.path.join(out, B._result_name(mocks[4])))
    B.run_resumable(mocks, {}, out, chunk=3, runner=runner)
    assert ran[-1] == [5]
