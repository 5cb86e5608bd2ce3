"""The batch executor (lpp_batch_*): many catalogues on mixed grids in one CUDA graph launch,
against single-plan estimates and, in FP64, against the oracle."""
import numpy as np
import pytest

from oracle import lpp_oracle as O
from tests.parity_util import assert_parity, default_edges, run_oracle

pytestmark = pytest.mark.gpu


def _mocks(n_mocks=6, counts=(20_000, 60_000), grids=(32, 64)):
    from paper_2202_11839_gb300 import batch as B
    return B.make_mocks(n_mocks, counts, grids, n_base=2, n_field=32)


def _close(a, b, tol):
    sc = np.abs(b.p).max(axis=1, keepdims=True)
    sc = np.where(sc > 0, sc, 1.0)
    return float((np.abs(a.p - b.p) / sc).max()) <= tol


def test_batch_graph_matches_single_plan_estimates():
    from paper_2202_11839_gb300 import batch as B
    from paper_2202_11839_gb300 import lpp as L
    mocks = _mocks()
    tuning = {32: B.Tuning(32, 4), 64: B.Tuning(64, 8)}
    run = B.BatchRun(mocks, tuning, slots_per_grid={32: 2, 64: 1}, use_graph=True)
    got = run.run()
    again = run.run()                 # a second graph launch gives the same estimates
    for j, m in enumerate(mocks):
        plan = run.plans[run.plan_of[j]]
        plan.assign(L.LPP_SHAPES, m.pos, None, None, m.shape, L.LPP_SHAPE_TENSOR6)
        want = plan.multipoles()
        # FP32 grids with shared-memory atomics: equal to rounding of the accumulation order
        assert _close(got[j], want, 1e-5), j
        assert _close(again[j], got[j], 1e-5), j
        np.testing.assert_array_equal(got[j].n_modes, want.n_modes)
        assert got[j].shot_plus == pytest.approx(want.shot_plus, rel=1e-12)
    run.close()


def test_batch_without_graph_and_new_contents():
    """Without a graph, and after the catalogue contents change in place (same buffers), the
    batch sees the new data: doubling every shape multiplies the shape x shape moments by 4
    and the cross moments by 2."""
    from paper_2202_11839_gb300 import batch as B
    mocks = _mocks(4)
    tuning = {32: B.Tuning(32, 8), 64: B.Tuning(64, 8)}
    run = B.BatchRun(mocks, tuning, use_graph=False)
    first = run.run()
    for m in mocks:
        m.shape.mul_(2.0)
    second = run.run()
    for a, b in zip(first, second):
        for i, (kind, ell) in enumerate(O.DEFAULT_MOMENTS):
            f = {"dd": 1.0, "cross": 2.0}.get(kind, 4.0)
            sc = max(np.abs(a.p[i]).max(), 1e-300)
            assert np.abs(b.p[i] - f * a.p[i]).max() <= 1e-5 * f * sc, (kind, ell)
    run.close()


def test_batch_fp64_matches_oracle():
    """Three FP64 catalogues on two plans (16^3 and 32^3, CIC and TSC) through one graph."""
    import torch
    from paper_2202_11839_gb300 import lpp as L
    from paper_2202_11839_gb300 import synthetic as S
    box = 300.0
    cfgs = [dict(n=16, box=box, observer=(150.0, 150.0, -900.0), scheme=2, interlace=False,
                 k_edges=default_edges(16, box)),
            dict(n=32, box=box, observer=(150.0, 150.0, -900.0), scheme=3, interlace=True,
                 k_edges=default_edges(32, box))]
    cats = []
    for j, count in enumerate((1500, 2500, 900)):
        rng = np.random.default_rng(40 + j)
        cats.append(dict(pos=S.uniform_positions(count, box, (0, 0, 0), 40 + j, 0, np.float64),
                         shape=rng.standard_normal((6, count))))
    plan_of = [0, 1, 0]
    plans = [L.Plan(c["n"], box, c["k_edges"], observer=c["observer"], scheme=c["scheme"], interlace=c["interlace"],
                    precision=L.LPP_FP64, moments=L.LPP_WANT_ALL | L.LPP_WANT_CROSS_B, max_shapes=2500)
             for c in cfgs]
    dev = [(torch.from_numpy(c["pos"]).cuda(), torch.from_numpy(c["shape"]).cuda()) for c in cats]
    parts = [plans[plan_of[j]].particles(L.LPP_SHAPES, dev[j][0], None, None, dev[j][1], L.LPP_SHAPE_TENSOR6)
             for j in range(3)]
    b = L.Batch(plans, plan_of, parts, None, use_graph=True, keep=dev)
    b.launch()
    got = b.results()
    for j in range(3):
        ref = run_oracle(cfgs[plan_of[j]], cats[j])
        assert_parity(got[j], ref, 1e-10, f"mock {j}")
    b.close()


def test_batch_reports_the_failing_mock():
    import torch
    from paper_2202_11839_gb300 import batch as B
    from paper_2202_11839_gb300 import lpp as L
    mocks = _mocks(3)
    mocks[1].pos[0, 5] = 2500.0          # outside the 2000 Mpc/h box
    run = B.BatchRun(mocks, {32: B.Tuning(32, 8), 64: B.Tuning(64, 8)})
    with pytest.raises(L.LppError) as e:
        run.run()
    assert e.value.status == L.LPP_ERR_DOMAIN and "mock 1" in str(e.value)
    run.close()
    torch.cuda.synchronize()


def test_batch_bad_arguments():
    import ctypes as C
    from paper_2202_11839_gb300 import batch as B
    from paper_2202_11839_gb300 import lpp as L
    lib = L.load_library()
    mocks = _mocks(2)
    plan = B.plan_for(32, 100, 8)        # capacity below the mocks' counts
    part = plan.particles(L.LPP_SHAPES, mocks[0].pos, None, None, mocks[0].shape, L.LPP_SHAPE_TENSOR6)
    h = C.c_void_p()
    one = (C.c_void_p * 1)(plan.h.value)
    two = (C.c_void_p * 2)(plan.h.value, plan.h.value)
    po = (C.c_int * 1)(0)
    parts = (L.Particles * 1)(part)
    assert lib.lpp_batch_create(one, 1, po, parts, None, 1, 1, C.byref(h)) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_batch_create(two, 2, po, parts, None, 1, 1, C.byref(h)) == L.LPP_ERR_INVALID_ARG
    bad = (C.c_int * 1)(3)
    assert lib.lpp_batch_create(one, 1, bad, parts, None, 1, 1, C.byref(h)) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_batch_launch(None, None) == L.LPP_ERR_INVALID_ARG


def test_resumable_batch_matches_one_batch(tmp_path):
    """run_resumable (batches of two mocks, each result written as its batch completes) gives
    the estimates of one batch over all mocks; a rerun reads the files back."""
    from paper_2202_11839_gb300 import batch as B
    mocks = _mocks(5)
    tuning = {32: B.Tuning(32, 8), 64: B.Tuning(64, 8)}
    run = B.BatchRun(mocks, tuning)
    whole = run.run()
    run.close()
    out = str(tmp_path / "res")
    parts = B.run_resumable(mocks, tuning, out, chunk=2)
    again = B.run_resumable(mocks, tuning, out, chunk=2, runner=lambda ms: pytest.fail("nothing to rerun"))
    for a, b, c in zip(whole, parts, again):
        assert _close(b, a, 1e-5)
        np.testing.assert_array_equal(b.p, c.p)
