"""lpp_plan_launch_count against the kernels the CUDA profiling interface records for one
estimate (torch.profiler's CUPTI activity trace), so the launch count the benchmark reports
is the library's real one."""
import numpy as np
import pytest

from tests.parity_util import default_edges, make_case

pytestmark = pytest.mark.gpu


def _plan(L, cat, n, interlace, n_rand):
    import torch
    box = 300.0
    plan = L.Plan(n, box, default_edges(n, box), observer=(150.0, 150.0, -900.0), scheme=L.LPP_TSC,
                  interlace=interlace, precision=L.LPP_FP32, moments=L.LPP_WANT_ALL,
                  max_shapes=cat["pos"].shape[1], max_randoms=n_rand)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    keep = [dev(cat["pos"]), dev(cat["w"]), dev(cat["shape"])]
    plan.assign(L.LPP_SHAPES, keep[0], keep[1], None, keep[2], L.LPP_SHAPE_TENSOR6)
    if n_rand:
        keep += [dev(cat["rpos"]), dev(cat["rw"]), dev(cat["rnbar"])]
        plan.assign(L.LPP_RANDOMS, keep[3], keep[4], keep[5])
    return plan, keep


def test_launch_count_matches_profiled_kernels():
    """Two plans (32^3 interlaced with randoms, 64^3 plain) in one profiler session: the
    device kernels recorded equal the sum of the two reported counts."""
    import torch
    from torch.profiler import ProfilerActivity, profile

    from paper_2202_11839_gb300 import lpp as L
    plans, keep = [], []
    for n, interlace, n_rand in ((32, True, 3000), (64, False, 0)):
        cat = make_case("tensor", n, 4000, 11, n_rand=n_rand, dtype=np.float32)
        p, k = _plan(L, cat, n, interlace, n_rand)
        p.multipoles()
        plans.append(p)
        keep.append(k)
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]) as prof:
        for p in plans:
            p.multipoles()
        torch.cuda.synchronize()
    kernels = [e for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA
               and "memcpy" not in e.name.lower() and "memset" not in e.name.lower()]
    if not kernels:
        pytest.skip("the profiler recorded no device activity")
    counts = [p.launch_count() for p in plans]
    assert min(counts) > 0
    assert sum(counts) == len(kernels), (counts, sorted({e.name for e in kernels}))
    # timing on or off launches the same kernels
    for p, c in zip(plans, counts):
        p.set_timing(True)
        p.multipoles()
        assert p.launch_count() == c
        p.close()
