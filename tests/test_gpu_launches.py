"""lpp_plan_launch_count against the kernels the CUDA profiling interface records for one
estimate (torch.profiler's CUPTI activity trace), so the launch count the benchmark reports
is the library's real one.  The profiling runs in a fresh interpreter: an activity trace
taken after other CUDA work in a long test process may come back empty."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
from torch.profiler import ProfilerActivity, profile
from paper_2202_11839_gb300 import lpp as L
from tests.parity_util import default_edges, make_case

def plan_for(n, interlace, n_rand):
    box = 300.0
    cat = make_case("tensor", n, 4000, 11, n_rand=n_rand, dtype=np.float32)
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

plans = [plan_for(32, True, 3000), plan_for(64, False, 0)]
for p, _ in plans:
    p.multipoles()
torch.cuda.synchronize()
with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]) as prof:
    for p, _ in plans:
        p.multipoles()
    torch.cuda.synchronize()
names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
kernels = [n for n in names if "memcpy" not in n.lower() and "memset" not in n.lower()]
counts = [p.launch_count() for p, _ in plans]
timed = []
for p, _ in plans:
    p.set_timing(True)
    p.multipoles()
    timed.append(p.launch_count())
print(json.dumps({"counts": counts, "timed": timed, "kernels": len(kernels), "names": sorted(set(kernels))}))
"""


def test_launch_count_matches_profiled_kernels():
    """Two plans (32^3 interlaced with randoms, 64^3 plain) in one profiler session: the
    device kernels recorded equal the sum of the two reported counts; timing on or off
    launches the same kernels."""
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert min(d["counts"]) > 0
    assert d["timed"] == d["counts"]
    if d["kernels"] == 0:
        pytest.skip("the profiler recorded no device activity")
    assert sum(d["counts"]) == d["kernels"], d


def test_launch_count_matches_graph_kernel_nodes():
    """Three mocks on two plans captured into one CUDA graph: the kernel nodes the CUDA
    runtime lists in the graph equal the sum of the counts the plans reported while the
    batch was captured; a second plain (uncaptured) batch counts the same."""
    from paper_2202_11839_gb300 import batch as B
    mocks = B.make_mocks(3, (20_000, 60_000), (32, 64), n_base=2, n_field=32)
    tuning = {32: B.Tuning(32, 4), 64: B.Tuning(64, 8)}
    run = B.BatchRun(mocks, tuning, use_graph=True)
    counted, nodes = run.batch.launch_count()
    assert counted > 0 and nodes == counted
    run.run()
    run.close()
    plain = B.BatchRun(mocks, tuning, use_graph=False)
    plain.run()
    counted2, nodes2 = plain.batch.launch_count()
    assert nodes2 == -1 and counted2 == counted
    plain.close()
