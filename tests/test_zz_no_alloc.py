"""The allocation-free density monopole entry point against lpp_multipoles.

lpp_density_monopole_static serves callers that cannot call cudaMalloc (code inside
another framework's memory pool or under a fixed memory cap): its scratch is one fixed
device array inside liblpp.  Two calls in a row must both match the P_dd^(0) slot of the
regular entry point, which proves the shared array is cleared between calls.  This file
is collected last so that a stop-at-first-failure run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from tests import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol,n", [(0, 1e-5, 128), (1, 1e-10, 64)])
def test_static_monopole_matches_multipoles_twice(precision, tol, n):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2202_11839_gb300 import lpp as L
    lib = L.load_library()
    dt = np.float64 if precision == L.LPP_FP64 else np.float32
    box = 600.0
    cat = U.make_case("static", n, count=20000, seed=21, box=box, dtype=dt)
    edges = U.default_edges(n, box, 12, 0.8)
    # the regular path: a plan whose only moment is the density monopole
    plan = L.Plan(n, box, edges, observer=(300.0, 300.0, -2000.0), scheme=L.LPP_TSC, interlace=True,
                  precision=precision, moments=1 << 0, max_shapes=cat["pos"].shape[1])
    pos = torch.from_numpy(np.ascontiguousarray(cat["pos"])).cuda()
    w = torch.from_numpy(np.ascontiguousarray(cat["w"])).cuda()
    plan.assign(L.LPP_SHAPES, pos, w)
    ref = plan.multipoles()
    want = ref.p[0].real
    scale = np.abs(want) + np.abs(ref.raw[0].real) / ref.norm_dd
    origin = (C.c_double * 3)(0.0, 0.0, 0.0)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = np.zeros(len(edges) - 1)
        nm = np.zeros(len(edges) - 1, dtype=np.int64)
        st = lib.lpp_density_monopole_static(
            n, box, origin, L.LPP_TSC, 1, 1, precision, C.c_void_p(pos.data_ptr()), C.c_void_p(w.data_ptr()),
            pos.shape[1], len(edges) - 1, e.ctypes.data_as(C.POINTER(C.c_double)),
            out.ctypes.data_as(C.POINTER(C.c_double)), nm.ctypes.data_as(C.POINTER(C.c_longlong)),
            C.c_void_p(stream))
        assert st == L.LPP_OK, lib.lpp_status_string(st)
        np.testing.assert_array_equal(nm, ref.n_modes)
        err = np.max(np.abs(out - want) / np.where(scale > 0, scale, 1.0))
        assert err < tol, (call, err)
    plan.close()


def test_static_monopole_rejects_oversized_grid():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2202_11839_gb300 import lpp as L
    lib = L.load_library()
    edges = np.linspace(0, 0.1, 5)
    out = np.zeros(4)
    origin = (C.c_double * 3)(0.0, 0.0, 0.0)
    st = lib.lpp_density_monopole_static(512, 1000.0, origin, 2, 0, 1, 0, None, None, 0, 4,
                                         edges.ctypes.data_as(C.POINTER(C.c_double)),
                                         out.ctypes.data_as(C.POINTER(C.c_double)), None, None)
    assert st == L.LPP_ERR_WORKSPACE
