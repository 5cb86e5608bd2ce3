"""The allocation-free density monopole entry point against lpp_multipoles.

lpp_density_monopole_static serves callers that cannot call cudaMalloc (code inside
another framework's memory pool or under a fixed memory cap): its scratch is one fixed
device array inside liblpp, and it runs its own scatter assignment and full 3D FFT.  Two
calls in a row must both match the P_dd^(0) slot of the regular entry point, which shows
that the shared array is cleared between calls; the cases cover CIC and TSC, with and
without interlacing, explicit and unit weights, both precisions and an empty catalogue.
This file is collected last so that a stop-at-first-failure run has already run every
other test.
"""
import ctypes as C

import numpy as np
import pytest

from tests import parity_util as U

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2202_11839_gb300 import lpp as L
    return L, L.load_library()


def _static(lib, n, box, scheme, interlace, precision, pos, w, count, edges, stream):
    out = np.zeros(len(edges) - 1)
    nm = np.zeros(len(edges) - 1, dtype=np.int64)
    origin = (C.c_double * 3)(0.0, 0.0, 0.0)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    st = lib.lpp_density_monopole_static(
        n, box, origin, scheme, interlace, 1, precision, C.c_void_p(pos.data_ptr()) if pos is not None else None,
        C.c_void_p(w.data_ptr()) if w is not None else None, count, len(edges) - 1,
        e.ctypes.data_as(C.POINTER(C.c_double)), out.ctypes.data_as(C.POINTER(C.c_double)),
        nm.ctypes.data_as(C.POINTER(C.c_longlong)), C.c_void_p(stream))
    return st, out, nm


CASES = [
    # precision, tolerance, n, scheme, interlace, weights
    (0, 1e-5, 128, 3, 1, True),
    (1, 1e-10, 64, 3, 1, True),
    (1, 1e-10, 128, 2, 0, True),
    (1, 1e-10, 32, 2, 0, False),
    (1, 1e-10, 32, 2, 1, True),
    (1, 1e-10, 32, 3, 0, False),
    (0, 1e-5, 32, 2, 1, False),
    (0, 1e-5, 32, 3, 0, True),
]


@pytest.mark.parametrize("precision,tol,n,scheme,interlace,weights", CASES)
def test_static_monopole_matches_multipoles_twice(precision, tol, n, scheme, interlace, weights):
    import torch
    L, lib = _lib()
    dt = np.float64 if precision == L.LPP_FP64 else np.float32
    box = 600.0
    cat = U.make_case("static", n, count=20000, seed=21 + n + scheme, box=box, dtype=dt)
    edges = U.default_edges(n, box, 12, 0.8)
    # the regular path: a plan whose only moment is the density monopole
    plan = L.Plan(n, box, edges, observer=(300.0, 300.0, -2000.0), scheme=scheme, interlace=bool(interlace),
                  precision=precision, moments=1 << 0, max_shapes=cat["pos"].shape[1])
    pos = torch.from_numpy(np.ascontiguousarray(cat["pos"])).cuda()
    w = torch.from_numpy(np.ascontiguousarray(cat["w"])).cuda() if weights else None
    plan.assign(L.LPP_SHAPES, pos, w)
    ref = plan.multipoles()
    plan.close()
    want = ref.p[0].real
    scale = np.abs(want) + np.abs(ref.raw[0].real) / ref.norm_dd
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        st, out, nm = _static(lib, n, box, scheme, interlace, precision, pos, w, pos.shape[1], edges, stream)
        assert st == L.LPP_OK, lib.lpp_status_string(st)
        np.testing.assert_array_equal(nm, ref.n_modes)
        err = np.max(np.abs(out - want) / np.where(scale > 0, scale, 1.0))
        assert err < tol, (call, err)


def test_static_monopole_empty_catalogue_gives_zeros():
    import torch
    L, lib = _lib()
    n, box = 32, 600.0
    edges = U.default_edges(n, box, 6, 0.8)
    pos = torch.zeros((3, 1), dtype=torch.float32, device="cuda")
    st, out, nm = _static(lib, n, box, 2, 0, L.LPP_FP32, pos, None, 0, edges, torch.cuda.current_stream().cuda_stream)
    assert st == L.LPP_OK
    assert np.all(out == 0.0)
    assert nm.sum() > 0


def test_static_monopole_rejects_oversized_grid():
    L, lib = _lib()
    edges = np.linspace(0, 0.1, 5)
    out = np.zeros(4)
    origin = (C.c_double * 3)(0.0, 0.0, 0.0)
    for n, prec in ((256, 0), (256, 1)):
        st = lib.lpp_density_monopole_static(n, 1000.0, origin, 2, 0, 1, prec, None, None, 0, 4,
                                             edges.ctypes.data_as(C.POINTER(C.c_double)),
                                             out.ctypes.data_as(C.POINTER(C.c_double)), None, None)
        assert st == L.LPP_ERR_WORKSPACE
