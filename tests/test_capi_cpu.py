"""Host-only checks of the C ABI: liblpp loads, exports every declared symbol, and
validates descriptors without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import lpp_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2202_11839_gb300 import lpp as L
    try:
        return L, L.load_library()
    except ImportError as e:  # build() must have run first
        pytest.fail(str(e))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lpp_[A-Za-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L, lib = _lib()
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTS), set(names) ^ set(L.EXPORTS)


def _desc(L, **kw):
    edges = np.linspace(0, 0.1, 5)
    d = L.PlanDesc()
    d.n, d.box = kw.get("n", 32), kw.get("box", 100.0)
    d.pole[:] = (-1, 0, 0)
    d.observer[:] = (0, 0, -500)
    d.scheme, d.interlace, d.compensate, d.precision = kw.get("scheme", 2), 0, 1, kw.get("precision", 0)
    d.moments = kw.get("moments", L.LPP_WANT_ALL)
    d.n_bins = len(edges) - 1
    d._edges = edges
    d.k_edges = edges.ctypes.data_as(C.POINTER(C.c_double))
    d.max_shapes = kw.get("max_shapes", 1000)
    d.batch = kw.get("batch", 0)
    return d


def test_plan_validation_on_host():
    L, lib = _lib()
    h = C.c_void_p()
    assert lib.lpp_plan_create(C.byref(_desc(L)), C.byref(h)) == L.LPP_OK
    sz = C.c_size_t()
    assert lib.lpp_plan_workspace_size(h, C.byref(sz)) == L.LPP_OK
    assert sz.value > 32 ** 3 * 8
    nf = C.c_int()
    assert lib.lpp_plan_field_count(h, C.byref(nf)) == L.LPP_OK
    # channels: cross 5+9+13, plus 2*(5+9), minus 2*(9+13+17), partners D, G1, G2
    assert nf.value == 27 + 28 + 78 + 3
    assert lib.lpp_plan_set_stream(h, None) == L.LPP_OK
    # multipoles before a workspace is set is refused
    r = L.Result()
    assert lib.lpp_multipoles(h, C.byref(r)) == L.LPP_ERR_NOT_READY
    lib.lpp_plan_destroy(h)
    for bad in (dict(n=48), dict(n=4), dict(n=2048)):
        assert lib.lpp_plan_create(C.byref(_desc(L, **bad)), C.byref(h)) == L.LPP_ERR_UNSUPPORTED
    for bad in (dict(scheme=4), dict(precision=3), dict(moments=0), dict(box=-1.0), dict(batch=99)):
        assert lib.lpp_plan_create(C.byref(_desc(L, **bad)), C.byref(h)) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_status_string(L.LPP_ERR_DOMAIN).decode() == "particle outside the domain"


def test_assign_validation_on_host():
    L, lib = _lib()
    h = C.c_void_p()
    assert lib.lpp_plan_create(C.byref(_desc(L, max_shapes=10)), C.byref(h)) == L.LPP_OK
    pos = np.zeros((3, 20), dtype=np.float32)
    p = L.Particles(pos.ctypes.data, None, None, None, 20, L.LPP_SHAPE_TENSOR6, 0)
    assert lib.lpp_assign(h, L.LPP_SHAPES, C.byref(p)) == L.LPP_ERR_INVALID_ARG   # over capacity
    p.count = 5
    p.shape_kind = L.LPP_SHAPE_NONE
    assert lib.lpp_assign(h, L.LPP_SHAPES, C.byref(p)) == L.LPP_ERR_INVALID_ARG   # shapes needed
    p.shape_kind = 7
    assert lib.lpp_assign(h, L.LPP_SHAPES, C.byref(p)) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_assign(h, 5, C.byref(p)) == L.LPP_ERR_INVALID_ARG
    p.on_host = 1
    p.shape_kind = L.LPP_SHAPE_TENSOR6
    p.shape = pos.ctypes.data
    assert lib.lpp_assign(h, L.LPP_SHAPES, C.byref(p)) == L.LPP_ERR_INVALID_ARG   # no host staging
    lib.lpp_plan_destroy(h)


def test_derive_eb_matches_oracle():
    """lpp_derive_eb (host arithmetic in the library) against the oracle's exact rationals."""
    L, _ = _lib()
    rng = np.random.default_rng(0)
    p = rng.standard_normal((10, 7)) + 1j * rng.standard_normal((10, 7))
    ge, ee, bb = L.derive_eb(p)
    oge, oee, obb = O.derived_eb(p)
    np.testing.assert_allclose(ge, oge, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(ee, oee, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(bb, obb, rtol=1e-13, atol=1e-13)


def test_template_tables_build_on_host():
    """lpp_template_create builds every host table without touching a GPU; bad inputs are refused."""
    L, lib = _lib()
    s = np.linspace(5.0, 3000.0, 50)
    q = np.zeros((5, s.size))
    q[0] = 1.0
    e = np.linspace(0, 0.2, 11)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    assert lib.lpp_template_create(dp(q), dp(s), s.size, dp(e), 10, 0.0, C.byref(h)) == L.LPP_OK
    sz = C.c_size_t()
    assert lib.lpp_template_workspace_size(h, C.byref(sz)) == L.LPP_OK
    assert sz.value > 16 * 4096 * 8
    assert lib.lpp_convolve_template(h, None, 1, None, None) == L.LPP_ERR_INVALID_ARG
    # slot masks: bits beyond the last slot are refused; the derived curves need slots 1..9
    assert lib.lpp_template_set_slots(h, C.c_uint(1 << L.LPP_N_MOMENTS)) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_template_set_slots(h, C.c_uint(L.TEMPLATE_EB_SLOTS & ~(1 << L.LPP_MOM_MINUS8))) == L.LPP_OK
    one = C.c_void_p(8)   # never dereferenced: the mask check comes first
    assert lib.lpp_convolve_template_eb(h, one, 1, one, one, None, None, None) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_template_set_slots(h, C.c_uint(L.TEMPLATE_EB_SLOTS)) == L.LPP_OK
    lib.lpp_template_destroy(h)
    bad = s[::-1].copy()
    assert lib.lpp_template_create(dp(q), dp(bad), s.size, dp(e), 10, 0.0, C.byref(h)) == L.LPP_ERR_INVALID_ARG


def test_gaussian_sigma_matches_oracle():
    from oracle import template_oracle as T
    L, _ = _lib()
    rng = np.random.default_rng(3)
    nb = 12
    edges = np.linspace(0.01, 0.2, nb + 1)
    p0 = rng.uniform(100.0, 20000.0, (4, nb))
    got = L.gaussian_sigma(p0, edges, 5.1e9, 3373.0, 210.0)
    want = T.gaussian_sigma(p0, edges, 5.1e9, 3373.0, 210.0)
    np.testing.assert_allclose(got, want, rtol=1e-13)
    with pytest.raises(L.LppError):
        L.gaussian_sigma(p0, edges[::-1], 5.1e9, 3373.0, 210.0)


def test_surrogate_state_layout_on_host():
    """The checkpoint size is the 32-byte header plus W (padded rows), b and both Adam moments
    of each layer in FP32; without a workspace there is no state to save or load."""
    L, lib = _lib()
    h = C.c_void_p()
    assert lib.lpp_surrogate_create(64, C.byref(h)) == L.LPP_OK
    sz = C.c_size_t()
    assert lib.lpp_surrogate_state_size(h, C.byref(sz)) == L.LPP_OK
    sizes = L.SURROGATE_SIZES
    pad = lambda k: (k + 15) // 16 * 16
    want = 32 + sum(3 * (o * pad(i) + o) * 4 for i, o in zip(sizes[:-1], sizes[1:]))
    assert sz.value == want
    buf = (C.c_ubyte * sz.value)()
    assert lib.lpp_surrogate_save_state(h, buf, sz, None) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_surrogate_load_state(h, buf, sz, None) == L.LPP_ERR_INVALID_ARG
    lib.lpp_surrogate_destroy(h)
