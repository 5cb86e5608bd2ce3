"""Window-convolved FFTLog templates on the GPU against the FP64 oracle (Sec. 3.2, Appendix D)."""
import numpy as np
import pytest

from oracle import template_oracle as T

pytestmark = pytest.mark.gpu

FAMILY_SCALE = {"dd": 0, "cross": 1, "plus": 4, "minus": 7}


def _window_table():
    """An anisotropic window: Q_l(s) decaying over the survey scale with l-dependent amplitudes."""
    s = np.linspace(5.0, 3600.0, 360)
    amp = np.array([1.0, -0.12, 0.05, -0.02, 0.008])
    q = amp[:, None] * np.exp(-(s / 1200.0) ** 2)[None, :] * (1.0 + 0.3 * np.cos(s / 400.0))[None, :]
    return q, s


def test_template_parity_fp64():
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    q, s = _window_table()
    edges = np.linspace(0.0, 0.2, 41)
    rng = np.random.default_rng(4)
    lo = np.array([0.0, 1.0, 0.6, -0.2, 0.1, 0.5])
    hi = np.array([3.0, 3.0, 1.0, 0.2, 0.3, 2.0])
    params = lo + (hi - lo) * rng.random((6, 6))
    tm = L.Template(q, s, edges, shot_plus=1234.5)
    out = tm(torch.from_numpy(params).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    mix = T.mixing_table()
    for i in range(params.shape[0]):
        ref = T.template(params[i], q, s, edges, shot_plus=1234.5, mixing=mix)
        for j, (kind, Lm) in enumerate(T.SLOTS):
            # per shell: relative to the value itself, with a floor of 1e-3 of the family's
            # largest value (an exact zero of a slot is compared against that floor)
            scale = np.abs(ref[j]) + 1e-3 * np.abs(ref[FAMILY_SCALE[kind]]).max()
            err = (np.abs(out[i, j] - ref[j]) / scale).max()
            assert err < 1e-10, (i, kind, Lm, err)
    tm.close()


def test_template_slot_mask():
    """lpp_template_set_slots: the masked-in slots are the full computation's, bit for bit, and
    the others zero; the derived curves come out the same from the nine slots they read."""
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    q, s = _window_table()
    edges = np.linspace(0.0, 0.2, 41)
    params = torch.from_numpy(np.array([[1.3, 1.8, 0.82, 0.05, 0.2, 1.0], [0.4, 2.5, 0.7, -0.1, 0.15, 0.6]])).cuda()
    tm = L.Template(q, s, edges, shot_plus=50.0)

    def run(fn):
        res = fn(params)
        torch.cuda.synchronize()
        return tuple(x.cpu().numpy() for x in res) if isinstance(res, tuple) else res.cpu().numpy()
    derived = lambda p: tm.derived(p, ref=None, sigma=None)
    full, eb_full = run(derived)
    tm.set_slots(L.TEMPLATE_EB_SLOTS)
    part, eb_part = run(derived)
    for j in range(L.LPP_N_MOMENTS):
        if (L.TEMPLATE_EB_SLOTS >> j) & 1:
            np.testing.assert_array_equal(part[:, j], full[:, j])
        else:
            assert np.all(part[:, j] == 0.0) and np.any(full[:, j] != 0.0), j
    np.testing.assert_array_equal(eb_part, eb_full)
    tm.set_slots((1 << L.LPP_MOM_MINUS12) | 1)
    only = run(tm)
    np.testing.assert_array_equal(only[:, L.LPP_MOM_MINUS12], full[:, L.LPP_MOM_MINUS12])
    np.testing.assert_array_equal(only[:, 0], full[:, 0])
    assert np.all(only[:, 1:L.LPP_MOM_MINUS12] == 0.0)
    tm.close()


def test_template_empty_batch_and_bad_args():
    import ctypes as C
    from paper_2202_11839_gb300 import lpp as L
    lib = L.load_library()
    q, s = _window_table()
    edges = np.linspace(0.0, 0.2, 5)
    tm = L.Template(q, s, edges)
    assert lib.lpp_convolve_template(tm.h, None, 0, None, None) == L.LPP_OK
    assert lib.lpp_convolve_template(tm.h, None, 3, None, None) == L.LPP_ERR_INVALID_ARG
    tm.close()


def test_template_png_parity_fp64():
    """Spin-2 PNG templates (lpp_template_set_png, Sec. 5) against the oracle at 1e-10 per shell."""
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    q, s = _window_table()
    edges = np.linspace(0.0, 0.2, 41)
    rng = np.random.default_rng(9)
    lo = np.array([0.0, 1.0, 0.6, -0.2, 0.1, 0.5])
    hi = np.array([3.0, 3.0, 1.0, 0.2, 0.3, 2.0])
    params = lo + (hi - lo) * rng.random((4, 6))
    tm = L.Template(q, s, edges, shot_plus=1234.5)
    mix = T.mixing_table()
    for png in ((-180.0, 0.17, 0.3), (40.0, 0.3, 0.25)):
        tm.set_png(*png)
        out = tm(torch.from_numpy(params).cuda()).cpu().numpy()
        for i in range(params.shape[0]):
            ref = T.template(params[i], q, s, edges, shot_plus=1234.5, mixing=mix, png=png)
            for j, (kind, Lm) in enumerate(T.SLOTS):
                scale = np.abs(ref[j]) + 1e-3 * np.abs(ref[FAMILY_SCALE[kind]]).max()
                err = (np.abs(out[i, j] - ref[j]) / scale).max()
                assert err < 1e-10, (png, i, kind, Lm, err)
    tm.set_png(0.0)
    out0 = tm(torch.from_numpy(params).cuda()).cpu().numpy()
    ref0 = T.template(params[0], q, s, edges, shot_plus=1234.5, mixing=mix)
    np.testing.assert_allclose(out0[0], ref0, rtol=1e-9, atol=1e-12 * np.abs(ref0).max())
    tm.close()
