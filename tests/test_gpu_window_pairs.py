"""Pair-count window multipoles (lpp_window_Q_pairs, Sec. 4.3) on the GPU against the FP64
oracle (window_pair_count_shells), element by element at 1e-10 of |Q_0| + |Q_l| per shell: a
polar-cap catalogue with weights and n-bar, a periodic box (minimal image), the empty
catalogue; and the pair count against the FFT estimate of the same randoms on a fine grid."""
import numpy as np
import pytest

from oracle import lpp_oracle as O
from paper_2202_11839_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    return L


def _err(q, ref):
    scale = np.abs(ref[0])[None, :] + np.abs(ref)
    return (np.abs(q - ref) / np.where(scale > 0, scale, 1.0)).max()


@pytest.mark.parametrize("periodic", [False, True])
def test_pair_count_matches_oracle(periodic):
    import torch
    L = _L()
    rng = np.random.default_rng(4)
    obs = (2000.0, 2000.0, 200.0)
    if periodic:
        box = 600.0
        pos = rng.uniform(0.0, box, (3, 3000))
        obs = (300.0, 300.0, -2000.0)
        edges = np.linspace(0.0, 250.0, 11)
    else:
        box = 0.0
        _, rand = S.survey_mock(10, 3500, 32, 4000.0, S.bbks_pk(0.2, 0.8), 1.0, 0.25, 8, obs, dtype=np.float64)
        pos = rand.pos
        edges = np.linspace(0.0, 1600.0, 17)
    n = pos.shape[1]
    w = rng.uniform(0.5, 1.5, n)
    nbar = rng.uniform(0.5, 2.0, n) * 1e-4
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    q = L.window_q_pairs(t(pos), t(w), t(nbar), obs, edges, alpha=0.3, box=box)
    ref = O.window_pair_count_shells(pos, w, nbar, 0.3, obs, edges, box=box)
    assert _err(q, ref) < 1e-10, _err(q, ref)
    # unit weights and n-bar (NULL pointers)
    q1 = L.window_q_pairs(t(pos), None, None, obs, edges, alpha=1.0, box=box)
    ref1 = O.window_pair_count_shells(pos, None, None, 1.0, obs, edges, box=box)
    assert _err(q1, ref1) < 1e-10


def test_pair_count_empty_and_bad_arguments():
    import ctypes as C
    import torch
    L = _L()
    pos = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    q = L.window_q_pairs(pos, None, None, (0, 0, 0), np.linspace(0, 10, 3))
    assert np.all(q == 0.0)
    lib = L.load_library()
    sz = C.c_size_t()
    assert lib.lpp_window_Q_pairs_workspace_size(0, C.byref(sz)) == L.LPP_ERR_INVALID_ARG
    assert lib.lpp_window_Q_pairs_workspace_size(300, C.byref(sz)) == L.LPP_ERR_INVALID_ARG


def test_pair_count_agrees_with_fft_window_on_a_cap():
    """The two estimators of Q_l on 60k randoms of the survey cap: the pair count of every pair
    and the FFT correlation on a 256^3 grid (box 4000, h = 15.6) agree in the shells well above
    the grid scale (50-1500 Mpc/h) to the grid's discreteness and the pairs' Poisson noise."""
    import torch
    L = _L()
    obs = (2000.0, 2000.0, 200.0)
    _, rand = S.survey_mock(10, 60000, 32, 4000.0, S.bbks_pk(0.2, 0.8), 1.0, 0.25, 9, obs, dtype=np.float64)
    edges = np.linspace(50.0, 1500.0, 30)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    qp = L.window_q_pairs(t(rand.pos), None, t(rand.nbar), obs, edges, alpha=1.0)
    plan = L.Plan(256, 4000.0, np.linspace(0, 0.1, 3), observer=obs, scheme=L.LPP_TSC, compensate=True,
                  precision=L.LPP_FP64, moments=1, max_shapes=1, max_randoms=rand.pos.shape[1])
    plan.assign(L.LPP_RANDOMS, t(rand.pos), None, t(rand.nbar))
    qf, _, _, _ = plan.window_q(edges)
    plan.close()
    np.testing.assert_allclose(qp[0], qf[0], rtol=0.03, atol=0.01 * np.abs(qf[0]).max())
    np.testing.assert_allclose(qp[1], qf[1], rtol=0.1, atol=0.03 * np.abs(qf[0]).max())


def test_padded_fft_window_agrees_with_pair_counts_at_large_separations():
    """The FFT window on a grid twice the survey box (origin moved by half a box, as the
    benchmark computes its template window) has no wrap-around: it agrees with the pair count
    out to 3500 Mpc/h, beyond the survey box's half size (the cap spans about 3100 Mpc/h)."""
    import torch
    L = _L()
    obs = (2000.0, 2000.0, 200.0)
    _, rand = S.survey_mock(10, 60000, 32, 4000.0, S.bbks_pk(0.2, 0.8), 1.0, 0.25, 9, obs, dtype=np.float64)
    edges = np.linspace(100.0, 3500.0, 35)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    qp = L.window_q_pairs(t(rand.pos), None, t(rand.nbar), obs, edges, alpha=1.0)
    plan = L.Plan(256, 8000.0, np.linspace(0, 0.1, 3), origin=(-2000.0, -2000.0, -2000.0), observer=obs,
                  scheme=L.LPP_TSC, compensate=True, precision=L.LPP_FP64, moments=1, max_shapes=1,
                  max_randoms=rand.pos.shape[1])
    plan.assign(L.LPP_RANDOMS, t(rand.pos), None, t(rand.nbar))
    qf, _, _, _ = plan.window_q(edges)
    plan.close()
    np.testing.assert_allclose(qp[0], qf[0], rtol=0.03, atol=0.01 * np.abs(qf[0]).max())
    np.testing.assert_allclose(qp[1], qf[1], rtol=0.1, atol=0.03 * np.abs(qf[0]).max())
