"""Window multipoles Q_l(s) on the GPU against the FP64 oracle (Eq. windowQ_ell, endpoint LOS)."""
import numpy as np
import pytest

from oracle import lpp_oracle as O

pytestmark = pytest.mark.gpu


def _cap_randoms(count, box, seed, dtype):
    """Randoms in a spherical cap-and-shell region of the box (an anisotropic window)."""
    rng = np.random.default_rng(seed)
    obs = np.array([box / 2, box / 2, 0.05 * box])
    r = rng.uniform(0.35 * box, 0.8 * box, 4 * count)
    mu = rng.uniform(0.55, 1.0, 4 * count)
    ph = rng.uniform(0, 2 * np.pi, 4 * count)
    st = np.sqrt(1 - mu * mu)
    p = np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * mu]) + obs[:, None]
    ok = np.all((p > 0) & (p < box), axis=0)
    p = p[:, ok][:, :count]
    w = rng.uniform(0.8, 1.2, p.shape[1])
    nbar = rng.uniform(0.5, 2.0, p.shape[1])
    return obs, p.astype(dtype), w.astype(dtype), nbar.astype(dtype)


def _run(L, prec, n, box, scheme, compensate, count, seed, with_density):
    import torch
    dt = np.float64 if prec == L.LPP_FP64 else np.float32
    obs, rp, rw, rn = _cap_randoms(count, box, seed, dt)
    s_edges = np.linspace(0.0, 0.35 * box, 9)
    plan = L.Plan(n, box, np.linspace(0, 0.1, 3), observer=tuple(obs), scheme=scheme, compensate=compensate,
                  precision=prec, moments=1, max_shapes=500, max_randoms=rp.shape[1])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    alpha = 1.0
    if with_density:
        dpos = rp[:, :400].copy()
        dw = (rw[:400] * 1.3).astype(dt)
        plan.assign(L.LPP_SHAPES, t(dpos), t(dw))
        alpha = float(np.sum(dw.astype(np.float64)) / np.sum(rw.astype(np.float64)))
    plan.assign(L.LPP_RANDOMS, t(rp), t(rw), t(rn))
    q, sm, npt, norm = plan.window_q(s_edges)
    plan.close()
    ref = O.window_multipoles(n, box, (0, 0, 0), tuple(obs), rp, rw, rn, alpha, s_edges, scheme=scheme,
                              compensate=compensate)
    return q, sm, npt, norm, ref


@pytest.mark.parametrize("prec,tol,n,scheme,comp,dens", [
    (1, 1e-10, 16, 2, True, False),
    (1, 1e-10, 32, 3, True, True),
    (1, 1e-10, 16, 3, False, True),
    (0, 1e-5, 32, 3, True, True),
    (0, 1e-5, 64, 2, True, False),
])
def test_window_parity(prec, tol, n, scheme, comp, dens):
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    q, sm, npt, norm, ref = _run(L, prec, n, 400.0, scheme, comp, 3000, 7, dens)
    np.testing.assert_array_equal(npt, ref.n_points)
    np.testing.assert_allclose(sm, ref.s_mean, rtol=1e-12)
    assert abs(norm - ref.norm) <= 1e-6 * abs(ref.norm)
    scale = np.abs(ref.q[0])[None, :] + np.abs(ref.q)
    err = np.abs(q - ref.q) / np.where(scale > 0, scale, 1.0)
    assert err.max() < tol, err.max(axis=1)
