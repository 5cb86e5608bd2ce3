"""Pins of the oracle's pair-count window multipoles (Sec. 4.3 pair counting, Eq. windowQ_ell
with the endpoint line of sight): window_pair_count_shells.

* a uniform sphere of radius R seen from far away: Q_0(s) = alpha (N - 1)/N times the
  shell average of the overlap fraction of two spheres, 1 - 3s/(4R) + s^3/(16 R^3) (a closed
  form), and Q_2 = 0 up to the pair-count noise;
* a uniform periodic box: Q_0 = alpha (N - 1)/N in every shell, Q_l>0 = 0 up to the noise
  (for continuous shells the direction average of L_l vanishes);
* points on grid nodes of a periodic box: the same pair sums as the grid-shell form
  window_pair_count (pinned to the FFT estimate), rescaled from the N_b h^3 grid volume of a
  shell to its continuous volume;
* a plain double loop over the ordered pairs of a tiny catalogue.
A wrong endpoint (xhat of r' instead of r), a missing factor alpha or 2l+1, or the shell
volume of a wrong power fails these tests.
"""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import lpp_oracle as O


def _sphere(count, radius, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(3, count))
    p /= np.linalg.norm(p, axis=0)
    return p * radius * np.cbrt(rng.random(count))


def test_uniform_sphere_overlap_closed_form():
    R, N = 500.0, 6000
    pos = _sphere(N, R, 3) + np.array([[0.0], [0.0], [1e6]])
    nbar = np.full(N, N / (4.0 * math.pi * R ** 3 / 3.0))
    edges = np.linspace(50.0, 900.0, 9)
    q = O.window_pair_count_shells(pos, None, nbar, 1.0, (0.0, 0.0, 0.0), edges)
    # shell average (s^2 weighted) of the overlap fraction
    want = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        s = np.linspace(lo, hi, 2001)
        f = 1.0 - 3.0 * s / (4.0 * R) + s ** 3 / (16.0 * R ** 3)
        want.append(np.trapezoid(f * s * s, s) / np.trapezoid(s * s, s))
    want = np.array(want) * (N - 1) / N
    np.testing.assert_allclose(q[0], want, rtol=0.04, atol=0.004)
    assert np.all(np.abs(q[1]) < 0.02)


def test_uniform_periodic_box_is_flat_and_isotropic():
    box, N = 300.0, 5000
    rng = np.random.default_rng(5)
    pos = rng.uniform(0.0, box, (3, N))
    nbar = np.full(N, N / box ** 3)
    edges = np.linspace(20.0, 140.0, 7)
    q = O.window_pair_count_shells(pos, None, nbar, 1.0, (box / 2, box / 2, -1e7), edges, box=box)
    np.testing.assert_allclose(q[0], (N - 1) / N, rtol=0.03)
    assert np.all(np.abs(q[1:]) < 0.05)


def test_on_nodes_equals_grid_shell_form_rescaled():
    n, box = 16, 160.0
    h = box / n
    rng = np.random.default_rng(31)
    cells = rng.choice(n ** 3, 150, replace=False)
    ix, iy, iz = np.unravel_index(cells, (n, n, n))
    pos = np.stack([ix * h, iy * h, iz * h]).astype(np.float64)
    w = rng.uniform(0.5, 1.5, 150)
    nbar = rng.uniform(0.5, 2.0, 150)
    obs = (box / 2, box / 2, -400.0)
    # edges between lattice distances so that no pair sits on an edge
    edges = (np.arange(7) + 0.5) * h
    grid = O.window_pair_count(n, box, obs, pos, w, nbar, 0.7, edges)
    shells = O.window_pair_count_shells(pos, w, nbar, 0.7, obs, edges, box=box)
    sx, sy, sz, _ = O._separations(n, box)
    q2 = sx * sx + sy * sy + sz * sz
    nb = np.array([np.sum((q2 > 0) & (h * np.sqrt(q2) >= lo) & (h * np.sqrt(q2) < hi))
                   for lo, hi in zip(edges[:-1], edges[1:])])
    vol = 4.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3) / 3.0
    np.testing.assert_allclose(shells, grid * (nb * h ** 3 / vol)[None, :], rtol=1e-12, atol=1e-15)


def test_tiny_double_loop():
    rng = np.random.default_rng(2)
    N = 40
    pos = rng.uniform(100.0, 200.0, (3, N))
    w = rng.uniform(0.5, 1.5, N)
    nbar = rng.uniform(0.5, 2.0, N)
    obs = (150.0, 150.0, -300.0)
    edges = np.array([0.0, 20.0, 45.0, 70.0, 120.0])
    alpha = 0.8
    norm = alpha * np.sum(nbar * w * w)
    want = np.zeros((5, 4))
    for i in range(N):
        xi = pos[:, i] - np.array(obs)
        xi /= np.linalg.norm(xi)
        for j in range(N):
            if i == j:
                continue
            d = pos[:, j] - pos[:, i]
            s = math.sqrt(d @ d)
            for b in range(4):
                if edges[b] <= s < edges[b + 1]:
                    for li, ell in enumerate((0, 2, 4, 6, 8)):
                        want[li, b] += w[i] * w[j] * eval_legendre(ell, (d @ xi) / s)
    for li, ell in enumerate((0, 2, 4, 6, 8)):
        want[li] *= (2 * ell + 1) * alpha * alpha / (norm * 4.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3) / 3.0)
    got = O.window_pair_count_shells(pos, w, nbar, alpha, obs, edges)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)
