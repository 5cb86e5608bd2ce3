"""Seeded synthetic catalogues for the LPP tensor-multipole estimator.

This module only draws inputs: particle positions, weights, mean densities and
3D shape tensors s_ij.  It holds none of the estimator's arithmetic (no line of
sight, no sky frame, no projection, no mass assignment, no Fourier-space
combination), so both the CUDA path and the CPU oracle can consume the same
catalogues without sharing method code.

Workloads follow the paper's validation setting (Sec. 4.1): a Gaussian density
field in a periodic box, its tidal tensor T_ij = (k_i k_j / k^2 - delta_ij / 3)
delta(k), and galaxy shapes s_ij = -A T_ij read at the galaxy positions, plus
isotropic shape noise.  The paper's Planck-2015 linear P(k) and BOSS footprint
are not available here; a power law, the BBKS fitting form and a polar-cap
shell stand in for them.

Tensor components are stored SoA in the order (xx, yy, zz, xy, xz, yz).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TENSOR_ORDER = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _rng(seed: int, stream: int) -> np.random.Generator:
    """Counter-style independent streams: Philox keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


# --------------------------------------------------------------------------- P(k)
def power_law_pk(amp: float = 1.0e4, k0: float = 0.1, slope: float = -1.5):
    def pk(k):
        k = np.asarray(k, dtype=np.float64)
        out = np.zeros_like(k)
        nz = k > 0
        out[nz] = amp * (k[nz] / k0) ** slope
        return out
    return pk


def bbks_pk(gamma: float = 0.2, sigma8: float = 0.8, n_s: float = 1.0, tilt: float = 0.0):
    """BBKS-shaped linear spectrum P(k) = A k^(n_s+tilt) T^2(k/Gamma), sigma_8-normalised."""

    def shape(k):
        k = np.asarray(k, dtype=np.float64)
        q = k / gamma
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.log(1.0 + 2.34 * q) / (2.34 * q) * (
                1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25
        t = np.where(q > 0, t, 1.0)
        return np.where(k > 0, k ** (n_s + tilt) * t * t, 0.0)

    # sigma_8 normalisation by log-spaced trapezoid quadrature (top hat, R = 8)
    lk = np.linspace(np.log(1e-5), np.log(1e3), 20001)
    k = np.exp(lk)
    x = 8.0 * k
    wth = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    integrand = shape(k) * wth ** 2 * k ** 3 / (2.0 * math.pi ** 2)
    s2 = np.trapezoid(integrand, lk)
    amp = sigma8 ** 2 / s2

    def pk(kk):
        return amp * shape(kk)
    return pk


# ------------------------------------------------------------------ grid fields
def fft_freq_grid(n: int, box: float):
    """Wave-vector components on an n^3 FFT grid, numpy fftfreq ordering."""
    kf = 2.0 * math.pi / box
    f = np.fft.fftfreq(n, d=1.0 / n) * kf
    return np.meshgrid(f, f, f, indexing="ij")


def gaussian_field_k(n: int, box: float, pk, seed: int, stream: int = 1,
                     fixed_amplitude: bool = False) -> np.ndarray:
    """Fourier-space Gaussian field delta(k) (complex, Hermitian), grid indexed [ix, iy, iz].

    Convention: delta(x) = (1/V) sum_k delta(k) e^{ik.x};  <|delta(k)|^2> = V P(k).
    With ``fixed_amplitude`` every mode has |delta(k)|^2 = V P(k) exactly (random phases).
    Modes at or above the Nyquist index are zeroed, and so is k = 0.
    """
    rng = _rng(seed, stream)
    vol = box ** 3
    g = rng.standard_normal((n, n, n))
    dk = np.fft.fftn(g)              # Hermitian white noise, <|dk|^2> = n^3
    if fixed_amplitude:
        mag = np.abs(dk)
        mag[mag == 0] = 1.0
        dk = dk / mag * math.sqrt(n ** 3)
    kx, ky, kz = fft_freq_grid(n, box)
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.sqrt(pk(kk) * vol / n ** 3)
    dk = dk * amp
    idx = np.fft.fftfreq(n, d=1.0 / n)
    nyq = np.abs(idx) >= n // 2
    dk[nyq, :, :] = 0
    dk[:, nyq, :] = 0
    dk[:, :, nyq] = 0
    dk[0, 0, 0] = 0
    return dk


def real_space(dk: np.ndarray, box: float) -> np.ndarray:
    n = dk.shape[0]
    return np.real(np.fft.ifftn(dk)) * n ** 3 / box ** 3


def tidal_tensor_grids(dk: np.ndarray, box: float) -> np.ndarray:
    """T_ij(x) = FT^-1[(k_i k_j / k^2 - delta_ij/3) delta(k)], shape (6, n, n, n)."""
    n = dk.shape[0]
    kx, ky, kz = fft_freq_grid(n, box)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    ks = (kx, ky, kz)
    out = np.empty((6, n, n, n), dtype=np.float64)
    for c, (i, j) in enumerate(TENSOR_ORDER):
        t = ks[i] * ks[j] / k2
        if i == j:
            t = t - 1.0 / 3.0
        out[c] = real_space(t * dk, box)
    return out


def read_ngp(grids: np.ndarray, pos: np.ndarray, box: float, origin) -> np.ndarray:
    """Nearest-grid-point read of grids (..., n, n, n) at positions (3, np)."""
    n = grids.shape[-1]
    h = box / n
    idx = [np.floor((pos[a] - origin[a]) / h + 0.5).astype(np.int64) % n for a in range(3)]
    return grids[..., idx[0], idx[1], idx[2]]


def shape_noise_tensor(count: int, sigma: float, seed: int, stream: int) -> np.ndarray:
    """Isotropic traceless symmetric Gaussian tensors, (6, count).

    The five traceless components along an orthonormal basis get variance 2 sigma^2,
    so that any projection onto a spin-2 basis e_ij (e.e* = 1) has variance sigma^2
    per real component.
    """
    rng = _rng(seed, stream)
    g = rng.standard_normal((5, count)) * (math.sqrt(2.0) * sigma)
    r2, r6 = math.sqrt(2.0), math.sqrt(6.0)
    basis = np.zeros((5, 3, 3))
    basis[0] = np.diag([1.0, -1.0, 0.0]) / r2
    basis[1] = np.diag([1.0, 1.0, -2.0]) / r6
    basis[2][0, 1] = basis[2][1, 0] = 1.0 / r2
    basis[3][0, 2] = basis[3][2, 0] = 1.0 / r2
    basis[4][1, 2] = basis[4][2, 1] = 1.0 / r2
    t = np.einsum("pc,pij->ijc", g, basis)
    return np.stack([t[i, j] for (i, j) in TENSOR_ORDER])


# --------------------------------------------------------------------- catalogues
@dataclass
class Catalogue:
    pos: np.ndarray                 # (3, n)
    w: np.ndarray | None = None     # (n,)
    nbar: np.ndarray | None = None  # (n,)
    shape: np.ndarray | None = None  # (6, n) tensor or (2, n) gamma

    @property
    def count(self) -> int:
        return int(self.pos.shape[1])

    def astype(self, dtype) -> "Catalogue":
        cv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=dtype)
        return Catalogue(cv(self.pos), cv(self.w), cv(self.nbar), cv(self.shape))


@dataclass
class Workload:
    name: str
    n: int
    box: float
    origin: tuple
    observer: tuple
    pole: tuple
    scheme: int                    # 2 = CIC, 3 = TSC
    interlace: bool
    shapes: Catalogue
    randoms: Catalogue | None = None
    density: Catalogue | None = None
    k_edges: np.ndarray = field(default_factory=lambda: np.zeros(0))
    dtype: str = "f32"
    extra: dict = field(default_factory=dict)


def uniform_positions(count: int, box: float, origin, seed: int, stream: int, dtype=np.float64):
    rng = _rng(seed, stream)
    p = rng.random((3, count)) * box
    for a in range(3):
        p[a] += origin[a]
    p = p.astype(dtype)
    # keep strictly inside [origin, origin + box) after rounding
    for a in range(3):
        hi = np.nextafter(np.asarray(origin[a] + box, dtype=dtype), np.asarray(origin[a], dtype=dtype))
        np.minimum(p[a], hi, out=p[a])
    return p


def periodic_tidal_mock(n_gal: int, n_field: int, box: float, pk, amp_a: float, sigma_noise: float,
                        seed: int, dtype=np.float64, origin=(0.0, 0.0, 0.0)) -> Catalogue:
    """Uniform galaxies in a periodic box with shapes s_ij = -A T_ij + noise (config-1 style)."""
    pos = uniform_positions(n_gal, box, origin, seed, 0, dtype)
    dk = gaussian_field_k(n_field, box, pk, seed, 1)
    tij = tidal_tensor_grids(dk, box)
    s = -amp_a * read_ngp(tij, pos.astype(np.float64), box, origin)
    if sigma_noise > 0:
        s = s + shape_noise_tensor(n_gal, sigma_noise, seed, 2)
    return Catalogue(pos=pos, w=None, nbar=None, shape=s.astype(dtype))


def poisson_tidal_mock(mean_count: float, n_field: int, box: float, pk, amp_a: float,
                       sigma_noise: float, seed: int, dtype=np.float32,
                       origin=(0.0, 0.0, 0.0)) -> Catalogue:
    """Poisson sampling of 1+delta (clipped at 0) with the same field's tidal shapes (config-2 style)."""
    dk = gaussian_field_k(n_field, box, pk, seed, 1)
    delta = real_space(dk, box)
    lam = np.maximum(0.0, 1.0 + delta)
    lam *= mean_count / lam.sum()
    rng = _rng(seed, 3)
    counts = rng.poisson(lam).ravel()
    cells = np.repeat(np.arange(counts.size), counts)
    ix, iy, iz = np.unravel_index(cells, (n_field,) * 3)
    h = box / n_field
    jit = rng.random((3, cells.size))
    pos = np.stack([(ix + jit[0]) * h + origin[0], (iy + jit[1]) * h + origin[1],
                    (iz + jit[2]) * h + origin[2]])
    perm = rng.permutation(cells.size)
    pos = pos[:, perm]
    tij = tidal_tensor_grids(dk, box)
    s = -amp_a * read_ngp(tij, pos, box, origin)
    if sigma_noise > 0:
        s = s + shape_noise_tensor(pos.shape[1], sigma_noise, seed, 2)
    pos = pos.astype(dtype)
    for a in range(3):
        hi = np.nextafter(np.asarray(origin[a] + box, dtype=dtype), np.asarray(origin[a], dtype=dtype))
        np.minimum(pos[a], hi, out=pos[a])
    return Catalogue(pos=pos, shape=s.astype(dtype))


def _cap_shell_points(count: int, rng, observer, r_mean, r_sigma, r_lo, r_hi, theta_max):
    """Points in a polar cap (axis +z about the observer) with Gaussian n(r) in [r_lo, r_hi]."""
    out = np.empty((3, 0))
    cos_min = math.cos(theta_max)
    need = count
    chunks = []
    while need > 0:
        m = int(need * 1.3) + 1024
        r = rng.normal(r_mean, r_sigma, m)
        # radial density n(r) r^2 dr: accept by r^2 weight on the Gaussian draw
        keep = (r > r_lo) & (r < r_hi) & (rng.random(m) < (r / r_hi) ** 2)
        r = r[keep]
        mu = cos_min + (1.0 - cos_min) * rng.random(r.size)
        ph = 2.0 * math.pi * rng.random(r.size)
        st = np.sqrt(1.0 - mu * mu)
        p = np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * mu])
        chunks.append(p[:, :need])
        need -= min(need, p.shape[1])
    out = np.concatenate(chunks, axis=1)
    for a in range(3):
        out[a] += observer[a]
    return out


def survey_mock(n_data: int, n_rand: int, n_field: int, box: float, pk, amp_a: float,
                sigma_noise: float, seed: int, observer, dtype=np.float32,
                r_mean=1400.0, r_sigma=200.0, r_lo=1000.0, r_hi=1800.0,
                theta_max=math.radians(60.0), origin=(0.0, 0.0, 0.0)):
    """Cap-and-shell survey (config-3 style): data selected from 1+delta, randoms from n(r)."""
    dk = gaussian_field_k(n_field, box, pk, seed, 1)
    delta = real_space(dk, box)
    rng = _rng(seed, 4)
    # data: draw from the selection function, thin by (1+delta)/max
    one_plus = np.maximum(0.0, 1.0 + delta)
    cap = one_plus.max()
    chunks = []
    have = 0
    while have < n_data:
        cand = _cap_shell_points(int((n_data - have) * cap * 1.2) + 4096, rng, observer,
                                 r_mean, r_sigma, r_lo, r_hi, theta_max)
        acc = rng.random(cand.shape[1]) * cap < read_ngp(one_plus, cand, box, origin)
        cand = cand[:, acc]
        chunks.append(cand[:, : n_data - have])
        have += min(cand.shape[1], n_data - have)
    pos_d = np.concatenate(chunks, axis=1)
    rng_r = _rng(seed + 1, 5)
    pos_r = _cap_shell_points(n_rand, rng_r, observer, r_mean, r_sigma, r_lo, r_hi, theta_max)
    # nbar(r) normalised so that sum over randoms of nbar dV matches n_data
    def nbar_of(p):
        r = np.sqrt(sum((p[a] - observer[a]) ** 2 for a in range(3)))
        return np.exp(-0.5 * ((r - r_mean) / r_sigma) ** 2)
    shell_vol = (2.0 * math.pi * (1.0 - math.cos(theta_max))) * (r_hi ** 3 - r_lo ** 3) / 3.0
    nb_r = nbar_of(pos_r)
    scale = n_data / (nb_r.mean() * shell_vol) if n_rand else 1.0
    tij = tidal_tensor_grids(dk, box)
    s = -amp_a * read_ngp(tij, pos_d, box, origin)
    if sigma_noise > 0:
        s = s + shape_noise_tensor(pos_d.shape[1], sigma_noise, seed, 2)
    data = Catalogue(pos=pos_d.astype(dtype), nbar=(nbar_of(pos_d) * scale).astype(dtype),
                     shape=s.astype(dtype))
    rand = Catalogue(pos=pos_r.astype(dtype), nbar=(nb_r * scale).astype(dtype))
    return data, rand


# ------------------------------------------------------------------ named workloads
def linear_edges(kmin: float, kmax: float, nb: int) -> np.ndarray:
    return np.linspace(kmin, kmax, nb + 1)


def workload_periodic_fp64(n_gal: int = 50_000, n: int = 64, box: float = 500.0,
                           seed: int = 0) -> Workload:
    """Periodic box L=500, 64^3 CIC, 50k uniform galaxies, power-law tidal shapes, sigma=0.2 (FP64)."""
    pk = power_law_pk(1.0e4, 0.1, -1.5)
    cat = periodic_tidal_mock(n_gal, n, box, pk, 1.0, 0.2, seed, np.float64)
    kny = math.pi * n / box
    return Workload("periodic_L500_N64_cic_fp64", n, box, (0.0, 0.0, 0.0), (0.0, 0.0, -3000.0),
                    (-1.0, 0.0, 0.0), 2, False, cat, k_edges=linear_edges(0.0, kny, 20),
                    dtype="f64")


def workload_periodic_tsc(n_gal: int = 2_000_000, n: int = 256, box: float = 2000.0,
                          n_field: int | None = None, seed: int = 0) -> Workload:
    """Periodic tidal mock L=2000, 256^3 TSC + interlacing, Poisson 2M galaxies, BBKS (FP32)."""
    pk = bbks_pk(0.2, 0.8)
    cat = poisson_tidal_mock(n_gal, n_field or n, box, pk, 1.0, 0.25, seed, np.float32)
    obs = (box / 2, box / 2, box / 2 - 4000.0)
    return Workload("periodic_L2000_N256_tsc_il", n, box, (0.0, 0.0, 0.0), obs, (-1.0, 0.0, 0.0),
                    3, True, cat, k_edges=linear_edges(0.0, 0.4, 40), dtype="f32")


def workload_survey(n_data: int = 1_500_000, n_rand: int = 15_000_000, n: int = 512,
                    box: float = 4000.0, n_field: int = 256, seed: int = 0) -> Workload:
    """Polar-cap shell survey 1000-1800 Mpc/h, theta<60 deg, n(r) peaked at 1400; 512^3 TSC+IL."""
    pk = bbks_pk(0.2, 0.8)
    obs = (box / 2, box / 2, 200.0)
    data, rand = survey_mock(n_data, n_rand, n_field, box, pk, 1.0, 0.25, seed, obs)
    return Workload("survey_cap_L4000_N512_tsc_il", n, box, (0.0, 0.0, 0.0), obs, (-1.0, 0.0, 0.0),
                    3, True, data, randoms=rand, k_edges=linear_edges(0.0, 0.2, 40), dtype="f32")


# ----------------------------------------------------------------- surrogate inputs
SURROGATE_RANGES = np.array([[0.0, 3.0], [1.0, 3.0], [0.6, 1.0], [-0.2, 0.2], [0.1, 0.3], [0.5, 2.0]])


def latin_hypercube(n: int, ranges=SURROGATE_RANGES, seed: int = 0) -> np.ndarray:
    """n points of a Latin hypercube over the box `ranges` ([dim, 2]): one point per stratum
    of every coordinate, strata shuffled independently, uniform within each stratum."""
    rng = _rng(seed, 11)
    d = len(ranges)
    u = (np.stack([rng.permutation(n) for _ in range(d)], axis=1) + rng.random((n, d))) / n
    return ranges[:, 0] + u * (ranges[:, 1] - ranges[:, 0])


def surrogate_init(seed: int = 0, sizes=(6, 256, 256, 256, 256, 320)):
    """Initial weights W [out, in] ~ U(-1/sqrt(in), 1/sqrt(in)) and zero biases (FP32)."""
    rng = _rng(seed, 12)
    layers = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / math.sqrt(fi)
        layers.append((rng.uniform(-lim, lim, (fo, fi)).astype(np.float32), np.zeros(fo, dtype=np.float32)))
    return layers
