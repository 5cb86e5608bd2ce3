"""Template emulator: the surrogate network (lpp_surrogate_*) trained on window-convolved
templates from the FFTLog path (lpp_convolve_template_eb), which stays its fallback and its
accuracy reference.

Emulated quantity: the Legendre multipoles gE_0,2, EE_0,2,4 and BB_0,2,4 of the window-
convolved template (Sec. 3.2, Eq. window_convolution_X_hankel; Sec. 2.4 for E/B) at 40
k-shells, 320 numbers, in units of their Gaussian error bar (lpp_gaussian_sigma) at the
fiducial parameters.  The template is exactly A b_g sigma_8^2 (gE) or A^2 sigma_8^2 (EE/BB)
times a shape that depends on (tilt, Gamma) alone, plus the shot-noise scale times a fixed
vector (Eq. all_convolutions with the linear-alignment model), so the network learns the
shape and the exact factors are applied in the decoding kernel (lpp_surrogate_map).

Every numerical step runs in the library's kernels: the templates (FFTLog, one CTA per
parameter set), the input encoding, the training steps (BF16 tensor-core GEMMs, Adam) and the
decoded prediction.  This module only draws parameter sets and minibatch schedules (host,
seeded) and moves arrays.
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass, field

import numpy as np

from . import lpp as L
from . import synthetic as S

PARAM_NAMES = ("A", "b_g", "sigma_8", "tilt", "Gamma", "shot")
FIDUCIAL = (1.5, 2.0, 0.8, 0.0, 0.2, 1.25)   # centre of the parameter box
FEED = (0, 0, 0, 1, 1, 0)                     # the network sees (tilt, Gamma)


@dataclass
class TrainConfig:
    n_train: int = 20000
    n_test: int = 2000
    batch: int = 256
    epochs: tuple = (450, 450, 450, 450)          # epochs per learning-rate phase
    lrs: tuple = (1e-3, 3e-4, 1e-4, 3e-5)
    base_nodes: int = 8                           # Lobatto nodes per (tilt, Gamma) axis of the baseline
    seed: int = 0


@dataclass
class Report:
    """Accuracy of the emulator against the FFTLog path on held-out parameter sets."""
    rms_sigma: float
    max_sigma: float
    p99_sigma: float
    per_curve_max: list = field(default_factory=list)
    baseline_rms_sigma: float = 0.0      # the interpolated baseline alone (network output 0)
    baseline_max_sigma: float = 0.0
    final_loss: float = 0.0
    train_seconds: float = 0.0
    data_seconds: float = 0.0


def unit_amplitude(params: np.ndarray) -> np.ndarray:
    """The same (tilt, Gamma) with A = b_g = sigma_8 = 1 and no shot noise."""
    p = np.array(params, dtype=np.float64, copy=True)
    p[:, 0] = 1.0
    p[:, 1] = 1.0
    p[:, 2] = 1.0
    p[:, 5] = 0.0
    return p


class Emulator:
    """Surrogate of one window (q table) and binning; see the module docstring.  The emulator
    sets the template's slot mask to TEMPLATE_EB_SLOTS (the slots its curves read)."""

    def __init__(self, template: L.Template, volume: float, noise_g: float, cfg: TrainConfig | None = None,
                 device=None):
        import torch
        self.torch = torch
        self.t = template
        # the curves read the cross, plus and minus slots up to L = 8: the template computes those alone
        template.set_slots(L.TEMPLATE_EB_SLOTS)
        self.cfg = cfg or TrainConfig()
        if template.nb * 8 != 320:
            raise ValueError("the surrogate emulates 8 curves x 40 shells")
        self.device = template.device if device is None else torch.device(device)
        self.ranges = S.SURROGATE_RANGES
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.device)
        # Gaussian error bars from the fiducial window-convolved monopoles without shot noise,
        # and P_BB = 0 (the linear-alignment model has no B modes; window leakage into B is
        # not given a cosmic variance of its own)
        fid = np.array([FIDUCIAL])
        fid[0, 5] = 0.0
        self.native_fid, eb64 = self._derived64(fid)
        p0 = np.stack([self.native_fid[0], eb64[0], eb64[2], np.zeros_like(eb64[0])])
        noise_e = 0.5 * FIDUCIAL[5] * template.shot_plus
        self.sigma = L.gaussian_sigma(p0, template.k_edges, volume, noise_g, noise_e).reshape(-1)
        # unit-amplitude shape at the fiducial (tilt, Gamma) and the shot-noise response
        _, u0 = self._derived64(unit_amplitude(np.array([FIDUCIAL])))
        _, s_vec = self._derived64(np.array([[0.0, 1.0, 1.0, FIDUCIAL[3], FIDUCIAL[4], 1.0]]))
        nb = template.nb
        pre = np.empty(320)
        A, b, s8 = FIDUCIAL[:3]
        pre[: 2 * nb] = A * b * s8 * s8
        pre[2 * nb:] = A * A * s8 * s8
        self.sd = dev(self.sigma / pre)             # network outputs in error bars at the fiducial amplitude
        self.shot = dev(s_vec.reshape(-1))
        self.sigma_dev = dev(self.sigma)
        # baseline: the unit-amplitude curves interpolated from a nodes x nodes Lobatto grid in
        # (tilt, Gamma); the network learns the remainder
        nn = self.cfg.base_nodes
        if nn >= 2:
            xs = -np.cos(np.pi * np.arange(nn) / (nn - 1))
            lo, hi = self.ranges[3:5, 0], self.ranges[3:5, 1]
            grid = np.array([[1.0, 1.0, 1.0, lo[0] + (xa + 1) * (hi[0] - lo[0]) / 2,
                              lo[1] + (xb + 1) * (hi[1] - lo[1]) / 2, 0.0] for xa in xs for xb in xs])
            self.base = dev(np.stack([self._derived64(grid[i:i + 1])[1].reshape(-1) for i in range(len(grid))]))
            self.mu = dev(np.zeros(320))
        else:
            self.base = None
            self.mu = dev(u0.reshape(-1))
        self.net = None

    def _derived64(self, params: np.ndarray):
        """Native slots [LPP_N_MOMENTS, nb] of one parameter set from the template kernel (FP64) and its
        derived curves [8, nb] in FP64 (lpp_derive_eb)."""
        torch = self.torch
        native = self.t(torch.from_numpy(np.ascontiguousarray(params, dtype=np.float64)).to(self.device))
        nat = native.cpu().numpy()[0]
        ge, ee, bb = L.derive_eb(nat.astype(np.complex128))
        return nat, np.concatenate([ge, ee, bb], axis=0)

    # -------------------------------------------------------------------- training
    def _make_net(self):
        layers = S.surrogate_init(self.cfg.seed)
        net = L.Surrogate(L.flatten_params(layers), batch=self.cfg.batch, stream=self.t.stream, device=self.device)
        net.set_map(self.ranges[:, 0], self.ranges[:, 1], FEED, self.mu, self.sd, self.shot, None, self.sigma_dev,
                    base=self.base, base_nodes=self.cfg.base_nodes if self.base is not None else 0, base_in=(3, 4))
        return net

    def training_set(self, n: int, seed: int):
        """Parameter sets (device FP64) and network targets (device FP32) for n LHS points."""
        torch = self.torch
        theta = S.latin_hypercube(n, self.ranges, seed)
        th = torch.from_numpy(theta).to(self.device)
        native = self.t(torch.from_numpy(unit_amplitude(theta)).to(self.device))
        return th, self.net.targets(th, native)

    def _fingerprint(self) -> str:
        c = self.cfg
        return json.dumps([c.n_train, c.batch, list(c.epochs), list(c.lrs), c.base_nodes, c.seed])

    def train(self, checkpoint: str | None = None, resume: str | None = None, phases: int | None = None):
        """Train on cfg.n_train Latin-hypercube templates, one Adam schedule per learning-rate
        phase.  checkpoint: after every phase, write the network's training state
        (lpp_surrogate_save_state), the next phase, the schedule generator's state and the
        losses so far to this .npz file.  resume: continue from such a file (the same
        TrainConfig; the training set is regenerated from its seed).  phases: stop after this
        many phases in total (None: all)."""
        import time
        torch = self.torch
        cfg = self.cfg
        self.net = self._make_net()
        t0 = time.perf_counter()
        th, y = self.training_set(cfg.n_train, cfg.seed)
        torch.cuda.synchronize(self.device)
        t1 = time.perf_counter()
        x = self.net.encode(th)
        rng = np.random.default_rng(cfg.seed + 1000)
        steps_per_epoch = cfg.n_train // cfg.batch
        losses = []
        first = 0
        if resume is not None:
            ck = np.load(resume, allow_pickle=False)
            if str(ck["config"]) != self._fingerprint():
                raise ValueError("checkpoint was written for another TrainConfig")
            self.net.load_state(ck["state"])
            rng.bit_generator.state = json.loads(str(ck["rng"]))
            first = int(ck["phase"])
            if ck["losses"].size:
                losses.append(torch.from_numpy(ck["losses"]).to(self.device))
        last = len(cfg.epochs) if phases is None else min(phases, len(cfg.epochs))
        for ph in range(first, last):
            epochs, lr = cfg.epochs[ph], cfg.lrs[ph]
            sched = np.concatenate([rng.permutation(cfg.n_train)[: steps_per_epoch * cfg.batch]
                                    for _ in range(epochs)]).astype(np.int32)
            sd = torch.from_numpy(sched).to(self.device)
            ls = torch.zeros(epochs * steps_per_epoch, dtype=torch.float64, device=self.device)
            self.net.train(x, y, sd, lr, ls)
            losses.append(ls)
            if checkpoint is not None:
                np.savez(checkpoint, state=self.net.save_state(), phase=np.int64(ph + 1),
                         rng=np.array(json.dumps(rng.bit_generator.state)), config=np.array(self._fingerprint()),
                         losses=torch.cat(losses).cpu().numpy() if losses else np.zeros(0))
        torch.cuda.synchronize(self.device)
        t2 = time.perf_counter()
        self.losses = torch.cat(losses).cpu().numpy() if losses else np.zeros(0)
        self.data_seconds, self.train_seconds = t1 - t0, t2 - t1
        return t1 - t0, t2 - t1

    # -------------------------------------------------------------------- judging
    def plain(self, params):
        """The FFTLog path's curves in error-bar units (the fallback and the accuracy reference)."""
        _, eb = self.t.derived(params, ref=None, sigma=self.sigma_dev)
        return eb

    def predict(self, params):
        return self.net.predict(params)

    def inside(self, theta: np.ndarray) -> np.ndarray:
        lo, hi = self.ranges[:, 0], self.ranges[:, 1]
        return np.all((theta >= lo) & (theta <= hi), axis=1)

    def templates(self, theta: np.ndarray):
        """Curves in error-bar units for host parameter sets [n, 6]: the network inside its
        training box, the FFTLog path (the fallback) outside it."""
        torch = self.torch
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        out = torch.empty((theta.shape[0], 320), dtype=torch.float32, device=self.device)
        ok = self.inside(theta)
        for sel, fn in ((ok, self.predict), (~ok, self.plain)):
            idx = np.nonzero(sel)[0]
            if idx.size:
                out[torch.from_numpy(idx).to(self.device)] = fn(torch.from_numpy(theta[idx]).to(self.device))
        return out

    def inference_net(self, batch: int = 8192):
        """A copy of the trained network that runs inference in chunks of `batch` rows."""
        net = L.Surrogate(self.net.params(), batch=batch, stream=self.t.stream, device=self.device)
        net.set_map(self.ranges[:, 0], self.ranges[:, 1], FEED, self.mu, self.sd, self.shot, None, self.sigma_dev,
                    base=self.base, base_nodes=self.cfg.base_nodes if self.base is not None else 0, base_in=(3, 4))
        return net

    def evaluate(self, n: int, seed: int) -> Report:
        torch = self.torch
        theta = S.latin_hypercube(n, self.ranges, seed)
        th = torch.from_numpy(theta).to(self.device)
        plain = self.plain(th).double()
        d = (self.predict(th).double() - plain).abs().cpu().numpy()
        # the baseline alone: the exact remainder y* that the network should output, scaled back
        y_true = self.net.targets(th, self.t(torch.from_numpy(unit_amplitude(theta)).to(self.device))).double()
        nb = self.t.nb
        pre = np.empty((n, 320))
        pre[:, : 2 * nb] = (theta[:, 0] * theta[:, 1] * theta[:, 2] ** 2)[:, None]
        pre[:, 2 * nb:] = (theta[:, 0] ** 2 * theta[:, 2] ** 2)[:, None]
        base_err = np.abs(pre * (y_true * self.sd / self.sigma_dev).cpu().numpy())
        return Report(rms_sigma=float(np.sqrt(np.mean(d * d))), max_sigma=float(d.max()),
                      p99_sigma=float(np.quantile(d, 0.99)),
                      per_curve_max=[float(d[:, c * nb:(c + 1) * nb].max()) for c in range(8)],
                      baseline_rms_sigma=float(np.sqrt(np.mean(base_err ** 2))),
                      baseline_max_sigma=float(base_err.max()),
                      final_loss=float(np.mean(self.losses[-50:])), train_seconds=self.train_seconds,
                      data_seconds=self.data_seconds)


def survey_volume(r_lo=1000.0, r_hi=1800.0, theta_max=math.radians(60.0)) -> float:
    """Volume of the polar-cap shell survey."""
    return 2.0 * math.pi * (1.0 - math.cos(theta_max)) * (r_hi ** 3 - r_lo ** 3) / 3.0
