"""Thin ctypes binding of liblpp (include/lpp.h).

Argument marshalling only: every step of the estimator runs in the CUDA library.
Device memory (the plan workspace, device catalogues) and streams come from
PyTorch.  Importing this module raises if liblpp.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LPP_CHECK=1 in the environment selects the bounds-checking build (build.build(check=True))
CHECK_LIB_PATH = os.path.join(_PKG, "liblpp_check.so")
LIB_PATH = CHECK_LIB_PATH if os.environ.get("LPP_CHECK", "0") not in ("", "0") else os.path.join(_PKG, "liblpp.so")

# ----------------------------------------------------------------- constants
LPP_OK, LPP_ERR_INVALID_ARG, LPP_ERR_CUDA, LPP_ERR_NOT_READY, LPP_ERR_WORKSPACE, LPP_ERR_UNSUPPORTED, \
    LPP_ERR_DOMAIN, LPP_ERR_BOUNDS = range(8)
LPP_CIC, LPP_TSC = 2, 3
LPP_FP32, LPP_FP64 = 0, 1
LPP_LOS_LOCAL, LPP_LOS_GLOBAL = 0, 1
LPP_SHAPES, LPP_DENSITY, LPP_RANDOMS = 0, 1, 2
LPP_SHAPE_NONE, LPP_SHAPE_GAMMA12, LPP_SHAPE_TENSOR6 = 0, 1, 2
LPP_N_MOMENTS = 14
LPP_MOM_DD0, LPP_MOM_CROSS2, LPP_MOM_CROSS4, LPP_MOM_CROSS6, LPP_MOM_PLUS0, LPP_MOM_PLUS2, LPP_MOM_PLUS4, \
    LPP_MOM_MINUS4, LPP_MOM_MINUS6, LPP_MOM_MINUS8, LPP_MOM_DD2, LPP_MOM_DD4, LPP_MOM_MINUS10, \
    LPP_MOM_MINUS12 = range(LPP_N_MOMENTS)
MOMENT_NAMES = ["dd0", "cross2", "cross4", "cross6", "plus0", "plus2", "plus4", "minus4", "minus6", "minus8",
                "dd2", "dd4", "minus10", "minus12"]
LPP_WANT_ALL = 0x3FF
LPP_WANT_DD2 = 1 << LPP_MOM_DD2
LPP_WANT_DD4 = 1 << LPP_MOM_DD4
LPP_WANT_DENSITY = LPP_WANT_DD2 | LPP_WANT_DD4
LPP_WANT_MINUS_HIGH = (1 << LPP_MOM_MINUS10) | (1 << LPP_MOM_MINUS12)
TEMPLATE_EB_SLOTS = 0x3FE   # the template slots the derived E/B curves read
GUARD_BYTES, GUARD_VALUE = 4096, 0xA5   # guard bands around a plan workspace that Plan allocates
LPP_WANT_CROSS_B = 1 << 16
KERNEL_KINDS = ["assign", "fft", "combine", "coeffs", "partner", "other"]


class LppError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class PlanDesc(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("box", C.c_double), ("origin", C.c_double * 3), ("observer", C.c_double * 3),
        ("pole", C.c_double * 3), ("scheme", C.c_int), ("interlace", C.c_int), ("compensate", C.c_int),
        ("precision", C.c_int), ("los_proj", C.c_int), ("los_est", C.c_int), ("los_global", C.c_double * 3),
        ("moments", C.c_uint), ("n_bins", C.c_int), ("k_edges", C.POINTER(C.c_double)),
        ("norm_override", C.c_double), ("subtract_shot", C.c_int), ("max_shapes", C.c_longlong),
        ("max_density", C.c_longlong), ("max_randoms", C.c_longlong), ("host_inputs", C.c_int),
        ("batch", C.c_int), ("fused_slots", C.c_int),
    ]


class Particles(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("w", C.c_void_p), ("nbar", C.c_void_p), ("shape", C.c_void_p),
                ("count", C.c_longlong), ("shape_kind", C.c_int), ("on_host", C.c_int)]


class Result(C.Structure):
    _fields_ = [("p", C.POINTER(C.c_double)), ("raw", C.POINTER(C.c_double)), ("k_mean", C.POINTER(C.c_double)),
                ("n_modes", C.POINTER(C.c_longlong)), ("norm_auto", C.c_double), ("norm_cross", C.c_double),
                ("norm_dd", C.c_double), ("shot_plus", C.c_double), ("shot_dd", C.c_double),
                ("alpha", C.c_double)]


EXPORTS = {
    "lpp_plan_create": (C.c_int, [C.POINTER(PlanDesc), C.POINTER(C.c_void_p)]),
    "lpp_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                   C.POINTER(C.c_void_p)]),
    "lpp_batch_destroy": (None, [C.c_void_p]),
    "lpp_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lpp_batch_results": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lpp_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "lpp_batch_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "lpp_plan_destroy": (None, [C.c_void_p]),
    "lpp_plan_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "lpp_plan_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lpp_plan_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lpp_plan_field_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "lpp_assign": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Particles)]),
    "lpp_clear": (C.c_int, [C.c_void_p, C.c_int]),
    "lpp_multipoles": (C.c_int, [C.c_void_p, C.POINTER(Result)]),
    "lpp_window_Q": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double)]),
    "lpp_template_create": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double),
                                      C.c_int, C.c_double, C.POINTER(C.c_void_p)]),
    "lpp_template_destroy": (None, [C.c_void_p]),
    "lpp_template_set_png": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
    "lpp_template_set_slots": (C.c_int, [C.c_void_p, C.c_uint]),
    "lpp_template_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "lpp_template_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "lpp_convolve_template": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lpp_convolve_template_eb": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p]),
    "lpp_surrogate_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "lpp_surrogate_destroy": (None, [C.c_void_p]),
    "lpp_surrogate_workspace_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "lpp_surrogate_set_workspace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_float), C.c_void_p]),
    "lpp_surrogate_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_void_p]),
    "lpp_surrogate_state_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "lpp_surrogate_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "lpp_surrogate_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "lpp_surrogate_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float,
                                      C.c_void_p, C.c_void_p]),
    "lpp_surrogate_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float),
                                          C.POINTER(C.c_double), C.c_void_p]),
    "lpp_surrogate_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lpp_gaussian_sigma": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_void_p]),
    "lpp_surrogate_set_map": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lpp_surrogate_targets": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lpp_surrogate_encode": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lpp_surrogate_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lpp_derive_eb": (C.c_int, [C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_double)]),
    "lpp_plan_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "lpp_plan_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "lpp_plan_path_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "lpp_plan_kernel_stats": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_double)]),
    "lpp_density_monopole_static": (C.c_int, [C.c_int, C.c_double, C.POINTER(C.c_double), C.c_int, C.c_int, C.c_int,
                                              C.c_int, C.c_void_p, C.c_void_p, C.c_longlong, C.c_int,
                                              C.POINTER(C.c_double), C.POINTER(C.c_double),
                                              C.POINTER(C.c_longlong), C.c_void_p]),
    "lpp_window_Q_pairs_workspace_size": (C.c_int, [C.c_int, C.POINTER(C.c_size_t)]),
    "lpp_window_Q_pairs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.POINTER(C.c_double),
                                     C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.c_void_p, C.c_size_t, C.c_void_p]),
    "lpp_status_string": (C.c_char_p, [C.c_int]),
    "lpp_plan_last_error": (C.c_char_p, [C.c_void_p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblpp.so; raises ImportError if it is missing (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} not built at {path}: run paper_2202_11839_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(lib, status: int, plan=None):
    if status != LPP_OK:
        msg = lib.lpp_status_string(status).decode()
        if plan:
            extra = lib.lpp_plan_last_error(plan).decode()
            if extra:
                msg += ": " + extra
        raise LppError(status, msg)


def _ptr(a):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


@dataclass
class Estimate:
    p: np.ndarray          # (LPP_N_MOMENTS, nb) complex, normalised
    raw: np.ndarray        # (LPP_N_MOMENTS, nb) complex
    k_mean: np.ndarray
    n_modes: np.ndarray
    norm_auto: float
    norm_cross: float
    norm_dd: float
    shot_plus: float
    shot_dd: float
    alpha: float
    extra: dict = field(default_factory=dict)


class Plan:
    """An LPP estimator plan on the current CUDA device.

    ``workspace`` must be a 256-byte aligned device buffer (a torch uint8 tensor) of at
    least ``workspace_bytes`` bytes; it is allocated here with torch if not given.
    """

    def __init__(self, n: int, box: float, k_edges, *, origin=(0.0, 0.0, 0.0), observer=(0.0, 0.0, 0.0),
                 pole=(-1.0, 0.0, 0.0), scheme: int = LPP_CIC, interlace: bool = False, compensate: bool = True,
                 precision: int = LPP_FP32, los_proj: int = LPP_LOS_LOCAL, los_est: int = LPP_LOS_LOCAL,
                 los_global=(0.0, 0.0, 1.0), moments: int = LPP_WANT_ALL, norm_override: float = 0.0,
                 subtract_shot: bool = True, max_shapes: int = 0, max_density: int = 0, max_randoms: int = 0,
                 host_inputs: bool = False, batch: int = 0, fused_slots: int = 0, stream=None, workspace=None,
                 device=None):
        import torch
        self.lib = load_library()
        self.torch = torch
        self.edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        self.nb = len(self.edges) - 1
        d = PlanDesc()
        d.n, d.box = n, box
        d.origin[:] = origin
        d.observer[:] = observer
        d.pole[:] = pole
        d.scheme, d.interlace, d.compensate, d.precision = scheme, int(interlace), int(compensate), precision
        d.los_proj, d.los_est = los_proj, los_est
        d.los_global[:] = los_global
        d.moments = moments
        d.n_bins = self.nb
        d.k_edges = self.edges.ctypes.data_as(C.POINTER(C.c_double))
        d.norm_override, d.subtract_shot = norm_override, int(subtract_shot)
        d.max_shapes, d.max_density, d.max_randoms = max_shapes, max_density, max_randoms
        d.host_inputs, d.batch, d.fused_slots = int(host_inputs), batch, fused_slots
        self.desc = d
        self.precision = precision
        self.dtype = np.float64 if precision == LPP_FP64 else np.float32
        self.tdtype = torch.float64 if precision == LPP_FP64 else torch.float32
        h = C.c_void_p()
        _check(self.lib, self.lib.lpp_plan_create(C.byref(d), C.byref(h)))
        self.h = h
        sz = C.c_size_t()
        _check(self.lib, self.lib.lpp_plan_workspace_size(h, C.byref(sz)), h)
        self.workspace_bytes = sz.value
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(self.lib, self.lib.lpp_plan_set_stream(h, C.c_void_p(self.stream.cuda_stream)), h)
        self._guard = None
        if workspace is None:
            # own allocation: the workspace sits between two guard bands of a fixed byte pattern
            # (GUARD_BYTES before, at least as many after) that guard_intact() checks
            workspace = torch.empty(self.workspace_bytes + 256 + 2 * GUARD_BYTES, dtype=torch.uint8, device=self.device)
            workspace.fill_(GUARD_VALUE)
            addr = workspace.data_ptr()
            off = (-(addr + GUARD_BYTES)) % 256 + GUARD_BYTES
            self._guard = (off, off + self.workspace_bytes)
        else:
            addr = workspace.data_ptr()
            off = (-addr) % 256
        self.workspace = workspace
        size = self.workspace_bytes if self._guard else workspace.numel() - off
        _check(self.lib, self.lib.lpp_plan_set_workspace(h, C.c_void_p(addr + off), C.c_size_t(size)), h)
        self._keep = {}
        if os.environ.get("LPP_TIMING", "0") not in ("", "0"):
            self.set_timing(True)   # per-kernel CUDA-event timers from the start (kernel_stats)

    def guard_intact(self) -> bool:
        """True when the guard bands around a workspace this plan allocated still hold their
        pattern (nothing of the library wrote outside its workspace); True for a caller's buffer."""
        if self._guard is None:
            return True
        lo, hi = self._guard
        self.torch.cuda.synchronize(self.device)
        return bool((self.workspace[:lo] == GUARD_VALUE).all().item()) and \
            bool((self.workspace[hi:] == GUARD_VALUE).all().item())

    def field_count(self) -> int:
        v = C.c_int()
        _check(self.lib, self.lib.lpp_plan_field_count(self.h, C.byref(v)), self.h)
        return v.value

    def set_timing(self, on: bool = True):
        _check(self.lib, self.lib.lpp_plan_set_timing(self.h, int(on)), self.h)

    def launch_count(self) -> int:
        """Kernels the last estimate launched."""
        v = C.c_longlong()
        _check(self.lib, self.lib.lpp_plan_launch_count(self.h, C.byref(v)), self.h)
        return v.value

    def path_stats(self) -> dict:
        """Forms of the fused assignment pass the last estimate ran (lpp_plan_path_stats)."""
        v = (C.c_longlong * 6)()
        _check(self.lib, self.lib.lpp_plan_path_stats(self.h, v), self.h)
        keys = ("one_slot_launches", "two_slot_launches", "two_slot_fixed_tiles", "two_slot_float_tiles",
                "one_slot_fixed_tiles", "one_slot_float_tiles")
        return dict(zip(keys, list(v)))

    def kernel_stats(self) -> dict:
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            ms, nl, b = C.c_double(), C.c_longlong(), C.c_double()
            _check(self.lib, self.lib.lpp_plan_kernel_stats(self.h, k, C.byref(ms), C.byref(nl), C.byref(b)), self.h)
            out[name] = {"ms": ms.value, "launches": nl.value, "bytes": b.value}
        return out

    def assign(self, role: int, pos, w=None, nbar=None, shape=None, shape_kind: int = LPP_SHAPE_NONE):
        """Attach a catalogue: torch CUDA tensors (referenced) or numpy arrays (copied)."""
        on_host = not hasattr(pos, "data_ptr") or not pos.is_cuda
        arrs = [pos, w, nbar, shape]
        for a in arrs:
            if a is None:
                continue
            if hasattr(a, "data_ptr"):
                if a.dtype != self.tdtype or not a.is_contiguous():
                    raise ValueError("catalogue tensors must be contiguous and match the plan precision")
            else:
                if a.dtype != self.dtype or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("catalogue arrays must be C-contiguous and match the plan precision")
        count = int(pos.shape[-1])
        p = Particles(_ptr(pos), _ptr(w), _ptr(nbar), _ptr(shape), count, shape_kind, int(on_host))
        self._keep[role] = arrs
        _check(self.lib, self.lib.lpp_assign(self.h, role, C.byref(p)), self.h)

    def clear(self, role: int):
        _check(self.lib, self.lib.lpp_clear(self.h, role), self.h)
        self._keep.pop(role, None)

    def multipoles(self) -> Estimate:
        nb = self.nb
        p = np.zeros((LPP_N_MOMENTS, nb, 2))
        raw = np.zeros((LPP_N_MOMENTS, nb, 2))
        km = np.zeros(nb)
        nm = np.zeros(nb, dtype=np.int64)
        r = Result()
        r.p = p.ctypes.data_as(C.POINTER(C.c_double))
        r.raw = raw.ctypes.data_as(C.POINTER(C.c_double))
        r.k_mean = km.ctypes.data_as(C.POINTER(C.c_double))
        r.n_modes = nm.ctypes.data_as(C.POINTER(C.c_longlong))
        _check(self.lib, self.lib.lpp_multipoles(self.h, C.byref(r)), self.h)
        return Estimate(p[..., 0] + 1j * p[..., 1], raw[..., 0] + 1j * raw[..., 1], km, nm, r.norm_auto,
                        r.norm_cross, r.norm_dd, r.shot_plus, r.shot_dd, r.alpha)

    def particles(self, role: int, pos, w=None, nbar=None, shape=None, shape_kind: int = LPP_SHAPE_NONE):
        """A device catalogue descriptor for lpp_batch_create (tensors are not copied)."""
        for a in (pos, w, nbar, shape):
            if a is not None and (not hasattr(a, "data_ptr") or not a.is_cuda or a.dtype != self.tdtype
                                  or not a.is_contiguous()):
                raise ValueError("batch catalogues must be contiguous CUDA tensors of the plan precision")
        count = int(pos.shape[-1]) if pos is not None else 0
        return Particles(_ptr(pos), _ptr(w), _ptr(nbar), _ptr(shape), count, shape_kind, 0)

    def window_q(self, s_edges):
        """Window multipoles Q_l(s), l = 0..8 even, from the assigned randoms: (q[5, nb], s_mean, n_points, I)."""
        e = np.ascontiguousarray(s_edges, dtype=np.float64)
        nb = len(e) - 1
        q = np.zeros((5, nb))
        sm = np.zeros(nb)
        npt = np.zeros(nb, dtype=np.int64)
        norm = C.c_double()
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(self.lib, self.lib.lpp_window_Q(self.h, nb, dp(e), dp(q), dp(sm),
                                               npt.ctypes.data_as(C.POINTER(C.c_longlong)), C.byref(norm)), self.h)
        return q, sm, npt, norm.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lpp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Template:
    """Window-convolved template evaluator (lpp_template_*): tables built once, many parameter sets."""

    def __init__(self, q_table, s, k_edges, shot_plus: float = 0.0, stream=None, device=None):
        import torch
        self.lib = load_library()
        q = np.ascontiguousarray(q_table, dtype=np.float64)
        sv = np.ascontiguousarray(s, dtype=np.float64)
        e = np.ascontiguousarray(k_edges, dtype=np.float64)
        self.k_edges = e
        self.shot_plus = float(shot_plus)
        self.nb = len(e) - 1
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        h = C.c_void_p()
        _check(self.lib, self.lib.lpp_template_create(dp(q), dp(sv), sv.size, dp(e), self.nb, shot_plus, C.byref(h)))
        self.h = h
        sz = C.c_size_t()
        _check(self.lib, self.lib.lpp_template_workspace_size(h, C.byref(sz)))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(sz.value + 256, dtype=torch.uint8, device=self.device)
        addr = self.workspace.data_ptr()
        off = (-addr) % 256
        _check(self.lib, self.lib.lpp_template_set_workspace(h, C.c_void_p(addr + off), C.c_size_t(sz.value),
                                                             C.c_void_p(self.stream.cuda_stream)))

    def set_png(self, f_nl: float, db_ia: float = 0.17, omega_m: float = 0.3):
        """Spin-2 PNG response of the shape spectra (lpp_template_set_png); f_nl = 0: Gaussian."""
        _check(self.lib, self.lib.lpp_template_set_png(self.h, float(f_nl), float(db_ia), float(omega_m)))

    def set_slots(self, mask: int):
        """Output slots to compute (lpp_template_set_slots); the others come back as zeros."""
        _check(self.lib, self.lib.lpp_template_set_slots(self.h, int(mask)))

    def __call__(self, params, out=None):
        """params: torch float64 CUDA tensor [n, 6]; returns a [n, LPP_N_MOMENTS, nb] float64 CUDA tensor."""
        import torch
        n = int(params.shape[0])
        if out is None:
            out = torch.empty((n, LPP_N_MOMENTS, self.nb), dtype=torch.float64, device=params.device)
        _check(self.lib, self.lib.lpp_convolve_template(self.h, C.c_void_p(params.data_ptr()), n,
                                                        C.c_void_p(out.data_ptr()),
                                                        C.c_void_p(self.stream.cuda_stream)))
        return out

    def derived(self, params, ref=None, sigma=None, out=None):
        """Native slots [n, LPP_N_MOMENTS, nb] (float64) and standardised derived curves [n, 8 * nb]
        (float32); the template's slot mask must hold TEMPLATE_EB_SLOTS."""
        import torch
        n = int(params.shape[0])
        if out is None:
            out = torch.empty((n, LPP_N_MOMENTS, self.nb), dtype=torch.float64, device=params.device)
        eb = torch.empty((n, 8 * self.nb), dtype=torch.float32, device=params.device)
        ptr = lambda a: C.c_void_p(a.data_ptr()) if a is not None else None
        _check(self.lib, self.lib.lpp_convolve_template_eb(self.h, ptr(params), n, ptr(out), ptr(eb), ptr(ref),
                                                           ptr(sigma), C.c_void_p(self.stream.cuda_stream)))
        return out, eb

    def close(self):
        if getattr(self, "h", None):
            self.lib.lpp_template_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SURROGATE_SIZES = (6, 256, 256, 256, 256, 320)


def flatten_params(layers) -> np.ndarray:
    """[(W [out, in], b [out]), ...] -> the FP32 parameter array of the C ABI."""
    return np.ascontiguousarray(np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers]),
                                dtype=np.float32)


def unflatten_params(flat):
    out, p = [], 0
    for fi, fo in zip(SURROGATE_SIZES[:-1], SURROGATE_SIZES[1:]):
        w = flat[p:p + fo * fi].reshape(fo, fi)
        p += fo * fi
        b = flat[p:p + fo]
        p += fo
        out.append((w, b))
    return out


class SurrogateMap(C.Structure):
    _fields_ = [("lo", C.c_double * 6), ("hi", C.c_double * 6), ("feed", C.c_int * 6), ("mu", C.c_void_p),
                ("sd", C.c_void_p), ("shot", C.c_void_p), ("ref", C.c_void_p), ("sigma", C.c_void_p),
                ("base", C.c_void_p), ("base_nodes", C.c_int), ("base_in", C.c_int * 2)]


class Surrogate:
    """The template surrogate network (lpp_surrogate_*) on the current CUDA device."""

    def __init__(self, params_flat, batch: int = 256, stream=None, device=None):
        import torch
        self.lib = load_library()
        self.batch = batch
        h = C.c_void_p()
        _check(self.lib, self.lib.lpp_surrogate_create(batch, C.byref(h)))
        self.h = h
        sz = C.c_size_t()
        _check(self.lib, self.lib.lpp_surrogate_workspace_size(h, C.byref(sz)))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(sz.value + 256, dtype=torch.uint8, device=self.device)
        addr = self.workspace.data_ptr()
        off = (-addr) % 256
        p = np.ascontiguousarray(params_flat, dtype=np.float32)
        _check(self.lib, self.lib.lpp_surrogate_set_workspace(h, C.c_void_p(addr + off), C.c_size_t(sz.value),
                                                              p.ctypes.data_as(C.POINTER(C.c_float)),
                                                              C.c_void_p(self.stream.cuda_stream)))

    def params(self) -> np.ndarray:
        n = sum(fo * fi + fo for fi, fo in zip(SURROGATE_SIZES[:-1], SURROGATE_SIZES[1:]))
        out = np.zeros(n, dtype=np.float32)
        _check(self.lib, self.lib.lpp_surrogate_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)),
                                                           C.c_void_p(self.stream.cuda_stream)))
        return out

    def save_state(self) -> np.ndarray:
        """The training state (lpp_surrogate_save_state) as a uint8 array."""
        sz = C.c_size_t()
        _check(self.lib, self.lib.lpp_surrogate_state_size(self.h, C.byref(sz)))
        buf = np.zeros(sz.value, dtype=np.uint8)
        _check(self.lib, self.lib.lpp_surrogate_save_state(self.h, C.c_void_p(buf.ctypes.data), C.c_size_t(sz.value),
                                                           C.c_void_p(self.stream.cuda_stream)))
        return buf

    def load_state(self, state):
        """Restore a state from save_state (lpp_surrogate_load_state)."""
        buf = np.ascontiguousarray(state, dtype=np.uint8)
        _check(self.lib, self.lib.lpp_surrogate_load_state(self.h, C.c_void_p(buf.ctypes.data), C.c_size_t(buf.size),
                                                           C.c_void_p(self.stream.cuda_stream)))

    def train(self, x, y, schedule, lr: float, losses=None):
        """x, y: float32 CUDA tensors; schedule: int32 CUDA tensor [n_steps * batch]."""
        n_steps = int(schedule.numel()) // self.batch
        _check(self.lib, self.lib.lpp_surrogate_train(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                      C.c_void_p(schedule.data_ptr()), n_steps, float(lr),
                                                      C.c_void_p(losses.data_ptr()) if losses is not None else None,
                                                      C.c_void_p(self.stream.cuda_stream)))

    def gradients(self, x, y, idx):
        n = sum(fo * fi + fo for fi, fo in zip(SURROGATE_SIZES[:-1], SURROGATE_SIZES[1:]))
        g = np.zeros(n, dtype=np.float32)
        loss = C.c_double()
        _check(self.lib, self.lib.lpp_surrogate_gradients(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                          C.c_void_p(idx.data_ptr()),
                                                          g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss),
                                                          C.c_void_p(self.stream.cuda_stream)))
        return g, loss.value

    def infer(self, x, out=None):
        import torch
        n = int(x.shape[0])
        if out is None:
            out = torch.empty((n, 320), dtype=torch.float32, device=x.device)
        _check(self.lib, self.lib.lpp_surrogate_infer(self.h, C.c_void_p(x.data_ptr()), n, C.c_void_p(out.data_ptr()),
                                                      C.c_void_p(self.stream.cuda_stream)))
        return out

    def set_map(self, lo, hi, feed, mu, sd, shot, ref=None, sigma=None, base=None, base_nodes=0, base_in=(3, 4)):
        """Parameter box, fed inputs and the output map (mu, sd, shot, ref, sigma, base: FP64
        CUDA tensors, kept alive by this object)."""
        m = SurrogateMap()
        for c in range(6):
            m.lo[c], m.hi[c], m.feed[c] = float(lo[c]), float(hi[c]), int(feed[c])
        ptr = lambda a: a.data_ptr() if a is not None else None
        m.mu, m.sd, m.shot, m.ref, m.sigma = ptr(mu), ptr(sd), ptr(shot), ptr(ref), ptr(sigma)
        m.base, m.base_nodes = ptr(base), int(base_nodes)
        m.base_in[0], m.base_in[1] = int(base_in[0]), int(base_in[1])
        self._map_refs = (mu, sd, shot, ref, sigma, base)
        _check(self.lib, self.lib.lpp_surrogate_set_map(self.h, C.byref(m)))

    def targets(self, params, native, out=None):
        import torch
        n = int(params.shape[0])
        if out is None:
            out = torch.empty((n, 320), dtype=torch.float32, device=params.device)
        _check(self.lib, self.lib.lpp_surrogate_targets(self.h, C.c_void_p(params.data_ptr()),
                                                        C.c_void_p(native.data_ptr()), n, C.c_void_p(out.data_ptr()),
                                                        C.c_void_p(self.stream.cuda_stream)))
        return out

    def encode(self, params, out=None):
        import torch
        n = int(params.shape[0])
        if out is None:
            out = torch.empty((n, 6), dtype=torch.float32, device=params.device)
        _check(self.lib, self.lib.lpp_surrogate_encode(self.h, C.c_void_p(params.data_ptr()), n,
                                                       C.c_void_p(out.data_ptr()), C.c_void_p(self.stream.cuda_stream)))
        return out

    def predict(self, params, out=None):
        """Emulated standardised derived curves [n, 320] (FP32) for FP64 params [n, 6]."""
        import torch
        n = int(params.shape[0])
        if out is None:
            out = torch.empty((n, 320), dtype=torch.float32, device=params.device)
        _check(self.lib, self.lib.lpp_surrogate_predict(self.h, C.c_void_p(params.data_ptr()), n,
                                                        C.c_void_p(out.data_ptr()),
                                                        C.c_void_p(self.stream.cuda_stream)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.lpp_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def window_q_pairs(pos, w, nbar, observer, s_edges, alpha: float = 1.0, box: float = 0.0, stream=None):
    """Window multipoles Q_l(s), l = 0..8 even, by pair counting (lpp_window_Q_pairs): pos, w,
    nbar are FP64 CUDA tensors ([3, n], [n] or None, [n] or None).  Returns q [5, n_s]."""
    import torch
    lib = load_library()
    e = np.ascontiguousarray(s_edges, dtype=np.float64)
    ns = len(e) - 1
    sz = C.c_size_t()
    _check(lib, lib.lpp_window_Q_pairs_workspace_size(ns, C.byref(sz)))
    ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=pos.device)
    addr = ws.data_ptr() + (-ws.data_ptr()) % 256
    for a in (pos, w, nbar):
        if a is not None and (a.dtype != torch.float64 or not a.is_contiguous() or not a.is_cuda):
            raise ValueError("pair-count inputs must be contiguous FP64 CUDA tensors")
    obs = (C.c_double * 3)(*observer)
    q = np.zeros((5, ns))
    st = stream if stream is not None else torch.cuda.current_stream(pos.device)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(lib, lib.lpp_window_Q_pairs(_ptr(pos), _ptr(w), _ptr(nbar), int(pos.shape[1]), obs, float(box),
                                       float(alpha), ns, dp(e), dp(q), C.c_void_p(addr), C.c_size_t(sz.value),
                                       C.c_void_p(st.cuda_stream)))
    return q


def derive_eb(p: np.ndarray):
    """Legendre multipoles (gE l=0,2; EE, BB l=0,2,4) from normalised native moments (>= 10, nb) complex."""
    lib = load_library()
    nb = p.shape[1]
    pr = np.ascontiguousarray(np.stack([p.real, p.imag], axis=-1), dtype=np.float64)
    ge = np.zeros((2, nb))
    ee = np.zeros((3, nb))
    bb = np.zeros((3, nb))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(lib, lib.lpp_derive_eb(dp(pr), nb, dp(ge), dp(ee), dp(bb)))
    return ge, ee, bb


def gaussian_sigma(p0: np.ndarray, k_edges, volume: float, noise_g: float, noise_e: float) -> np.ndarray:
    """Gaussian error bars [8, nb] of the derived multipoles from the monopoles p0 [4, nb]
    (P_gg, P_gE, P_EE, P_BB without shot noise) (lpp_gaussian_sigma)."""
    lib = load_library()
    p = np.ascontiguousarray(p0, dtype=np.float64).reshape(4, -1)
    nb = p.shape[1]
    k = np.ascontiguousarray(k_edges, dtype=np.float64)
    out = np.zeros((8, nb))
    dp = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(lib, lib.lpp_gaussian_sigma(dp(p), dp(k), nb, float(volume), float(noise_g), float(noise_e), dp(out)))
    return out


class Batch:
    """Many catalogues through a set of plans in one launch (lpp_batch_*), optionally one CUDA graph."""

    def __init__(self, plans, plan_of, shapes, randoms=None, use_graph: bool = True, keep=None):
        self.lib = load_library()
        self.plans = list(plans)
        self.plan_of = list(plan_of)
        self._keep = keep                 # the tensors behind the descriptors
        n = len(self.plan_of)
        ph = (C.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        po = (C.c_int * n)(*self.plan_of)
        sh = (Particles * n)(*shapes)
        rd = (Particles * n)(*randoms) if randoms is not None else None
        h = C.c_void_p()
        st = self.lib.lpp_batch_create(ph, len(self.plans), po, sh, rd, n, int(use_graph), C.byref(h))
        if st != LPP_OK:
            raise LppError(st, self.lib.lpp_status_string(st).decode())
        self.h = h

    def _check(self, st):
        if st != LPP_OK:
            raise LppError(st, self.lib.lpp_status_string(st).decode() + ": " +
                           self.lib.lpp_batch_last_error(self.h).decode())

    def launch(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.lpp_batch_launch(self.h, C.c_void_p(s.cuda_stream)))

    def results(self):
        n = len(self.plan_of)
        bufs = []
        rs = (Result * n)()
        for j in range(n):
            nb = self.plans[self.plan_of[j]].nb
            p = np.zeros((LPP_N_MOMENTS, nb, 2))
            raw = np.zeros((LPP_N_MOMENTS, nb, 2))
            km = np.zeros(nb)
            nm = np.zeros(nb, dtype=np.int64)
            rs[j].p = p.ctypes.data_as(C.POINTER(C.c_double))
            rs[j].raw = raw.ctypes.data_as(C.POINTER(C.c_double))
            rs[j].k_mean = km.ctypes.data_as(C.POINTER(C.c_double))
            rs[j].n_modes = nm.ctypes.data_as(C.POINTER(C.c_longlong))
            bufs.append((p, raw, km, nm))
        self._check(self.lib.lpp_batch_results(self.h, rs))
        out = []
        for j, (p, raw, km, nm) in enumerate(bufs):
            r = rs[j]
            out.append(Estimate(p[..., 0] + 1j * p[..., 1], raw[..., 0] + 1j * raw[..., 1], km, nm, r.norm_auto,
                                r.norm_cross, r.norm_dd, r.shot_plus, r.shot_dd, r.alpha))
        return out

    def launch_count(self):
        """(kernels the mocks' estimates enqueued, kernel nodes of the captured graph or -1)."""
        a, b = C.c_longlong(), C.c_longlong()
        self._check(self.lib.lpp_batch_launch_count(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.lpp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
