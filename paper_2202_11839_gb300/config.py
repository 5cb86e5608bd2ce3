"""Plan descriptors from JSON configurations: the lpp_plan_desc fields by name.

A configuration is a JSON object with the grid (`n`, `box`, optional `origin`), the
geometry (`observer`, `pole`, `los_proj`, `los_est`, `los_global`: "local" / "global"), the
assignment (`scheme`: "cic" / "tsc", `interlace`, `compensate`), `precision` ("fp32" /
"fp64"), the shells (`k_edges`: a list of edges, or {"lo", "hi", "n"} for n linear shells),
`moments` (slot names as in lpp.MOMENT_NAMES, or "all" for the ten of LPP_WANT_ALL, plus
"cross_b" for the B parts of the cross moments), the capacities (`max_shapes`,
`max_density`, `max_randoms`) and the tuning fields (`batch`, `fused_slots`).  Missing fields
take the library defaults.  `configs/` holds the workloads of the benchmark and the tests.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import lpp as L

CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")
_SCHEMES = {"cic": L.LPP_CIC, "tsc": L.LPP_TSC}
_PRECISIONS = {"fp32": L.LPP_FP32, "fp64": L.LPP_FP64}
_LOS = {"local": L.LPP_LOS_LOCAL, "global": L.LPP_LOS_GLOBAL}
_KEYS = {"n", "box", "origin", "observer", "pole", "scheme", "interlace", "compensate", "precision", "los_proj",
         "los_est", "los_global", "k_edges", "moments", "norm_override", "subtract_shot", "max_shapes",
         "max_density", "max_randoms", "host_inputs", "batch", "fused_slots", "name", "comment"}


def load(name_or_path: str) -> dict:
    """A configuration by file path, or by name from configs/ (with or without .json)."""
    path = name_or_path
    if not os.path.exists(path):
        path = os.path.join(CONFIG_DIR, name_or_path if name_or_path.endswith(".json") else name_or_path + ".json")
    with open(path) as f:
        return json.load(f)


def moment_mask(names) -> int:
    """The lpp_plan_desc.moments bitmask of a list of slot names ("all", "cross_b" allowed)."""
    if isinstance(names, str):
        names = [names]
    mask = 0
    for nm in names:
        if nm == "all":
            mask |= L.LPP_WANT_ALL
        elif nm == "cross_b":
            mask |= L.LPP_WANT_CROSS_B
        elif nm in L.MOMENT_NAMES:
            mask |= 1 << L.MOMENT_NAMES.index(nm)
        else:
            raise ValueError(f"unknown moment slot {nm!r}")
    return mask


def edges(spec) -> np.ndarray:
    if isinstance(spec, dict):
        return np.linspace(float(spec["lo"]), float(spec["hi"]), int(spec["n"]) + 1)
    e = np.asarray(spec, dtype=np.float64)
    if e.ndim != 1 or e.size < 2 or not np.all(np.diff(e) > 0):
        raise ValueError("k_edges must increase")
    return e


def plan_args(cfg: dict):
    """(n, box, k_edges, keyword arguments of lpp.Plan) for a configuration."""
    unknown = set(cfg) - _KEYS
    if unknown:
        raise ValueError(f"unknown configuration fields: {sorted(unknown)}")
    kw = {}
    for k in ("origin", "observer", "pole", "los_global"):
        if k in cfg:
            v = tuple(float(x) for x in cfg[k])
            if len(v) != 3:
                raise ValueError(f"{k} needs three components")
            kw[k] = v
    if "scheme" in cfg:
        kw["scheme"] = _SCHEMES[cfg["scheme"].lower()]
    if "precision" in cfg:
        kw["precision"] = _PRECISIONS[cfg["precision"].lower()]
    for k in ("los_proj", "los_est"):
        if k in cfg:
            kw[k] = _LOS[cfg[k].lower()]
    for k in ("interlace", "compensate", "subtract_shot", "host_inputs"):
        if k in cfg:
            kw[k] = bool(cfg[k])
    for k in ("max_shapes", "max_density", "max_randoms", "batch", "fused_slots"):
        if k in cfg:
            kw[k] = int(cfg[k])
    if "norm_override" in cfg:
        kw["norm_override"] = float(cfg["norm_override"])
    if "moments" in cfg:
        kw["moments"] = moment_mask(cfg["moments"])
    return int(cfg["n"]), float(cfg["box"]), edges(cfg["k_edges"]), kw


def plan_from_config(cfg, **overrides) -> L.Plan:
    """An lpp.Plan from a configuration (dict, file path or name); overrides take precedence."""
    if not isinstance(cfg, dict):
        cfg = load(cfg)
    n, box, e, kw = plan_args(cfg)
    kw.update(overrides)
    return L.Plan(n, box, e, **kw)
