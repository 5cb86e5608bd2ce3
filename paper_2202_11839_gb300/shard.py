"""One estimate over the ranks of a process group, sharded by moment slot.

The channel fields of different moment slots are independent once the partner fields
(delta, gamma_1, gamma_2) are known (Sec. 3.1.2: every estimator is a sum over its own
harmonic channels).  So a rank builds its plan with a subset of the slots (the plan's
`moments` mask), recomputes the partner fields it needs locally (three grids, cheaper than
sending them), and computes only its slots' channels.  Each normalised row is then complete
on the rank that owns it (its shot noise is subtracted there once), and an all-reduce (sum)
of the (2, LPP_N_MOMENTS, n_bins, 2) FP64 array of normalised and raw rows, each row non-zero on
exactly one rank, gives every rank the whole estimate; the shell counts, mean |k|,
normalisations and shot noises, the same on every rank that computed them, travel in a
second, max all-reduce of 2 n_bins + 6 numbers.

`partition` balances the ranks by channel count (longest first onto the least loaded rank);
`gather` performs the exchange; `sharded_multipoles` runs a rank's plan and gathers.
"""
from __future__ import annotations

import numpy as np

from . import lpp as L

# channels of each moment slot (2L + 1 real harmonics per projected part; the derived slots
# dd0 and plus0 come from the partner fields alone; the density multipoles have one part)
_SLOT_L = {L.LPP_MOM_CROSS2: 2, L.LPP_MOM_CROSS4: 4, L.LPP_MOM_CROSS6: 6, L.LPP_MOM_PLUS2: 2,
           L.LPP_MOM_PLUS4: 4, L.LPP_MOM_MINUS4: 4, L.LPP_MOM_MINUS6: 6, L.LPP_MOM_MINUS8: 8,
           L.LPP_MOM_DD2: 2, L.LPP_MOM_DD4: 4, L.LPP_MOM_MINUS10: 10, L.LPP_MOM_MINUS12: 12}
_CROSS = (L.LPP_MOM_CROSS2, L.LPP_MOM_CROSS4, L.LPP_MOM_CROSS6)
_ONE_PART = (L.LPP_MOM_DD2, L.LPP_MOM_DD4)


def slot_channels(slot: int, cross_b: bool) -> int:
    """Channel fields a plan computes for moment slot `slot`."""
    if slot not in _SLOT_L:
        return 0
    parts = (2 if cross_b else 1) if slot in _CROSS else (1 if slot in _ONE_PART else 2)
    return (2 * _SLOT_L[slot] + 1) * parts


def partition(moments: int, world: int) -> list[int]:
    """Moment masks for ranks 0 .. world-1: every requested slot on exactly one rank, ranks
    balanced by channel count (a slot's weight is its channels + 1, so the derived slots
    also spread).  LPP_WANT_CROSS_B, if set, goes to every rank.  A rank may get 0 (no
    slot: it computes nothing and contributes zeros)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cross_b = bool(moments & L.LPP_WANT_CROSS_B)
    slots = [s for s in range(L.LPP_N_MOMENTS) if moments & (1 << s)]
    slots.sort(key=lambda s: (-(slot_channels(s, cross_b) + 1), s))
    load = [0] * world
    masks = [0] * world
    for s in slots:
        r = min(range(world), key=lambda i: (load[i], i))
        masks[r] |= 1 << s
        load[r] += slot_channels(s, cross_b) + 1
    extra = L.LPP_WANT_CROSS_B if cross_b else 0
    return [m | extra if m else 0 for m in masks]


def gather(est, owned_mask: int, pg=None, device=None):
    """The whole estimate on every rank from each rank's estimate of its own slots.

    est: this rank's estimate (an lpp.Estimate, or any object with its fields), or None when
    the rank owns no slot; owned_mask: its moment mask.  pg: torch.distributed (or None for
    one process); device: where the exchanged tensors live (a CUDA device under NCCL, "cpu"
    under gloo).  Rows the rank does not own are zeroed before the sum, so each row comes
    from its owner alone.  The shell means of |k|, the mode counts, normalisations, shot
    noises and alpha are the same on every rank that computed them (zero elsewhere): a
    maximum over the ranks recovers them.  Returns an lpp.Estimate."""
    if est is None and pg is None:
        raise ValueError("a single process must own every slot")
    nb = est.p.shape[1] if est is not None else 0
    if pg is not None:
        import torch
        n = torch.tensor([nb], dtype=torch.int64, device=device)
        pg.all_reduce(n, op=pg.ReduceOp.MAX)
        nb = int(n.item())
    rows = np.zeros((2, L.LPP_N_MOMENTS, nb, 2))
    meta = np.zeros(2 * nb + 6)
    if est is not None:
        for s in range(L.LPP_N_MOMENTS):
            if owned_mask & (1 << s):
                rows[0, s, :, 0], rows[0, s, :, 1] = np.real(est.p[s]), np.imag(est.p[s])
                rows[1, s, :, 0], rows[1, s, :, 1] = np.real(est.raw[s]), np.imag(est.raw[s])
        meta[:nb] = est.k_mean
        meta[nb:2 * nb] = est.n_modes
        meta[2 * nb:] = [est.norm_auto, est.norm_cross, est.norm_dd, est.shot_plus, est.shot_dd, est.alpha]
    if pg is not None:
        import torch
        t = torch.from_numpy(rows).to(device)
        pg.all_reduce(t)
        m = torch.from_numpy(meta).to(device)
        pg.all_reduce(m, op=pg.ReduceOp.MAX)
        rows, meta = t.cpu().numpy(), m.cpu().numpy()
    return L.Estimate(rows[0, ..., 0] + 1j * rows[0, ..., 1], rows[1, ..., 0] + 1j * rows[1, ..., 1],
                      meta[:nb].copy(), meta[nb:2 * nb].astype(np.int64), *[float(v) for v in meta[2 * nb:]])


def sharded_multipoles(make_plan, assign, moments: int, pg=None, device=None):
    """One estimate with this rank's share of the moment slots.

    make_plan(mask) -> lpp.Plan with that moments mask; assign(plan) attaches the
    catalogues.  Returns (the whole estimate, this rank's mask)."""
    world = pg.get_world_size() if pg is not None else 1
    rank = pg.get_rank() if pg is not None else 0
    mask = partition(moments, world)[rank]
    est = None
    if mask:
        plan = make_plan(mask)
        assign(plan)
        est = plan.multipoles()
    return gather(est, mask, pg, device), mask
