"""Moment-slot sharding of one estimate (paper_2202_11839_gb300/shard.py): the partition
covers every requested slot once and balances the ranks, and two gloo ranks that each hold
an estimate of their own slots end up with the whole estimate.  Each rank's estimate comes
from the FP64 oracle on a small catalogue, the ten tensor-estimator slots and the density
quadrupole and hexadecapole (its rows outside the rank's slots must not leak into the
result)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sh():
    sys.path.insert(0, ROOT)
    from paper_2202_11839_gb300 import lpp as L
    from paper_2202_11839_gb300 import shard as SH
    return L, SH


@pytest.mark.parametrize("with_b", [False, True])
@pytest.mark.parametrize("moments", [0x3FF, 0xFFF, 0x3FFF, 0x3FE, (1 << 5) | (1 << 9) | (1 << 11), 1 << 4,
                                     (1 << 12) | (1 << 13)])
def test_partition_covers_each_slot_once_and_balances(moments, with_b):
    L, SH = _sh()
    extra = L.LPP_WANT_CROSS_B if with_b else 0
    want = moments | extra
    ns = L.LPP_N_MOMENTS
    weight = {s: SH.slot_channels(s, with_b) + 1 for s in range(ns)}
    for world in range(1, 13):
        masks = SH.partition(want, world)
        assert len(masks) == world
        slots = [s for m in masks for s in range(ns) if m & (1 << s)]
        assert sorted(slots) == [s for s in range(ns) if moments & (1 << s)]
        for m in masks:
            assert (m & L.LPP_WANT_CROSS_B) == (extra if m else 0)
        loads = [sum(weight[s] for s in range(ns) if m & (1 << s)) for m in masks]
        assert max(loads) - min(loads) <= max(weight[s] for s in slots)


def test_slot_channels_match_the_plan_tables():
    L, SH = _sh()
    # 133 channels for the ten slots without the B-mode cross parts, 160 with; 5 + 9 more for
    # the density quadrupole and hexadecapole
    assert sum(SH.slot_channels(s, False) for s in range(10)) == 133
    assert sum(SH.slot_channels(s, True) for s in range(10)) == 160
    assert SH.slot_channels(L.LPP_MOM_DD2, True) == 5 and SH.slot_channels(L.LPP_MOM_DD4, False) == 9
    # and 2 x 21 + 2 x 25 for the minus moments L = 10, 12
    assert SH.slot_channels(L.LPP_MOM_MINUS10, False) == 42 and SH.slot_channels(L.LPP_MOM_MINUS12, True) == 50


def _oracle_estimate():
    """Oracle estimate in the library's fourteen slots: the tensor-estimator slots, the density
    l = 2, 4 and the minus moments L = 10, 12."""
    sys.path.insert(0, ROOT)
    from oracle import lpp_oracle as O
    from tests import parity_util as U
    cfg = dict(n=16, box=300.0, observer=(150.0, 150.0, -800.0), scheme=3, interlace=True,
               k_edges=U.default_edges(16, 300.0), oracle_moments=tuple(O.MOMENTS))
    cat = U.make_case("shard", 16, count=1200, seed=7, n_rand=2500)
    ref = U.run_oracle(cfg, cat)
    dens = U.run_oracle_density(cfg, cat)
    # the library's slot order: the oracle's ten default moments, the density l = 2, 4, then
    # the minus moments L = 10, 12
    ref.p = np.concatenate([ref.p[:10], dens.p[1:], ref.p[10:12]])
    ref.raw = np.concatenate([ref.raw[:10], dens.raw[1:], ref.raw[10:12]])
    assert ref.p.shape[0] == 14 and O.MOMENTS[0] == ("dd", 0) and O.MOMENTS[10] == ("minus", 10)
    return ref


def test_single_process_gather_is_the_identity():
    L, SH = _sh()
    ref = _oracle_estimate()
    out = SH.gather(ref, L.LPP_WANT_ALL | L.LPP_WANT_DENSITY | L.LPP_WANT_MINUS_HIGH)
    np.testing.assert_array_equal(out.p, ref.p)
    np.testing.assert_array_equal(out.raw, ref.raw)
    np.testing.assert_array_equal(out.n_modes, ref.n_modes)
    assert out.norm_auto == ref.norm_auto and out.shot_plus == ref.shot_plus


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, moments, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, SH = _sh()
    ref = _oracle_estimate()
    mask = SH.partition(moments, world)[rank]
    mine = None
    if mask:
        # the rank's own estimate: the oracle's rows of its slots, garbage elsewhere (which
        # gather must drop)
        mine = L.Estimate(ref.p.copy(), ref.raw.copy(), ref.k_mean, ref.n_modes, ref.norm_auto, ref.norm_cross,
                          ref.norm_dd, ref.shot_plus, ref.shot_dd, ref.alpha)
        for s in range(L.LPP_N_MOMENTS):
            if not mask & (1 << s):
                mine.p[s] = 1e30 * (rank + 1)
                mine.raw[s] = -1e30
    out = SH.gather(mine, mask, dist, "cpu")
    want = ref.p.copy()
    for s in range(L.LPP_N_MOMENTS):
        if not moments & (1 << s):
            want[s] = 0
    q.put((rank, mask, np.array_equal(out.p, want), np.array_equal(out.n_modes, ref.n_modes),
           out.norm_auto == ref.norm_auto and out.alpha == ref.alpha))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("moments", [0x3FFF, (1 << 5) | (1 << 9)])
def test_two_gloo_ranks_gather_the_whole_estimate(moments):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2 if moments == 0x3FFF else 3       # the second case leaves one rank without a slot
    procs = [ctx.Process(target=_rank, args=(r, world, port, moments, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert any(mask == 0 for _, mask, *_ in out) == (world == 3)
    for rank, mask, p_ok, n_ok, meta_ok in out:
        assert p_ok and n_ok and meta_ok, rank


def _dropout_rank(rank, world, port, q):
    """Rank 1 leaves between steps (after joining the group, before the exchange); rank 0's
    gather must end with an error, not wait for it."""
    import datetime
    import time

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(0)
    L, SH = _sh()
    nb = 4
    zero = np.zeros((L.LPP_N_MOMENTS, nb), dtype=np.complex128)
    est = L.Estimate(zero, zero.copy(), np.zeros(nb), np.zeros(nb, dtype=np.int64), 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    t0 = time.time()
    try:
        SH.gather(est, L.LPP_WANT_ALL, dist, "cpu")
        q.put(("no error", time.time() - t0))
    except Exception as e:   # the peer is gone: the collective fails
        q.put((type(e).__name__, time.time() - t0))
    os._exit(0)


def test_a_rank_that_leaves_ends_the_exchange_with_an_error():
    """Failure detection on the host: one of two gloo ranks exits without joining the
    exchange of a sharded estimate; the other's gather raises within the group's timeout
    (10 s) instead of hanging."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dropout_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    kind, elapsed = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert kind != "no error", kind
    assert elapsed < 60.0, elapsed
