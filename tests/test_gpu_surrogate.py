"""The surrogate network's CUDA kernels against the FP64 oracle (same BF16 rounding points).

Tolerances: both sides round the same operands to BF16; the GPU accumulates in FP32 and may
round an activation or gradient to the neighbouring BF16 value where the FP32 and FP64 sums
straddle a rounding boundary (relative 2^-8 on that element).  Norm-wise relative errors of
a few 1e-3 cover that; index or transpose mistakes give O(1) errors.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2202_11839_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _setup(batch=64, seed=5):
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    layers = S.surrogate_init(seed)
    rng = np.random.default_rng(seed)
    layers = [(w, (rng.standard_normal(b.shape) * 0.05).astype(np.float32)) for w, b in layers]
    x = rng.uniform(-1, 1, (batch, 6)).astype(np.float32)
    y = rng.standard_normal((batch, 320)).astype(np.float32)
    net = L.Surrogate(L.flatten_params(layers), batch=batch)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return L, net, layers, x, y, t


def _oracle_params(layers):
    return [w.astype(np.float64) for w, b in layers], [b.astype(np.float64) for w, b in layers]


def test_forward_matches_oracle():
    L, net, layers, x, y, t = _setup()
    out = net.infer(t(x)).cpu().numpy()
    ws, bs = _oracle_params(layers)
    ref, _ = M.forward(ws, bs, x.astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 2e-3
    net.close()


def test_gradients_match_oracle():
    import torch
    L, net, layers, x, y, t = _setup()
    idx = t(np.arange(64, dtype=np.int32))
    g, loss = net.gradients(t(x), t(y), idx)
    ws, bs = _oracle_params(layers)
    rl, gws, gbs = M.loss_and_grads(ws, bs, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - rl) <= 1e-4 * rl
    got = L.unflatten_params(g)
    for li in range(5):
        gw, gb = got[li]
        ew = np.linalg.norm(gw - gws[li]) / np.linalg.norm(gws[li])
        eb = np.linalg.norm(gb - gbs[li]) / np.linalg.norm(gbs[li])
        assert ew < 5e-3 and eb < 5e-3, (li, ew, eb)
    # the network is unchanged by the gradient call
    np.testing.assert_array_equal(net.params(), L.flatten_params(layers))
    net.close()


def test_one_adam_step_matches_oracle():
    import torch
    L, net, layers, x, y, t = _setup()
    sched = t(np.arange(64, dtype=np.int32))
    losses = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.train(t(x), t(y), sched, 1e-3, losses)
    torch.cuda.synchronize()
    ws, bs = _oracle_params(layers)
    rl, gws, gbs = M.loss_and_grads(ws, bs, x.astype(np.float64), y.astype(np.float64))
    st = M.adam_state(ws, bs)
    M.adam_step(ws, bs, gws, gbs, st, lr=1e-3)
    got = L.unflatten_params(net.params())
    for li in range(5):
        w0, b0 = layers[li]
        dw_gpu = got[li][0] - w0
        dw_ref = ws[li] - w0
        # Adam's first step is +-lr per element wherever the gradient is not tiny; compare the moves
        agree = np.mean(np.sign(dw_gpu) == np.sign(dw_ref))
        assert agree > 0.99, (li, agree)
        assert np.max(np.abs(dw_gpu - dw_ref)) < 1.5e-3
    assert abs(float(losses[0]) - rl) <= 1e-4 * rl
    net.close()


def test_training_reduces_the_loss():
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    rng = np.random.default_rng(8)
    n = 2048
    x = rng.uniform(-1, 1, (n, 6)).astype(np.float32)
    basis = rng.standard_normal((6, 320)).astype(np.float32) / 3
    y = np.tanh(x @ basis).astype(np.float32)
    net = L.Surrogate(L.flatten_params(S.surrogate_init(1)), batch=128)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    steps = 400
    sched = np.concatenate([rng.permutation(n)[:128] for _ in range(steps)]).astype(np.int32)
    losses = torch.zeros(steps, dtype=torch.float64, device="cuda")
    net.train(t(x), t(y), t(sched), 2e-3, losses)
    l = losses.cpu().numpy()
    assert l[-20:].mean() < 0.05 * l[:5].mean(), (l[:5], l[-20:])
    net.close()


# ------------------------------------------------------------------ the template emulator
def _window_table():
    s = np.linspace(5.0, 3600.0, 360)
    amp = np.array([1.0, -0.12, 0.05, -0.02, 0.008])
    q = amp[:, None] * np.exp(-(s / 1200.0) ** 2)[None, :] * (1.0 + 0.3 * np.cos(s / 400.0))[None, :]
    return q, s


SURVEY_NOISE_G = 5.06e9 / 1.5e6
SURVEY_SHOT_PLUS = 2 * 0.25 ** 2 * SURVEY_NOISE_G


def _template():
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    q, s = _window_table()
    return L.Template(q, s, np.linspace(0.0, 0.2, 41), shot_plus=SURVEY_SHOT_PLUS)


def test_template_derived_curves_match_host_derivation():
    """The template kernel's derived curves equal lpp_derive_eb applied to its native slots,
    and its standardisation is (value - ref) / sigma."""
    import torch
    from paper_2202_11839_gb300 import lpp as L
    tm = _template()
    params = S.latin_hypercube(5, seed=9)
    th = torch.from_numpy(params).cuda()
    native, eb = tm.derived(th)
    native = native.cpu().numpy()
    eb = eb.double().cpu().numpy()
    rng = np.random.default_rng(2)
    ref = rng.standard_normal(320) * 100.0
    sig = rng.uniform(1.0, 50.0, 320)
    _, ebs = tm.derived(th, ref=torch.from_numpy(ref).cuda(), sigma=torch.from_numpy(sig).cuda())
    ebs = ebs.double().cpu().numpy()
    for i in range(5):
        ge, ee, bb = L.derive_eb(native[i].astype(np.complex128))
        want = np.concatenate([ge, ee, bb]).reshape(-1)
        scale = np.abs(want).max()
        assert np.abs(eb[i] - want).max() < 1e-6 * scale
        np.testing.assert_allclose(ebs[i], (want - ref) / sig, rtol=1e-5, atol=1e-6 * scale / sig.min())
    tm.close()


def test_predict_is_decoded_network_output():
    """lpp_surrogate_predict = encode -> network -> (pre_c (mu + sd y) + shot s - ref) / sigma."""
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    layers = S.surrogate_init(3)
    net = L.Surrogate(L.flatten_params(layers), batch=64)
    rng = np.random.default_rng(8)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    mu, sd, shot = rng.standard_normal(320) * 10, rng.uniform(0.5, 2.0, 320), rng.uniform(0, 5, 320)
    ref, sig = rng.standard_normal(320), rng.uniform(1.0, 3.0, 320)
    lo, hi = S.SURROGATE_RANGES[:, 0], S.SURROGATE_RANGES[:, 1]
    feed = (1, 0, 1, 1, 0, 1)
    maps = [dev(mu), dev(sd), dev(shot), dev(ref), dev(sig)]
    net.set_map(lo, hi, feed, *maps)
    theta = S.latin_hypercube(150, seed=4)      # three chunks, the last one ragged
    th = dev(theta)
    x = net.encode(th).cpu().numpy()
    want_x = np.where(np.array(feed) > 0, 2 * (theta - lo) / (hi - lo) - 1, 0.0)
    np.testing.assert_allclose(x, want_x, atol=1e-6)
    y = net.infer(torch.from_numpy(x).cuda()).double().cpu().numpy()
    got = net.predict(th).double().cpu().numpy()
    A, b, s8, sh = theta[:, 0:1], theta[:, 1:2], theta[:, 2:3], theta[:, 5:6]
    pre = np.concatenate([np.repeat(A * b * s8 ** 2, 80, 1), np.repeat(A * A * s8 ** 2, 240, 1)], axis=1)
    want = (pre * (mu + sd * y) + sh * shot - ref) / sig
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-4)
    net.close()


def test_targets_decode_back_to_the_template():
    """Decoding the training targets (instead of the network's outputs) reproduces the FFTLog
    path: lpp_surrogate_targets and the decoding share the baseline and the exact factors."""
    import torch
    from paper_2202_11839_gb300 import surrogate as SG
    tm = _template()
    em = SG.Emulator(tm, SG.survey_volume(), SURVEY_NOISE_G, SG.TrainConfig(base_nodes=4))
    em.net = em._make_net()
    theta = S.latin_hypercube(40, seed=31)
    th, y = em.training_set(40, seed=31)
    y = y.double().cpu().numpy()
    # host decode with the Lobatto baseline
    xs = -np.cos(np.pi * np.arange(4) / 3)
    lo, hi = S.SURROGATE_RANGES[:, 0], S.SURROGATE_RANGES[:, 1]
    x = 2 * (theta - lo) / (hi - lo) - 1

    def lag(v):
        return np.array([np.prod([(v - xs[j]) / (xs[i] - xs[j]) for j in range(4) if j != i]) for i in range(4)])

    base = em.base.cpu().numpy()
    sd, shot, sig = em.sd.cpu().numpy(), em.shot.cpu().numpy(), em.sigma_dev.cpu().numpy()
    A, b, s8, sh = theta[:, 0:1], theta[:, 1:2], theta[:, 2:3], theta[:, 5:6]
    pre = np.concatenate([np.repeat(A * b * s8 ** 2, 80, 1), np.repeat(A * A * s8 ** 2, 240, 1)], axis=1)
    bl = np.stack([np.einsum("a,b,abj->j", lag(x[r, 3]), lag(x[r, 4]), base.reshape(4, 4, 320))
                   for r in range(len(theta))])
    got = (pre * (bl + sd * y) + sh * shot) / sig
    want = em.plain(th).double().cpu().numpy()
    assert np.abs(got - want).max() < 1e-3, np.abs(got - want).max()
    tm.close()


def test_emulator_accuracy_and_speed():
    """Train on 20k Latin-hypercube templates from the FFTLog path; evaluate on 2k held-out
    parameter sets in units of the Gaussian error bar: every output within 1% of its error
    bar (the emulator's accuracy target).  The trained network beats its interpolated
    baseline by a wide margin and is much faster than the FFTLog path."""
    import torch
    from paper_2202_11839_gb300 import surrogate as SG
    tm = _template()
    em = SG.Emulator(tm, SG.survey_volume(), SURVEY_NOISE_G)
    em.train()
    rep = em.evaluate(2000, seed=77)
    print("emulator", rep)
    assert rep.max_sigma <= 0.01 and rep.p99_sigma < 0.002, rep
    assert rep.rms_sigma * 10 < rep.baseline_rms_sigma, rep
    # speed: one batch of 8192 parameter sets through each path
    net = em.inference_net(8192)
    th = torch.from_numpy(S.latin_hypercube(8192, seed=78)).cuda()
    times = {}
    for name, fn in (("plain", em.plain), ("surrogate", net.predict)):
        fn(th)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(tm.stream)
        fn(th)
        e1.record(tm.stream)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1)
    print("templates/s", {k: 8192 / (v * 1e-3) for k, v in times.items()})
    assert times["surrogate"] * 10 < times["plain"], times
    # the large-batch copy gives the same curves
    np.testing.assert_allclose(net.predict(th[:300]).cpu().numpy(), em.predict(th[:300]).cpu().numpy(),
                               rtol=0, atol=1e-5)
    # outside the box the FFTLog path answers
    out_box = np.array([[3.5, 2.0, 0.8, 0.0, 0.2, 1.0]])
    got = em.templates(out_box).double().cpu().numpy()
    want = em.plain(torch.from_numpy(out_box).cuda()).double().cpu().numpy()
    np.testing.assert_array_equal(got, want)
    tm.close()


def test_state_checkpoint_round_trip():
    """lpp_surrogate_save_state / load_state: a network loaded from a checkpoint continues the
    training as the saved one does (same Adam step count and moments), and a buffer with
    another magic number, a short buffer or a flipped payload bit is refused."""
    import torch
    L, net, layers, x, y, t = _setup(batch=64, seed=3)
    rng = np.random.default_rng(12)
    sched = lambda: t(rng.integers(0, 64, 64 * 20).astype(np.int32))
    net.train(t(x), t(y), sched(), 1e-3)
    state = net.save_state()
    other = L.Surrogate(L.flatten_params(S.surrogate_init(9)), batch=64)
    other.load_state(state)
    np.testing.assert_array_equal(other.params(), net.params())
    s2 = sched()
    net.train(t(x), t(y), s2, 1e-3)
    other.train(t(x), t(y), s2, 1e-3)
    a, b = net.params(), other.params()
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(a))
    # a fresh network (step 0, zero moments) trained on the same schedule ends elsewhere
    fresh = L.Surrogate(L.flatten_params(S.surrogate_init(9)), batch=64)
    fresh.load_state(state)
    bad = state.copy()
    bad[0] ^= 0xFF
    with pytest.raises(L.LppError):
        fresh.load_state(bad)
    with pytest.raises(L.LppError):
        fresh.load_state(state[:-4])
    flipped = state.copy()
    flipped[len(state) // 2] ^= 0x01   # one payload bit: the checksum refuses it
    with pytest.raises(L.LppError):
        fresh.load_state(flipped)
    for m in (net, other, fresh):
        m.close()


def test_emulator_training_resumes_from_a_checkpoint(tmp_path):
    """Emulator.train(checkpoint=...) after one phase, then train(resume=...) in a new
    emulator, ends where an uninterrupted training ends (the schedules continue from the saved
    generator state; the network from the saved Adam state)."""
    from paper_2202_11839_gb300 import surrogate as SG
    tm = _template()
    cfg = SG.TrainConfig(n_train=2048, n_test=64, batch=256, epochs=(3, 3), lrs=(1e-3, 3e-4), base_nodes=4)
    whole = SG.Emulator(tm, SG.survey_volume(), SURVEY_NOISE_G, cfg)
    whole.train()
    path = str(tmp_path / "emu.npz")
    first = SG.Emulator(tm, SG.survey_volume(), SURVEY_NOISE_G, cfg)
    first.train(checkpoint=path, phases=1)
    second = SG.Emulator(tm, SG.survey_volume(), SURVEY_NOISE_G, cfg)
    second.train(resume=path)
    a, b = whole.net.params(), second.net.params()
    assert second.losses.size == whole.losses.size
    assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(a))
    other = SG.Emulator(tm, SG.survey_volume(), SURVEY_NOISE_G, SG.TrainConfig(n_train=4096, epochs=(3, 3),
                                                                               lrs=(1e-3, 3e-4), base_nodes=4))
    with pytest.raises(ValueError):
        other.train(resume=path)
    for e in (whole, first, second, other):
        if e.net is not None:
            e.net.close()
    tm.close()


def test_predict_baseline_matches_fp64_decoding():
    """With an 8 x 8 Lobatto baseline: lpp_surrogate_predict (the baseline summed in
    float-float arithmetic on the FP32 pipes) against the same decoding in FP64 on the host.
    The base is 1e5 plus O(1) values and mu = -1e5 (the Lagrange weights sum to 1), so the
    baseline cancels to O(1): a plain FP32 sum would be off by about 1e-2 there, the float-float
    sum agrees to the FP32 rounding of the stored prediction.  A second set_map with another
    base is picked up."""
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    net = L.Surrogate(L.flatten_params(S.surrogate_init(5)), batch=64)
    rng = np.random.default_rng(21)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    nodes = 8
    mu, sd, shot = -1e5 + rng.standard_normal(320), rng.uniform(0.5, 2.0, 320), rng.uniform(0, 5, 320)
    sig = rng.uniform(1.0, 3.0, 320)
    lo, hi = S.SURROGATE_RANGES[:, 0], S.SURROGATE_RANGES[:, 1]
    feed = (0, 0, 0, 1, 1, 0)
    theta = S.latin_hypercube(150, seed=6)
    th = dev(theta)
    xs = -np.cos(np.pi * np.arange(nodes) / (nodes - 1))

    def lag(v):
        return np.array([np.prod([(v - xs[j]) / (xs[i] - xs[j]) for j in range(nodes) if j != i])
                         for i in range(nodes)])

    x = 2 * (theta - lo) / (hi - lo) - 1
    A, b, s8, sh = theta[:, 0:1], theta[:, 1:2], theta[:, 2:3], theta[:, 5:6]
    pre = np.concatenate([np.repeat(A * b * s8 ** 2, 80, 1), np.repeat(A * A * s8 ** 2, 240, 1)], axis=1)
    for seed in (1, 2):
        base = 1e5 + np.random.default_rng(seed).standard_normal((nodes * nodes, 320))
        keep = [dev(mu), dev(sd), dev(shot), dev(sig), dev(base.reshape(-1))]
        net.set_map(lo, hi, feed, keep[0], keep[1], keep[2], None, keep[3], base=keep[4], base_nodes=nodes,
                    base_in=(3, 4))
        xin = net.encode(th)
        y = net.infer(xin).double().cpu().numpy()
        got = net.predict(th).double().cpu().numpy()
        bl = np.stack([np.einsum("a,b,abj->j", lag(x[r, 3]), lag(x[r, 4]), base.reshape(nodes, nodes, 320))
                       for r in range(len(theta))])
        want = (pre * (mu + bl + sd * y) + sh * shot) / sig
        # the prediction is stored in FP32: compare to its rounding
        assert np.max(np.abs(got - want) / (np.abs(want) + 1.0)) < 1e-5, (seed, np.max(np.abs(got - want)))
    net.close()
