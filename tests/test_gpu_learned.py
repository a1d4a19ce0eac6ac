"""Learned cardinality correction on the GPU: the device traffic generator, the features and
linear-counting estimates of episodes run through a batch (routers-only and scan modes)
against the oracle, the MLP's forward pass and gradients against the FP64 oracle network,
one Adam step against its published update rule, and a trained network's median relative
error against plain linear counting."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1805_09246_b300.synth import episodes as ep
from tests.test_gpu_parity import close_enough, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def S():
    from paper_1805_09246_b300 import sse
    return sse


def learn():
    from paper_1805_09246_b300 import learn as mod
    return mod


def small_cfg(**kw):
    base = dict(hosts=6, k=16, query_slice=23, card_min=50, card_max=20000, active_max=24, noise_pairs=700)
    base.update(kw)
    return ep.EpisodeConfig(**base)


def test_device_generator_matches_host_twin():
    cfg = small_cfg(card_max=2e5, noise_pairs=5000)
    t = ep.sample_hosts(cfg, 4, np.random.default_rng(3))
    dev = ep.DeviceTable(t)
    for s in (0, 7, 16, 23):
        views = dev.fill(s, cfg.noise_pairs, 77)
        torch.cuda.synchronize()
        got = np.concatenate([v.cpu().numpy().view(np.uint32) for v in views])
        want, per_router = ep.fill_cpu(t, s, cfg.noise_pairs, 77)
        assert [len(v) for v in views] == per_router.tolist()
        assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", [0, 1])
def test_episode_features_and_estimates_match_oracle(seed):
    """Episodes through the batch (routers-only steps, then a scan step that leaves slice Q
    open) give the oracle's features, linear-counting estimates and flags at slice Q."""
    sse, L = S(), learn()
    cfg = small_cfg()
    routers = 3
    p = sse.Params(k=cfg.k, seed=seed)
    smp = L.episodes(p, cfg, routers * cfg.hosts, routers=routers, seed=seed)
    table, gseed = L.draw_group(cfg, routers, np.random.default_rng(seed))
    orcs = [oracle.Oracle(oracle_params(p), track_exact=True) for _ in range(routers)]
    for s in range(cfg.query_slice + 1):
        pairs, per_router = ep.fill_cpu(table, s, cfg.noise_pairs, gseed)
        start = 0
        for r, o in enumerate(orcs):
            if s:
                o.advance()
            o.scan(pairs[start:start + int(per_router[r])])
            start += int(per_router[r])
    H = cfg.hosts
    x = smp.x.cpu().numpy()
    lc = smp.lc.cpu().numpy()
    flags = smp.flags.cpu().numpy()
    for r, o in enumerate(orcs):
        hosts = table.ip[r * H:(r + 1) * H]
        sl = slice(r * H, (r + 1) * H)
        np.testing.assert_allclose(x[sl], o.features(hosts), rtol=1e-6, atol=1e-6)
        e = o.estimate(hosts)
        assert close_enough(lc[sl], e["est"])
        assert np.array_equal(flags[sl], e["flags"])
        assert np.array_equal(smp.exact[sl].astype(np.uint32), o.exact_counts(hosts))


def random_net(n_in, hidden, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1, 1, omlp.param_count(n_in, hidden)).astype(np.float32)
    w[: hidden * n_in] *= np.sqrt(3.0 / n_in)
    w[hidden * n_in:] *= np.sqrt(3.0 / hidden)
    return w


@pytest.mark.parametrize("n_in,hidden,n", [(18, 64, 256), (7, 5, 33), (18, 64, 1)])
def test_forward_and_gradients_match_fp64_oracle(n_in, hidden, n):
    sse = S()
    m = sse.MLP(n_in, hidden=hidden, max_batch=512, seed=1)
    w32 = random_net(n_in, hidden, 2)
    m.set_params(w32)
    f, bits, _ = m.params()
    assert np.array_equal(f, w32)
    wb = bits.astype(np.uint32) << 16
    assert np.array_equal(wb.view(np.float32).astype(np.float64), omlp.bf16(w32))  # RNE to BF16
    theta = omlp.bf16(w32)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 8, (n, n_in)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = m.forward(xd).cpu().numpy().astype(np.float64)
    y_ref = omlp.forward(theta, x, n_in, hidden)
    assert np.abs(y - y_ref).max() <= 1e-5 * (1 + np.abs(y_ref).max())
    # gradients over a gathered subset of rows (the training path) and over all rows
    rows = np.sort(rng.choice(n, size=max(1, n // 2), replace=False)).astype(np.int32)
    for sel in (rows, None):
        rd = torch.from_numpy(sel).cuda() if sel is not None else None
        loss = m.gradients(xd, td, rd)
        g = m.params()[2].astype(np.float64)
        xs, ts = (x[sel], t[sel]) if sel is not None else (x, t)
        loss_ref, g_ref = omlp.gradient(theta, xs, ts, n_in, hidden)
        assert abs(loss - loss_ref) <= 1e-5 * (1 + loss_ref)
        assert np.abs(g - g_ref).max() <= 1e-4 * (np.abs(g_ref).max() + 1e-6)


def test_adam_step_follows_update_rule():
    """One Adam step (Kingma and Ba 2015, bias-corrected moments) from zero moments."""
    sse = S()
    m = sse.MLP(18, hidden=64, max_batch=64, seed=4)
    w32 = random_net(18, 64, 5)
    m.set_params(w32)
    rng = np.random.default_rng(6)
    x = torch.from_numpy(rng.uniform(0, 8, (64, 18)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(0, 1, 64).astype(np.float32)).cuda()
    m.gradients(x, t)
    g = m.params()[2].astype(np.float64)
    lr = 1e-3
    m.adam(lr)
    f, bits, _ = m.params()
    mh = (0.1 * g) / (1 - 0.9)
    vh = (0.001 * g * g) / (1 - 0.999)
    want = w32.astype(np.float64) - lr * mh / (np.sqrt(vh) + 1e-8)
    assert np.abs(f - want).max() <= 1e-6
    assert np.array_equal(bits.astype(np.uint32) << 16, omlp.bf16(f).astype(np.float32).view(np.uint32))


def test_epoch_replay_equals_the_steps():
    """sse_mlp_train_epoch replays an epoch from one CUDA graph (each minibatch's gradient
    shares, then Adam summing them, with programmatic dependent launch between the kernels):
    parameters, gradients and loss equal, bit for bit, the same minibatches taken one step at a
    time through sse_mlp_gradients and sse_mlp_adam. Two epochs, the last minibatch of each
    partial."""
    sse = S()
    n, batch, lr = 3000, 512, 2e-3
    rng = np.random.default_rng(8)
    x = torch.from_numpy(rng.uniform(0, 8, (n, 18)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(0, 1, n).astype(np.float32)).cuda()
    w32 = random_net(18, 64, 9)
    a = sse.MLP(18, hidden=64, max_batch=batch, seed=4)
    b = sse.MLP(18, hidden=64, max_batch=batch, seed=4)
    a.set_params(w32)
    b.set_params(w32)
    for _ in range(2):
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        la = a.train_epoch(x, t, perm, batch, lr)
        for b0 in range(0, n, batch):
            lb = b.gradients(x, t, rows=perm[b0:b0 + batch])
            b.adam(lr)
        assert la == lb
        for pa, pb in zip(a.params(), b.params()):
            assert np.array_equal(pa, pb)


def test_training_lowers_loss_and_learned_beats_linear_counting():
    """A network trained on GPU episodes (the library's own kernels) has a lower median
    relative error on held-out episodes than plain linear counting, and a much lower one on
    the hosts where the gate hands the estimate to it (linear counting saturates there)."""
    L = learn()
    cfg = ep.EpisodeConfig()
    res = L.run(n_train=150_000, n_test=40_000, routers=64, epochs=20, cfg=cfg, seed=11)
    assert res["losses"][-1] < res["losses"][0]
    test = res["test"]
    lc = test.lc.cpu().numpy().astype(np.float64)
    est = test.learned.cpu().numpy().astype(np.float64)
    exact = test.exact
    assert np.isfinite(est).all() and (est > 0).all()
    gated = L.active_cells(test.x, cfg.k) >= res["gate"]
    used = est != lc
    assert used.any() and not (used & ~gated).any()  # the network only acts above the gate
    rel = lambda e, m: float(np.median(np.abs(e[m] - exact[m]) / exact[m]))
    assert res["err_learned"] < res["err_lc"], (res["err_learned"], res["err_lc"])
    assert rel(est, gated) < 0.6 * rel(lc, gated), (rel(est, gated), rel(lc, gated))
    print(f"median relative error: learned {res['err_learned']:.4f}, linear counting {res['err_lc']:.4f}; "
          f"above the gate ({gated.mean():.1%} of hosts): learned {rel(est, gated):.4f}, "
          f"linear counting {rel(lc, gated):.4f}")
