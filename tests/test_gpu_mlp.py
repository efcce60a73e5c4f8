"""Density-reconstruction MLP on the GPU against the FP64 oracle (oracle/mlp.py):
forward probabilities, loss and gradient, Adam steps (with and without a row
gather), the feature / target kernels and the batched density, and a training
run in which the learned reconstruction beats plain Jackson KPM on held-out
graphs at the same cheap moment budget."""
import numpy as np
import pytest
import torch

import oracle
import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")

U = 2.0**-24  # unit roundoff of float32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()
    yield


def _flatten(params):
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in params]).astype(np.float32)


def _unflatten(flat, sizes):
    out, o = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        w = np.asarray(flat[o:o + fi * fo], np.float64).reshape(fo, fi)
        o += fi * fo
        b = np.asarray(flat[o:o + fo], np.float64)
        o += fo
        out.append((w, b))
    return out


def _net(sizes, seed):
    """A GPU network and the oracle's copy of its (float32-exact) parameters."""
    rng = np.random.default_rng(seed)
    params = oracle.mlp_init(sizes, rng)
    params = [(w, rng.normal(0, 0.1, b.shape)) for w, b in params]
    flat = _flatten(params)
    net = nd.dos_mlp_create(sizes, seed=seed)
    assert nd.dos_mlp_param_count(net) == flat.size
    nd.dos_mlp_set_params(net, torch.from_numpy(flat).cuda())
    return net, _unflatten(flat, sizes)


def _data(rows, sizes, seed):
    rng = np.random.default_rng(seed + 1000)
    x = rng.normal(size=(rows, sizes[0])).astype(np.float32)
    t = rng.random((rows, sizes[-1])) ** 3
    t = (t / t.sum(axis=1, keepdims=True)).astype(np.float32)
    return x, t


def _clear_rows(states, x, margin=1e-4):
    """Rows of x whose hidden pre-activations stay at least `margin` away from
    0 under every parameter set in `states`: there the float32 and float64
    forward passes (errors far below the margin) take the same ReLU decisions,
    so an element-by-element comparison is meaningful."""
    keep = np.ones(x.shape[0], bool)
    for params in states:
        _, zs, _ = oracle.mlp_forward(params, np.asarray(x, np.float64))
        for z in zs[:-1]:
            keep &= np.abs(z).min(axis=1) > margin
    return np.nonzero(keep)[0]


# sizes spanning several 64-wide tiles with ragged tails, one single-layer net
SHAPES = [([37, 70, 65, 50], 130), ([200, 256, 129, 64], 257), ([5, 3], 1), ([99, 256, 256, 50], 64)]


def _logit_error_bound(params, x):
    """First-order bound on |z_gpu - z| for the logits.  Each float32 output is
    a dot of K products accumulated with fused multiply-adds plus a bias, so
    its rounding error is at most gamma_{K+1} (|W| |a| + |b|), gamma_n = n u /
    (1 - n u); an input error e propagates as |W| e (ReLU is 1-Lipschitz)."""
    a = np.asarray(x, np.float64)
    e = np.zeros_like(a)
    for l, (w, b) in enumerate(params):
        k = w.shape[1] + 1
        gam = k * U / (1 - k * U)
        e = e @ np.abs(w).T + gam * (np.abs(a) @ np.abs(w).T + np.abs(b))
        z = a @ w.T + b
        a = np.maximum(z, 0.0) if l + 1 < len(params) else z
    return e, a


@pytest.mark.parametrize("sizes,rows", SHAPES)
def test_forward_matches_oracle(sizes, rows):
    net, params = _net(sizes, 1)
    x, _ = _data(rows, sizes, 1)
    p = nd.dos_mlp_forward(net, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    p_ref, _, _ = oracle.mlp_forward(params, x.astype(np.float64))
    # softmax: |dp_i| <= p_i (|dz_i| + max_j |dz_j|) plus the rounding of the
    # max-shift, the log-sum and expf/logf (a few ulp each)
    e, z = _logit_error_bound(params, x)
    shift = np.abs(z - z.max(axis=1, keepdims=True))
    logs = np.log(np.exp(z - z.max(axis=1, keepdims=True)).sum(axis=1, keepdims=True))
    rel = e + e.max(axis=1, keepdims=True) + 2 * U * (shift + np.abs(logs)) + (sizes[-1] + 8) * U
    bound = 2.0 * p_ref * rel + 1e-30
    assert np.all(np.abs(p - p_ref) <= bound), float(np.max(np.abs(p - p_ref) / bound))
    assert np.allclose(p.sum(axis=1), 1.0, atol=(sizes[-1] + 8) * U)


@pytest.mark.parametrize("sizes,rows", SHAPES)
def test_loss_and_gradient_match_oracle(sizes, rows):
    net, params = _net(sizes, 2)
    x, t = _data(rows, sizes, 2)
    keep = _clear_rows([params], x)
    assert keep.size >= 0.9 * rows
    x, t = np.ascontiguousarray(x[keep]), np.ascontiguousarray(t[keep])
    loss, grad = nd.dos_mlp_loss_grad(net, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    loss_ref, g_ref = oracle.mlp_loss_grad(params, x.astype(np.float64), t.astype(np.float64))
    # fp32 sums of at most K + rows ~ 520 terms: relative error below 520 u ~ 3e-5
    # of the absolute-value sum; 2e-4 of the block's largest entry leaves room
    # for a cancellation factor of ~6
    assert abs(float(loss.item()) - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref))
    g = _unflatten(grad.cpu().numpy(), sizes)
    for (gw, gb), (rw, rb) in zip(g, g_ref):
        for a, r in ((gw, rw), (gb, rb)):
            assert np.abs(a - r).max() <= 2e-4 * max(np.abs(r).max(), 1e-12), np.abs(a - r).max() / np.abs(r).max()


@pytest.mark.parametrize("use_idx", [False, True])
def test_adam_steps_match_oracle(use_idx):
    sizes, rows = [37, 70, 65, 50], 130
    net, params = _net(sizes, 3)
    x, t = _data(rows, sizes, 3)
    lr = 1e-2
    rows_sel = np.random.default_rng(9).permutation(rows)[:77] if use_idx else np.arange(rows)

    def trajectory(sel):
        m = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
        v = [(np.zeros_like(w), np.zeros_like(b)) for w, b in params]
        out, ref = [], params
        for step in (1, 2, 3):
            loss_ref, g = oracle.mlp_loss_grad(ref, x[sel].astype(np.float64), t[sel].astype(np.float64))
            out.append((ref, loss_ref, g))
            ref, m, v = oracle.adam_step(ref, g, m, v, step, lr)
            out[-1] += (ref,)
        return out

    # drop rows with a ReLU decision near 0 at any of the states visited
    for _ in range(4):
        traj = trajectory(rows_sel)
        keep = _clear_rows([st[0] for st in traj] + [traj[-1][3]], x[rows_sel])
        if keep.size == rows_sel.size:
            break
        rows_sel = rows_sel[keep]
    assert keep.size == rows_sel.size and rows_sel.size >= 0.8 * (77 if use_idx else rows)
    if use_idx:
        idx_d = torch.from_numpy(rows_sel.astype(np.int32)).cuda()
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    else:
        idx_d = None
        xd = torch.from_numpy(np.ascontiguousarray(x[rows_sel])).cuda()
        td = torch.from_numpy(np.ascontiguousarray(t[rows_sel])).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    for step, (_, loss_ref, g, ref) in zip((1, 2, 3), traj):
        nd.dos_mlp_train_step(net, xd, td, lr, idx=idx_d, loss=loss)
        assert abs(float(loss.item()) - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
        got = _unflatten(nd.dos_mlp_get_params(net).cpu().numpy(), sizes)
        gmax = max(max(np.abs(gw).max(), np.abs(gb).max()) for gw, gb in g)
        for (aw, ab), (rw, rb), (gw, gb) in zip(got, ref, g):
            for a, r, gg in ((aw, rw, gw), (ab, rb, gb)):
                # an Adam update is lr * m_hat / (sqrt(v_hat) + eps), a ratio
                # of gradient sums: where the gradient is well above its own
                # rounding error the update direction agrees to ~1e-3 of lr
                # per step; near-zero gradients may move by up to lr
                well = np.abs(gg) > 1e-3 * gmax
                assert np.abs(a - r)[well].max(initial=0.0) <= step * (2e-3 * lr) + 4 * U * np.abs(r).max()
                assert np.abs(a - r).max() <= step * 2 * lr


def test_features_targets_and_batched_density():
    graphs = [sg.erdos_renyi(300, 0.03, 1), sg.barabasi_albert(400, 3, 2), sg.chung_lu(500, 2.5, 6.0, 3),
              sg.cycle(64)]
    src, dst, offs = sg.union(graphs)
    g = nd.dos_build_csr_batched(torch.from_numpy(src), torch.from_numpy(dst), offs)
    d = nd.dos_moments_batched(g, 40, 16, 7)
    for b in (1, 50, 333):
        h = nd.dos_density_batched(d, b).cpu().numpy()
        dh = d.cpu().numpy()
        for k in range(len(graphs)):
            assert np.abs(h[k] - oracle.histogram(dh[k], b)).max() <= 1e-12
        hn = nd.dos_density_batched(d, b, kernel="none").cpu().numpy()
        assert np.abs(hn[0] - oracle.histogram(dh[0], b, kernel="none")).max() <= 1e-12
        for kk in (1, 7, 40):
            x = nd.dos_mlp_features(torch.from_numpy(h).cuda(), d, kk).cpu().numpy()
            assert np.array_equal(x, oracle.mlp_features(h, dh, kk).astype(np.float32))
        tt = nd.dos_hist_normalize(torch.from_numpy(h - 0.3 / b).cuda()).cpu().numpy()
        t_ref = oracle.normalize_hist(h - 0.3 / b)
        assert np.abs(tt - t_ref).max() <= 4 * U * max(t_ref.max(), 1.0)


def test_errors_are_reported():
    with pytest.raises(nd.DosError):
        nd.dos_mlp_create([4], seed=0)
    with pytest.raises(nd.DosError):
        nd.dos_mlp_create([4, 0, 3], seed=0)
    net = nd.dos_mlp_create([4, 8, 3], seed=0)
    x = torch.zeros((2, 4), dtype=torch.float32, device="cuda")
    t = torch.full((2, 3), 1 / 3, dtype=torch.float32, device="cuda")
    with pytest.raises(nd.DosError):
        nd.dos_mlp_train_step(net, x, t, lr=0.0)
    # He-uniform init from SplitMix64: weights inside +-sqrt(6 / fan_in), biases 0
    p = nd.dos_mlp_get_params(net).cpu().numpy()
    w1, b1 = p[:32], p[32:40]
    assert np.abs(w1).max() <= np.sqrt(6 / 4) and np.abs(w1).max() > 0.5 and not b1.any()
    assert np.array_equal(p, nd.dos_mlp_get_params(nd.dos_mlp_create([4, 8, 3], seed=0)).cpu().numpy())


# ---------------------------------------------------------------------------
# the learned reconstruction beats Jackson KPM at the same cheap budget
# ---------------------------------------------------------------------------
B_BINS, M_CHEAP, NZ_CHEAP, M_TARGET, NZ_TARGET = 50, 50, 4, 500, 256


def _cheap_and_target(graphs, seed):
    src, dst, offs = sg.union([(s, d, n) for s, d, n, _ in graphs])
    g = nd.dos_build_csr_batched(torch.from_numpy(src), torch.from_numpy(dst), offs)
    d_cheap = nd.dos_moments_batched(g, M_CHEAP, NZ_CHEAP, seed)
    h_cheap = nd.dos_density_batched(d_cheap, B_BINS)
    x = nd.dos_mlp_features(h_cheap, d_cheap, M_CHEAP)
    d_t = nd.dos_moments_batched(g, M_TARGET, NZ_TARGET, seed + 1)
    t = nd.dos_hist_normalize(nd.dos_density_batched(d_t, B_BINS))
    return x, t, h_cheap


def test_learned_reconstruction_beats_jackson_on_held_out_graphs():
    train = list(sg.batch_graphs(2048, 11, n_min=300, n_max=800))
    test = list(sg.batch_graphs(64, 12, n_min=300, n_max=800))
    x, t, _ = _cheap_and_target(train, 100)
    x_te, _, h_te = _cheap_and_target(test, 200)
    net = nd.dos_mlp_create([x.shape[1], 256, 256, B_BINS], seed=5)
    steps, batch = 3000, 256
    gen = torch.Generator().manual_seed(0)
    idx_all = torch.randint(0, x.shape[0], (steps, batch), generator=gen, dtype=torch.int32).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    first = None
    for s in range(steps):
        nd.dos_mlp_train_step(net, x, t, 1e-3, idx=idx_all[s], loss=loss)
        if s == 0:
            first = float(loss.item())
    assert float(loss.item()) < first
    p_te = nd.dos_mlp_forward(net, x_te).cpu().numpy()
    h_te = h_te.cpu().numpy()
    l1_mlp, l1_kpm = [], []
    for k, (s, d, n, _) in enumerate(test):
        ref = oracle.build_csr(s, d, n)
        lam = np.linalg.eigvalsh(oracle.dense_h(ref))
        exact = oracle.exact_histogram(lam, B_BINS)
        l1_mlp.append(oracle.l1(p_te[k], exact))
        l1_kpm.append(oracle.l1(h_te[k], exact))
    l1_mlp, l1_kpm = float(np.mean(l1_mlp)), float(np.mean(l1_kpm))
    print(f"held-out mean L1: learned {l1_mlp:.4f}, Jackson KPM {l1_kpm:.4f}")
    assert l1_mlp < 0.8 * l1_kpm


def test_hist_assemble_matches_oracle():
    rng = np.random.default_rng(4)
    for b in (2, 7, 200):
        p = rng.random((3, b)).astype(np.float32)
        p /= p.sum(axis=1, keepdims=True)
        spikes = [(0.0, 0.125), (-1.0, 0.01), (1.0 / np.sqrt(2), 0.02), (-0.5, 0.03)]
        h = nd.dos_hist_assemble(torch.from_numpy(p).cuda(), scale=0.7, spikes=spikes).cpu().numpy()
        pts = oracle.point_mass_histogram([s[0] for s in spikes], [s[1] for s in spikes], b)
        ref = 0.7 * p.astype(np.float64) + pts
        assert np.abs(h - ref).max() <= 1e-15


def test_learned_reconstruct_assembles_filtered_density():
    """learned.reconstruct = (r/N) * network output + zero spike, on a graph
    with twins and isolated nodes; features equal the oracle's definition."""
    from paper_1905_09758_gb300 import learned

    s, d, n = sg.add_twin_leaves(*sg.chung_lu(3000, 2.5, 8.0, 5), 100, 6)
    n += 7  # seven isolated nodes
    g, f = learned.filtered_operator(torch.from_numpy(s), torch.from_numpy(d), n)
    m_in, bins = 20, 40
    net = nd.dos_mlp_create([bins + m_in - 1, 16, bins], seed=1)
    rec = learned.Reconstructor(net, m_in, 4, bins, stats=False)
    h = learned.reconstruct(rec, g, f, seed=9).cpu().numpy()
    x = learned.features(g, f, m_in, 4, 9, bins, stats=False)
    dd = nd.dos_moments(g, m_in, 4, 9, filter=f).cpu().numpy()
    # the GPU histogram equals the oracle's to ~1e-12, so the float32 features
    # agree to one rounding
    x_ref = oracle.mlp_features(oracle.histogram(dd, bins)[None], dd[None], m_in)[0]
    assert np.all(np.abs(x.cpu().numpy()[0] - x_ref) <= 2 * U * np.maximum(np.abs(x_ref), 1e-3))
    p = nd.dos_mlp_forward(net, x).cpu().numpy()[0].astype(np.float64)
    ref = oracle.build_csr(s, d, n)
    _, removed = oracle.twin_classes(ref)
    n_tot = ref.n + ref.n_isolated
    want = (ref.n - removed) / n_tot * p + oracle.point_mass_histogram([0.0], [(removed + ref.n_isolated) / n_tot], bins)
    assert np.abs(h - want).max() <= 1e-12
    assert abs(h.sum() - 1.0) <= 1e-6


def test_degree_stats_and_stat_features_match_oracle():
    """dos_graph_stats equals the oracle's degree statistics exactly (integer
    sums), and the feature rows with them agree with the oracle's definition
    to float32 rounding."""
    from paper_1905_09758_gb300 import learned

    s, d, n = sg.add_twin_leaves(*sg.chung_lu(4000, 2.3, 9.0, 15), 80, 16)
    n += 5
    ref = oracle.build_csr(s, d, n)
    g, f = learned.filtered_operator(torch.from_numpy(s), torch.from_numpy(d), n)
    for nz in (1, 8, 64):
        st = nd.dos_graph_stats(g, nz).cpu().numpy()
        assert np.array_equal(st, oracle.graph_stats(ref.deg, nz)), (st, oracle.graph_stats(ref.deg, nz))
    m_in, bins = 12, 30
    x = learned.features(g, f, m_in, 8, 4, bins).cpu().numpy()[0]
    assert x.shape == (bins + m_in - 1 + 4,)
    dd = nd.dos_moments(g, m_in, 8, 4, filter=f).cpu().numpy()
    x_ref = oracle.mlp_features(oracle.histogram(dd, bins)[None], dd[None], m_in,
                                stats=[oracle.graph_stats(ref.deg, 8)])[0]
    assert np.all(np.abs(x - x_ref) <= 2 * U * np.maximum(np.abs(x_ref), 1e-3))


def test_training_sets_share_one_cheap_run():
    """learned.training_sets: the rows for each input size equal the features
    of a run with exactly that many moments (the doubled recurrence's first
    moments do not depend on how many follow), and the targets equal
    training_set's."""
    from paper_1905_09758_gb300 import learned

    graphs = [sg.add_twin_leaves(*sg.chung_lu(1500, 2.5, 8.0, 40 + k), 30, 50 + k) for k in range(3)]
    xs, t = learned.training_sets(graphs, [8, 13], nz_in=4, m_ref=40, nz_ref=16, bins=30, seed=9)
    for m in (8, 13):
        x1, t1 = learned.training_set(graphs, m, 4, 40, 16, 30, seed=9)
        assert torch.equal(xs[m], x1), m
        assert torch.equal(t, t1)


def test_checkpoint_and_resume_training(tmp_path):
    """learned.save / load with Adam's state (dos_mlp_get_state / set_state):
    a run interrupted after 30 of 50 steps, written to disk, read back into a
    new handle and resumed ends bit for bit where the uninterrupted run ends;
    a parameters-only file reproduces the forward pass."""
    from paper_1905_09758_gb300 import learned

    g = torch.Generator().manual_seed(5)
    bins, m_in = 12, 6
    x = torch.randn(64, bins + m_in - 1, generator=g).cuda()
    t = torch.rand(64, bins, generator=g)
    t = (t / t.sum(1, keepdim=True)).cuda()
    kw = dict(hidden=(32, 24), steps=50, batch=16, lr=1e-2, seed=3)
    full = learned.train(x, t, m_in, 4, **kw)
    part = learned.train(x, t, m_in, 4, stop=30, **kw)
    assert nd.dos_mlp_get_state(part.net)["step"] == 30
    learned.save(part, tmp_path / "ck.npz")
    back = learned.load(tmp_path / "ck.npz")
    assert (back.m_in, back.nz_in, back.bins, back.stats, back.sizes) == (m_in, 4, bins, False, part.sizes)
    done = learned.train(x, t, m_in, 4, resume=back, **kw)
    a, b = nd.dos_mlp_get_state(full.net), nd.dos_mlp_get_state(done.net)
    assert a["step"] == b["step"] == 50
    for k in ("params", "m", "v"):
        assert torch.equal(a[k], b[k]), k
    learned.save(full, tmp_path / "p.npz", with_optimizer=False)
    only = learned.load(tmp_path / "p.npz")
    assert nd.dos_mlp_get_state(only.net)["step"] == 0
    assert torch.equal(nd.dos_mlp_forward(only.net, x[:5]), nd.dos_mlp_forward(full.net, x[:5]))
    with pytest.raises(nd.DosError):
        nd.dos_mlp_set_state(only.net, {"params": a["params"], "m": a["m"], "v": a["v"], "step": -1})
