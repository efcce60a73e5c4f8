"""Failure detection without a GPU fault: every device allocation the library
makes during a call is made to fail in turn (dos_test_fail_alloc, a host-side
hook that answers like an out-of-memory cudaMalloc).  Each time the call must
report DOS_ENOMEM with the injected message, and the library must stay usable:
the same call made right after gives the result of an undisturbed run.  No
kernel is launched on a failed allocation, so nothing here can fault the GPU."""
import numpy as np
import pytest
import torch

import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()
    yield
    nd.dos_test_fail_alloc(-1)


def _edges():
    s, d, n = sg.chung_lu(6000, 2.5, 12.0, 7)
    s, d, n = sg.add_twin_leaves(s, d, n, 300, 8)
    hub = np.zeros(2500, np.int64)  # a heavy row (degree >= 2048)
    return np.concatenate([s, hub]), np.concatenate([d, 1 + np.arange(2500, dtype=np.int64)]), n


SRC, DST, N = _edges()


def _graph(host=False, order="degree"):
    s, d = torch.from_numpy(SRC), torch.from_numpy(DST)
    if not host:
        s, d = s.cuda(), d.cuda()
    return nd.dos_build_csr(s, d, N, order=order)


def _export(g):
    return {k: v.cpu().numpy() for k, v in nd.dos_graph_export(g).items()}


def _ops():
    g = _graph()
    f = nd.dos_motif_filter(g)

    def build_device():
        return _export(_graph())

    def build_host():
        return _export(_graph(host=True))

    def motif_filter():
        return nd.dos_filter_export(nd.dos_motif_filter(g)).cpu().numpy()

    def moments():
        return nd.dos_moments(g, 40, 20, 3).cpu().numpy()

    def moments_filtered_bf16():
        return nd.dos_moments(g, 40, 20, 3, prec="bf16", filter=f).cpu().numpy()

    def ldos_node_major():
        c, d = nd.ldos_moments(g, 12, 70, 5, layout="node")  # several probe tiles: the fold scratch
        return np.concatenate([c.cpu().numpy().ravel(), d.cpu().numpy()])

    def whole_graph_density():
        d = nd.dos_moments(g, 30, 16, 9, filter=f)
        return nd.dos_density(d, 50, g=g, filter=f).cpu().numpy()

    def lanczos():
        a, b = nd.dos_lanczos(g, 8, 16, 1)[:2]
        return np.concatenate([a.cpu().numpy().ravel(), b.cpu().numpy().ravel()])

    def batch():
        parts = [sg.erdos_renyi(300 + 50 * k, 0.02, 40 + k) for k in range(5)]
        off = np.cumsum([0] + [p[2] for p in parts])
        s = np.concatenate([p[0] + o for p, o in zip(parts, off[:-1])])
        d = np.concatenate([p[1] + o for p, o in zip(parts, off[:-1])])
        gb = nd.dos_build_csr_batched(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), list(off))
        return nd.dos_moments_batched(gb, 20, 16, 2).cpu().numpy()

    def mlp():
        net = nd.dos_mlp_create([14, 16, 8], seed=1)
        x = torch.linspace(-1, 1, 4 * 14, device="cuda").view(4, 14)
        t = torch.full((4, 8), 1.0 / 8, device="cuda")
        nd.dos_mlp_train_step(net, x, t, 1e-2)
        return nd.dos_mlp_forward(net, x).cpu().numpy()

    return {k: v for k, v in locals().items() if callable(v) and not k.startswith("_") and k not in ("g", "f")}


def _same(a, b, exact):
    if isinstance(a, dict):
        return a.keys() == b.keys() and all(_same(a[k], b[k], exact) for k in a)
    return np.array_equal(a, b) if exact else np.allclose(a, b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name", ["build_device", "build_host", "motif_filter", "moments", "moments_filtered_bf16",
                                  "ldos_node_major", "whole_graph_density", "lanczos", "batch", "mlp"])
def test_every_allocation_failure_is_reported_and_recovered(name):
    op = _ops()[name]
    ref = op()
    exact = name not in ("batch", "lanczos")  # FP64 atomics / reductions: compare to rounding
    failures = 0
    for k in range(200):
        nd.dos_test_fail_alloc(k)
        try:
            op()
            fired = False
        except nd.DosError as e:
            assert e.status == nd.DOS_ENOMEM, (k, e)
            assert "injected allocation failure" in str(e), (k, e)
            fired = True
        finally:
            nd.dos_test_fail_alloc(-1)
        if not fired:
            break
        failures += 1
        assert _same(op(), ref, exact), (name, k)  # the library is usable again, its answer unchanged
    else:
        pytest.fail("more than 200 allocations in one call")
    assert failures >= 1, "the call made no device allocation"


def test_allocation_free_entry_needs_no_allocation():
    """With the hook armed to fail the very next allocation,
    dos_moments_noalloc still runs: it takes no device memory of its own."""
    g = _graph()
    ref = nd.dos_moments(g, 20, 8, 4).cpu().numpy()
    out = torch.empty(20, dtype=torch.float64, device="cuda")
    nd.dos_test_fail_alloc(0)
    try:
        nd.dos_moments_noalloc(g, 20, 8, 4, out)
        torch.cuda.synchronize()
        # the hook is still armed: the next library allocation is the one that fails
        with pytest.raises(nd.DosError) as e:
            nd.dos_moments(g, 20, 8, 4)
        assert e.value.status == nd.DOS_ENOMEM
    finally:
        nd.dos_test_fail_alloc(-1)
    assert np.array_equal(out.cpu().numpy(), ref)
