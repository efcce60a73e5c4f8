"""Batches of graphs: dos_build_csr_batched + dos_moments_batched against the
oracle run on each graph alone (the batch operator is block diagonal, so each
graph's moments are its own), and the plan autotuner."""
import numpy as np
import pytest
import torch

import oracle
import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")

TOL_D = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()
    yield
    nd.dos_set_plan(0, 0)


def _batch(count=24, seed=5):
    rng = np.random.default_rng(seed)
    graphs = []
    for g in range(count):
        n = int(rng.integers(200, 2500))
        kind = g % 4
        if kind == 0:
            graphs.append(sg.erdos_renyi(n, float(rng.uniform(4, 20)) / n, 100 + g))
        elif kind == 1:
            graphs.append(sg.barabasi_albert(n, int(rng.integers(2, 16)), 200 + g))
        elif kind == 2:
            graphs.append(sg.chung_lu(n, float(rng.uniform(2.1, 3.0)), float(rng.uniform(4, 20)), 300 + g))
        else:
            # a hub above the heavy-row threshold, plus isolated nodes
            s, d, nn = sg.erdos_renyi(n, 6.0 / n, 400 + g)
            hub = np.zeros(2100, np.int64)
            leaves = np.arange(1, 2101, dtype=np.int64) % nn
            graphs.append((np.concatenate([s, hub]), np.concatenate([d, leaves]), max(nn, 2101)))
    return graphs


def _reference(graphs, offs, m, nz, seed):
    out = []
    for (s, d, n), o in zip(graphs, offs[:-1]):
        ref = oracle.build_csr(s, d, n)
        z = oracle.probes(seed, ref.old_id.astype(np.int64) + int(o), nz)  # global ids key the probes
        out.append(oracle.kpm_doubled(ref, z, m) / (ref.n * nz))
    return np.array(out)


def test_batched_moments_match_each_graph():
    graphs = _batch()
    src, dst, offs = sg.union(graphs)
    g = nd.dos_build_csr_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), offs)
    info = nd.dos_batch_info(g)
    assert info["n_graphs"] == len(graphs)
    for k, (s, d, n) in enumerate(graphs):
        ref = oracle.build_csr(s, d, n)
        assert info["graph_n"][k] == ref.n and info["graph_isolated"][k] == ref.n_isolated
    m, nz, seed = 40, 16, 7
    d_gpu = nd.dos_moments_batched(g, m, nz, seed).cpu().numpy()
    d_ref = _reference(graphs, offs, m, nz, seed)
    assert d_gpu.shape == d_ref.shape
    assert np.abs(d_gpu - d_ref).max() <= TOL_D
    # replay of the captured sequence, then a new seed (re-captured)
    d_again = nd.dos_moments_batched(g, m, nz, seed).cpu().numpy()
    assert np.abs(d_again - d_gpu).max() <= 1e-12
    d_new = nd.dos_moments_batched(g, m, nz, seed + 1).cpu().numpy()
    assert np.abs(d_new - _reference(graphs, offs, m, nz, seed + 1)).max() <= TOL_D


def test_batched_bf16_and_odd_moment_count():
    graphs = _batch(count=10, seed=9)
    src, dst, offs = sg.union(graphs)
    g = nd.dos_build_csr_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), offs)
    d_gpu = nd.dos_moments_batched(g, 31, 20, 3, prec="bf16").cpu().numpy()
    d_ref = _reference(graphs, offs, 31, 20, 3)
    assert np.abs(d_gpu - d_ref).max() <= 2.0 * 2.0 ** -8


def test_batch_with_an_edgeless_graph_and_union_as_single_graph():
    graphs = [sg.erdos_renyi(300, 0.03, 1), (np.zeros(0, np.int64), np.zeros(0, np.int64), 50), sg.cycle(40)]
    src, dst, offs = sg.union(graphs)
    g = nd.dos_build_csr_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), offs)
    d = nd.dos_moments_batched(g, 10, 8, 1).cpu().numpy()
    assert np.all(np.isnan(d[1])) and np.all(np.isfinite(d[[0, 2]]))
    ref_c = oracle.build_csr(*sg.cycle(40))
    z = oracle.probes(1, ref_c.old_id.astype(np.int64) + int(offs[2]), 8)
    assert np.abs(d[2] - oracle.kpm_doubled(ref_c, z, 10) / (40 * 8)).max() <= TOL_D
    # the same handle as one graph: the moments of the union
    ref_u = oracle.build_csr(src, dst, int(offs[-1]))
    z = oracle.probes(4, ref_u.old_id, 8)
    du = nd.dos_moments(g, 10, 8, 4).cpu().numpy()
    assert np.abs(du - oracle.kpm_doubled(ref_u, z, 10) / (ref_u.n * 8)).max() <= TOL_D


def test_edges_between_graphs_are_rejected():
    src = np.array([0, 1, 2], np.int64)
    dst = np.array([1, 2, 5], np.int64)  # 2-5 joins graph 0 (ids 0..3) and graph 1 (ids 4..7)
    with pytest.raises(nd.DosError) as e:
        nd.dos_build_csr_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), [0, 4, 8])
    assert e.value.status == nd.DOS_EINVAL
    with pytest.raises(nd.DosError):
        nd.dos_build_csr_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), [1, 8])


def test_autotune_picks_a_plan_and_keeps_results():
    s, d, n = sg.chung_lu(20000, 2.5, 10.0, 3)
    ref = oracle.build_csr(s, d, n)
    g = nd.dos_build_csr(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    plan = nd.dos_autotune(g, 24)
    assert plan["tile_width"] in (4, 8, 16, 32, 64) and 1 <= plan["ctas_per_sm"] <= 3
    assert nd.dos_get_plan(g, 24)["tile_width"] == plan["tile_width"]
    dm = nd.dos_moments(g, 30, 24, 2).cpu().numpy()
    z = oracle.probes(2, ref.old_id, 24)
    assert np.abs(dm - oracle.kpm_doubled(ref, z, 30) / (ref.n * 24)).max() <= TOL_D
