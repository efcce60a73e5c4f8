"""The bench's own accuracy references (scipy/numpy, no oracle on the bench
path) checked here against the oracle on small graphs (CPU only)."""
import os
import sys

import numpy as np

import oracle
import synthgraphs as sg

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


def test_adjacency_matches_the_oracle_csr():
    src, dst, n = sg.random_geometric(800, 0.05, 3)
    # duplicates, a self-loop and isolated nodes on top
    src = np.concatenate([src, src[:50], [7]])
    dst = np.concatenate([dst, dst[:50], [7]])
    a = bench._adjacency(src, dst, n + 5)
    ref = oracle.build_csr(src, dst, n + 5)
    assert a.shape == (ref.n, ref.n)
    assert np.array_equal(a.indptr, ref.row_ptr)
    assert np.array_equal(a.indices, ref.col)
    assert np.all(a.data == 1.0)


def test_unit_probe_diagonal_is_the_exact_ldos():
    src, dst, n = sg.erdos_renyi(300, 0.03, 5)
    a = bench._adjacency(src, dst, n)
    ref = oracle.build_csr(src, dst, n)
    lam, q = oracle.exact_eigs(ref)
    sample = np.array([0, 3, 77, ref.n - 1])
    got = bench._unit_probe_diagonal(a, sample, 25)
    assert np.abs(got - oracle.exact_ldos(lam, q, 25)[sample]).max() <= 1e-12


def test_cpu_sample_times_the_oracle_on_worker_processes():
    """The CPU baseline's sample: the oracle's CSR shared with spawned workers
    that split the probe columns; one timing per repetition."""
    spec = dict(bench.CPU_SAMPLE, N=20_000, Nz=3)
    cs = bench.CpuSample(spec)
    try:
        times = cs.run(2, 2)
        assert len(times) == 2 and all(t > 0 for t in times)
        assert cs.cores == min(3, len(os.sched_getaffinity(0)))
        assert cs.bytes_per_step() == bench.step_bytes(cs.n, cs.nnz, 3, False)
        assert "N=20,000" in cs.describe(2)
    finally:
        cs.close()


def test_bfs_order_is_a_breadth_first_numbering():
    """bench.bfs_order (the --row-order measurement's breadth-first numbering):
    a permutation in which ranks grow with the BFS level from the largest-degree
    node, every reached node is numbered after a neighbour on the previous
    level, and nodes of other components follow."""
    import scipy.sparse.csgraph as csg
    import torch

    s1, d1, n1 = sg.grid2d(9, 7)
    s2, d2, n2 = sg.erdos_renyi(40, 0.1, 2)
    src = np.concatenate([s1, s2 + n1])
    dst = np.concatenate([d1, d2 + n1])
    n = n1 + n2 + 3  # three isolated nodes
    rank = bench.bfs_order(torch.from_numpy(src), torch.from_numpy(dst), n).numpy()
    assert np.array_equal(np.sort(rank), np.arange(n))
    import scipy.sparse as sp

    a = sp.coo_matrix((np.ones(2 * src.size), (np.concatenate([src, dst]), np.concatenate([dst, src]))),
                      shape=(n, n)).tocsr()
    a.data[:] = 1.0
    deg = np.diff(a.indptr)
    root = int(np.argmax(deg))
    assert rank[root] == 0
    level = csg.shortest_path(a, unweighted=True, indices=root)
    reached = np.isfinite(level)
    lv = level[reached]
    order = np.argsort(rank[reached])
    assert np.all(np.diff(lv[order]) >= 0)  # levels never decrease along the numbering
    assert rank[reached].max() < rank[~reached].min()
    for v in np.nonzero(reached)[0]:
        if v == root:
            continue
        nb = a.indices[a.indptr[v]:a.indptr[v + 1]]
        assert np.any(level[nb] == level[v] - 1)
