"""Oracle pins: probe generator and CSR construction (CPU only)."""
import os

import numpy as np
import pytest

import oracle
import synthgraphs as sg
from conftest import GOLDEN


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "splitmix64_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, i, v = line.split()
            rows.append((int(s), int(i), int(v)))
    return rows


def test_splitmix64_known_answers():
    for seed, idx, val in _kat():
        assert int(oracle.splitmix64(seed, idx)) == val


def test_probes_follow_definition_bitwise():
    # z[i, j] is bit (j & 63) of the output at counter ((j >> 6) << 32) | old_id
    old = np.array([0, 5, 77, 2**31 - 1], np.int64)
    z = oracle.probes(99, old, 130)
    assert set(np.unique(z)) <= {-1.0, 1.0}
    for r, o in enumerate(old):
        for j in (0, 1, 63, 64, 127, 129):
            word = int(oracle.splitmix64(99, ((j >> 6) << 32) | int(o)))
            bit = (word >> (j & 63)) & 1
            assert z[r, j] == (1.0 - 2.0 * bit)


def test_probes_are_balanced_and_uncorrelated():
    z = oracle.probes(7, np.arange(20000), 64)
    assert abs(z.mean()) < 0.01
    c = (z.T @ z) / z.shape[0]
    off = c - np.diag(np.diag(c))
    assert np.abs(off).max() < 0.05
    assert np.allclose(np.diag(c), 1.0)


def _brute_csr(src, dst, n):
    adj = [set() for _ in range(n)]
    for u, v in zip(src, dst):
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    keep = [i for i in range(n) if adj[i]]
    new = {o: k for k, o in enumerate(keep)}
    rows = [sorted(new[j] for j in adj[o]) for o in keep]
    return keep, rows


@pytest.mark.parametrize("case", ["dups_loops_isolated", "er", "cl", "empty", "single_edge"])
def test_build_csr_matches_brute_force(case):
    if case == "dups_loops_isolated":
        src = np.array([0, 1, 1, 3, 3, 5, 2, 0, 6])
        dst = np.array([1, 0, 1, 5, 5, 3, 2, 6, 0])
        n = 9  # nodes 2, 4, 7, 8 end up isolated (2 only has a self-loop)
    elif case == "er":
        src, dst, n = sg.erdos_renyi(300, 0.02, 3)
    elif case == "cl":
        src, dst, n = sg.chung_lu(500, 2.5, 6.0, 4)
    elif case == "empty":
        src, dst, n = np.zeros(0, np.int64), np.zeros(0, np.int64), 4
    else:
        src, dst, n = np.array([2]), np.array([7]), 10
    g = oracle.build_csr(src, dst, n)
    keep, rows = _brute_csr(list(src), list(dst), n)
    assert g.n == len(keep)
    assert g.n_isolated == n - len(keep)
    assert list(g.old_id) == keep
    for i, r in enumerate(rows):
        assert list(g.col[g.row_ptr[i]:g.row_ptr[i + 1]]) == r
        assert g.deg[i] == len(r)
    d = g.deg.astype(np.float64)
    assert np.array_equal(g.s64, 1.0 / np.sqrt(d))
    assert np.array_equal(g.s32, (1.0 / np.sqrt(d)).astype(np.float32))


def test_build_csr_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.build_csr([0, 5], [1, 1], 5)
    with pytest.raises(ValueError):
        oracle.build_csr([-1], [1], 5)


def test_h_is_symmetric_with_unit_top_eigenvalue():
    src, dst, n = sg.erdos_renyi(200, 0.05, 11)
    g = oracle.build_csr(src, dst, n)
    h = oracle.dense_h(g)
    assert np.array_equal(h, h.T)
    lam, q = oracle.exact_eigs(g)
    # D^{1/2} 1 is an eigenvector of H with eigenvalue 1 on every component
    assert abs(lam[-1] - 1.0) < 1e-12
    assert lam[0] >= -1.0 - 1e-12
    v = np.sqrt(g.deg.astype(float))
    assert np.allclose(h @ v, v)
