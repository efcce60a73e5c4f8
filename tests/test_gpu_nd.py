"""Nested dissection PDOS (§3.3, Algorithm 1) on the GPU against the exact
diagonal of T_m(H) from the FP64 oracle's dense eigendecomposition."""
import numpy as np
import pytest
import torch

import oracle
import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")

U32 = 2.0**-24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()
    yield


def _graph(src, dst, n):
    return nd.dos_build_csr(torch.from_numpy(np.asarray(src, np.int64)).cuda(),
                            torch.from_numpy(np.asarray(dst, np.int64)).cuda(), n)


def _tol(m):
    """FP32 recurrence: ~1e-5 over tens of steps, plus the edge amplification
    m^2 u of a relative perturbation at eigenvalues +-1 (|T_m'(+-1)| = m^2;
    grids are bipartite, so both ends are eigenvalues)."""
    return 1e-5 + np.arange(m)[:, None] ** 2 * U32


def _two_grids_and_isolated():
    s1, d1, n1 = sg.grid2d(12, 9)
    s2, d2, n2 = sg.grid2d(7, 15)
    src = np.concatenate([s1, s2 + n1])
    dst = np.concatenate([d1, d2 + n1])
    return src, dst, n1 + n2 + 5  # five isolated nodes


GRAPHS = {
    "grid": sg.grid2d(20, 30),
    "rgg": sg.random_geometric(1500, 0.05, 3),
    "er": sg.erdos_renyi(400, 0.02, 4),
    "path": sg.path(300),
    "disconnected": _two_grids_and_isolated(),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("leaf", [1, 8, 64])
def test_nd_pdos_is_the_exact_diagonal(name, leaf):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m = 40
    c, stats = nd.dos_pdos_nd(g, m, leaf_size=leaf)
    lam, q = oracle.exact_eigs(ref)
    exact = oracle.exact_ldos(lam, q, m).T  # (M, N)
    c = c.cpu().numpy()
    assert c.shape == (m, ref.n)
    assert np.all(c[0] == 1.0)
    assert np.all(np.abs(c - exact) <= _tol(m)), float(np.abs(c - exact).max())
    assert stats["tree_nodes"] >= 1 and stats["block_entries"] >= ref.n


def test_single_leaf_is_the_dense_recurrence():
    src, dst, n = GRAPHS["er"]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    c, stats = nd.dos_pdos_nd(g, 30, leaf_size=ref.n)
    assert stats["tree_nodes"] == 1 and stats["block_entries"] == ref.n * ref.n
    lam, q = oracle.exact_eigs(ref)
    assert np.all(np.abs(c.cpu().numpy() - oracle.exact_ldos(lam, q, 30).T) <= _tol(30))


def test_exact_against_the_stochastic_estimator():
    """ND needs no probes: its error is rounding, far below the stochastic
    diagonal estimator's sampling error (Eq. (12), Nz = 64)."""
    src, dst, n = GRAPHS["rgg"]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m = 30
    c_nd, _ = nd.dos_pdos_nd(g, m)
    c_st, _ = nd.ldos_moments(g, m, 64, 5)
    lam, q = oracle.exact_eigs(ref)
    exact = oracle.exact_ldos(lam, q, m).T
    err_nd = np.abs(c_nd.cpu().numpy() - exact).max()
    err_st = np.abs(c_st.cpu().numpy() - exact).max()
    assert err_nd < 1e-4 < 0.05 < err_st


def test_refuses_too_many_block_entries():
    g = _graph(*GRAPHS["er"])
    with pytest.raises(nd.DosError) as e:
        nd.dos_pdos_nd(g, 10, leaf_size=8, max_entries=1000)
    assert e.value.status == nd.DOS_ENOMEM
