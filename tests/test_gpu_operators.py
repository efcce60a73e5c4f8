"""KPM on the adjacency and Laplacian matrices (Eq. (5) shift and scale) on
the GPU against the FP64 oracle on the same probes; the normalised Laplacian
and the normalised adjacency as special cases."""
import numpy as np
import pytest
import torch

import oracle
import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")

TOL_D = 1e-5
U32 = 2.0**-24


def _tol(m):
    """Per-moment bound: the FP32 recurrence's 1e-5 plus the edge
    amplification of a relative operator perturbation u: |T_m'(+-1)| = m^2,
    and a loose Gershgorin interval (A, D - A) can put most of the spectrum
    near an edge of [-1, 1]."""
    return TOL_D + np.arange(m) ** 2 * U32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()
    yield
    nd.dos_set_plan(0, 0)


def _graph(src, dst, n):
    return nd.dos_build_csr(torch.from_numpy(np.asarray(src)).cuda(), torch.from_numpy(np.asarray(dst)).cuda(), n)


def _hub():
    s, d, n = sg.erdos_renyi(4000, 0.003, 2)
    hub = np.zeros(3000, np.int64)
    return np.concatenate([s, hub]), np.concatenate([d, 1 + np.arange(3000, dtype=np.int64)]), n


GRAPHS = {"er2000": sg.erdos_renyi(2000, 0.005, 1), "ba": sg.barabasi_albert(3000, 4, 3), "hub": _hub(),
          "cl": sg.chung_lu(6000, 2.5, 12.0, 7)}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
def test_operator_moments_match_oracle(name, op):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m, nz = 60, 24
    d, iv = nd.dos_moments_op(g, op, m, nz, 31)
    assert iv == oracle.gershgorin_interval(ref, op)
    z = oracle.probes(31, ref.old_id, nz)
    d_ref = oracle.kpm_operator(ref, z, m, op, iv)
    assert np.all(np.abs(d.cpu().numpy() - d_ref) <= _tol(m))
    # an explicit, tighter interval from the dense spectrum's bounds
    lam = np.linalg.eigvalsh(oracle.operator_matrix(ref, op).toarray()) if ref.n <= 3000 else None
    if lam is not None:
        tight = (float(lam.min()) - 1e-3, float(lam.max()) + 1e-3)
        d2, iv2 = nd.dos_moments_op(g, op, m, nz, 31, interval=tight)
        assert iv2 == tight
        assert np.all(np.abs(d2.cpu().numpy() - oracle.kpm_operator(ref, z, m, op, tight)) <= _tol(m))


def test_normalized_operators_reduce_to_h():
    src, dst, n = GRAPHS["er2000"]
    g = _graph(src, dst, n)
    m, nz = 41, 16
    dh = nd.dos_moments(g, m, nz, 5).cpu().numpy()
    d0, iv0 = nd.dos_moments_op(g, "normalized_adjacency", m, nz, 5)
    assert iv0 == (-1.0, 1.0) and np.array_equal(d0.cpu().numpy(), dh)
    dl, ivl = nd.dos_moments_op(g, "normalized_laplacian", m, nz, 5)
    sign = (-1.0) ** np.arange(m)
    assert ivl == (0.0, 2.0) and np.array_equal(dl.cpu().numpy(), sign * dh)


def test_operator_moments_low_precision_storage():
    src, dst, n = GRAPHS["ba"]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    z = oracle.probes(3, ref.old_id, 16)
    for op in ("adjacency", "laplacian"):
        d_ref = oracle.kpm_operator(ref, z, 50, op, oracle.gershgorin_interval(ref, op))
        for prec, u in (("bf16", 2.0**-8), ("fp16", 2.0**-11)):
            d, _ = nd.dos_moments_op(g, op, 50, 16, 3, prec=prec)
            assert np.abs(d.cpu().numpy() - d_ref).max() <= 4 * u


def test_operator_errors():
    g = _graph(*GRAPHS["er2000"])
    with pytest.raises(ValueError):
        nd.dos_moments_op(g, "nope", 10, 4, 1)
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    iv = (nd._binding.C.c_double * 2)()
    st = nd.lib().dos_moments_op(g.handle, 7, 0.0, 0.0, 10, 4, 1, 0, out.data_ptr(), iv, None)
    assert st == nd.DOS_EINVAL
