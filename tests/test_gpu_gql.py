"""Gauss quadrature and Lanczos (§3.2) on the GPU against the FP64 oracle:
Lanczos coefficients, Gauss exactness of the rules' Chebyshev moments against
the oracle's KPM moments on the same probes, the FP64 rule and histogram
kernels on the oracle's own coefficients, and early stops (breakdown)."""
import numpy as np
import pytest
import torch

import oracle
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


def _graph(src, dst, n):
    return nd.dos_build_csr(torch.from_numpy(np.asarray(src)).cuda(), torch.from_numpy(np.asarray(dst)).cuda(), n)


GRAPHS = {
    "er2000": sg.erdos_renyi(2000, 0.005, 1),
    "cl_twins": sg.add_twin_leaves(*sg.chung_lu(6000, 2.5, 12.0, 7), 300, 8),
    "ba": sg.barabasi_albert(3000, 4, 3),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("nz", [1, 5, 16, 37])
def test_lanczos_coefficients_match_oracle(name, nz):
    """FP32 vectors against the FP64 oracle over 10 steps.  Each coefficient is
    an inner product of O(1)-norm vectors, so a few float32 rounding steps per
    iteration give errors near 1e-6; without reorthogonalisation they grow
    from step to step, and 1e-4 bounds 10 steps."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m = 10
    a, b, st = nd.dos_lanczos(g, m, nz, 19)
    z = oracle.probes(19, ref.old_id, nz)
    ar, br, sr = oracle.lanczos(ref, z, m)
    assert np.array_equal(st.cpu().numpy(), sr)
    assert np.abs(a.cpu().numpy() - ar).max() <= 1e-4
    assert np.abs(b.cpu().numpy() - br).max() <= 1e-4
    assert np.abs(a.cpu().numpy()[:, 0] - ar[:, 0]).max() <= 1e-6


@pytest.mark.parametrize("name", list(GRAPHS))
def test_gauss_rules_are_exact_against_kpm(name):
    """The rules' moments equal the KPM moments of the same probes up to degree
    2M - 1; at FP32 this holds to the KPM tolerance (1e-5)."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m, nz = 20, 16
    a, b, st = nd.dos_lanczos(g, m, nz, 23)
    d = nd.dos_gql_moments(a, b, st, 2 * m).cpu().numpy()
    mu, _ = oracle.kpm_direct(ref, oracle.probes(23, ref.old_id, nz), 2 * m)
    assert abs(d[0] - 1.0) <= 1e-12
    assert np.abs(d - mu / (ref.n * nz)).max() <= 1e-5


def test_rule_and_histogram_kernels_on_oracle_coefficients():
    """The FP64 stages (bisection nodes, Christoffel weights, Chebyshev
    recurrence on the tridiagonal, binning) on the oracle's coefficients."""
    src, dst, n = GRAPHS["cl_twins"]
    ref = oracle.build_csr(src, dst, n)
    z = oracle.probes(29, ref.old_id, 12)
    ar, br, sr = oracle.lanczos(ref, z, 40)
    a, b = torch.from_numpy(ar).cuda(), torch.from_numpy(br).cuda()
    st = torch.from_numpy(sr.astype(np.int32)).cuda()
    nodes, weights = nd.dos_gauss_rules(a, b, st)
    nodes, weights = nodes.cpu().numpy(), weights.cpu().numpy()
    for j, (tau, w) in enumerate(oracle.gauss_rules(ar, br, sr)):
        k = sr[j]
        assert np.abs(nodes[j, :k] - tau).max() <= 1e-12
        assert np.abs(weights[j, :k] - w).max() <= 1e-10
        assert not nodes[j, k:].any() and not weights[j, k:].any()
    d = nd.dos_gql_moments(a, b, st, 100).cpu().numpy()
    assert np.abs(d - oracle.gql_moments(ar, br, sr, 100)).max() <= 1e-11
    for bins in (7, 200):
        h = nd.dos_gql_histogram(torch.from_numpy(nodes).cuda(), torch.from_numpy(weights).cuda(), bins).cpu().numpy()
        assert np.abs(h - oracle.gql_histogram(ar, br, sr, bins)).max() <= 1e-10


def test_breakdown_stops_a_probe():
    # K_n: the Krylov space of a generic probe has dimension 2
    g = _graph(*sg.complete(40))
    a, b, st = nd.dos_lanczos(g, 8, 6, 3)
    assert np.all(st.cpu().numpy() == 2)
    nodes, weights = nd.dos_gauss_rules(a, b, st)
    tau = nodes.cpu().numpy()[:, :2]
    assert np.allclose(np.sort(tau, axis=1), [[-1.0 / 39, 1.0]] * 6, atol=1e-6)
    assert np.allclose(weights.cpu().numpy().sum(axis=1), 1.0, atol=1e-12)


def test_errors():
    g = _graph(*GRAPHS["er2000"])
    for kw in (dict(M=0, Nz=4), dict(M=4, Nz=0), dict(M=4, Nz=129)):
        with pytest.raises(nd.DosError):
            nd.dos_lanczos(g, kw["M"], kw["Nz"], 1)
