"""Traces and diagonals of matrix functions (§6) on the GPU against the FP64
oracle: LDOS moments of A and D - A (Eq. (12) on X~ of Eq. (5)) on the same
probes, Chebyshev coefficients, the trace and diagonal contractions, and the
Estrada index and subgraph centrality end to end.

Tolerances (derived from the arithmetic):
* LDOS entries on X~: the FP32 bound of H's LDOS test (1e-4 for M <= 100:
  a random walk of per-step roundings carried by |U_{m-s}| <= m - s + 1) plus
  the edge amplification m^2 u of a relative operator perturbation at
  eigenvalues near +-1 (a tight interval puts the spectrum's ends there).
* Coefficients: FP64 sums of K = max(4M, 256) terms in another order:
  1e-12 of the largest coefficient.
* Trace: N sum_m |g_m| tol_m (the DOS moments' bound carried by the
  coefficients), plus 1e-12 relative.
* Diagonal: sum_m |g_m| tol_m (the LDOS bound) plus the FP32 contraction,
  M u sum_m |g_m C_m| (products and sums of g_m / max|g| in FP32).
"""
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
    return nd.dos_build_csr(torch.from_numpy(np.asarray(src)).cuda(), torch.from_numpy(np.asarray(dst)).cuda(), n)


def _hub():
    s, d, n = sg.erdos_renyi(4000, 0.003, 2)
    return np.concatenate([s, np.zeros(3000, np.int64)]), np.concatenate([d, 1 + np.arange(3000)]), n


GRAPHS = {"er2000": sg.erdos_renyi(2000, 0.005, 1), "ba": sg.barabasi_albert(3000, 4, 3), "hub": _hub()}


def _tol_c(m):
    return 1e-4 + np.arange(m) ** 2 * U32


def _tol_d(m):
    return 1e-5 + np.arange(m) ** 2 * U32


def _interval(name, op, kind):
    ref = oracle.build_csr(*GRAPHS[name])
    if kind == "gershgorin":
        return oracle.gershgorin_interval(ref, op)
    # the oracle's own Ritz interval (FP64 Lanczos on the same probes)
    return oracle.spectral_interval(ref, op, oracle.probes(41, ref.old_id, 8), 30, bound="ritz")


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
@pytest.mark.parametrize("kind", ["gershgorin", "ritz"])
def test_ldos_op_matches_oracle(name, op, kind):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m, nz = 60, 20
    iv = _interval(name, op, kind)
    c, d, iv2 = nd.ldos_moments_op(g, op, m, nz, 7, interval=iv)
    assert iv2 == tuple(iv)
    d_ref, c_ref = oracle.ldos_operator(ref, oracle.probes(7, ref.old_id, nz), m, op, iv)
    c = c.cpu().numpy()
    assert np.all(c[0] == 1.0)
    assert np.all(np.abs(c.T - c_ref) <= _tol_c(m)[None, :])
    assert np.all(np.abs(d.cpu().numpy() - d_ref) <= _tol_d(m))
    # the doubled DOS path on the same operator estimates the same moments
    d2, _ = nd.dos_moments_op(g, op, m, nz, 7, interval=iv)
    assert np.all(np.abs(d2.cpu().numpy() - d.cpu().numpy()) <= 2 * _tol_d(m))


def test_ldos_op_normalized_operators_reduce_to_h():
    g = _graph(*GRAPHS["ba"])
    m, nz = 31, 16
    c_h, d_h = nd.ldos_moments(g, m, nz, 9)
    c0, d0, iv0 = nd.ldos_moments_op(g, "normalized_adjacency", m, nz, 9)
    assert iv0 == (-1.0, 1.0) and torch.equal(c0, c_h) and torch.equal(d0, d_h)
    c3, d3, iv3 = nd.ldos_moments_op(g, "normalized_laplacian", m, nz, 9)
    sign = torch.tensor((-1.0) ** np.arange(m), device="cuda")
    assert iv3 == (0.0, 2.0)
    assert torch.equal(c3, c_h * sign[:, None].float()) and torch.equal(d3, d_h * sign)


@pytest.mark.parametrize("fn,p,interval", [("exp", 1.0, (-12.0, 30.0)), ("exp", -0.5, (0.0, 40.0)),
                                           ("resolvent", 0.02, (-12.0, 30.0)), ("exp", 3.0, (-1.0, 1.0))])
@pytest.mark.parametrize("m", [1, 7, 200])
def test_coefficients_match_oracle(fn, p, interval, m):
    g = nd.dos_fn_coeffs(fn, p, interval, m).cpu().numpy()
    ref = oracle.cheb_coeffs(fn, p, interval, m)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [1000, 1001, 4096 + 3])
@pytest.mark.parametrize("m", [5, 100, 2100])
def test_diag_kernel_on_oracle_moments(n, m):
    """The contraction alone, on FP32 moments derived from the oracle's (both
    vector widths: n % 4 == 0 and ragged; more moments than one staged
    chunk of coefficients)."""
    rng = np.random.default_rng(n + m)
    cm = rng.uniform(-1.0, 1.0, (m, n)).astype(np.float32)
    coef = oracle.cheb_coeffs("exp", 2.0, (-3.0, 5.0), m)
    out = nd.dos_fn_diag(torch.from_numpy(cm).cuda(), torch.from_numpy(coef).cuda()).cpu().numpy()
    want = oracle.diag_fn(cm.T.astype(np.float64), coef)
    bound = (m + 2) * U32 * (np.abs(coef)[None, :] @ np.abs(cm.astype(np.float64))).ravel()
    assert np.all(np.abs(out - want) <= bound)


@pytest.mark.parametrize("name", ["er2000", "ba"])
@pytest.mark.parametrize("op,fn,p", [("adjacency", "exp", 1.0), ("adjacency", "resolvent", 0.05),
                                     ("laplacian", "exp", -0.1)])
def test_trace_and_diag_match_oracle(name, op, fn, p):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m, nz = 60, 16
    iv = _interval(name, op, "ritz")
    if fn == "resolvent" and not (1 - p * iv[0]) * (1 - p * iv[1]) > 0:
        pytest.skip("pole inside the interval")
    z = oracle.probes(5, ref.old_id, nz)
    coef_ref = oracle.cheb_coeffs(fn, p, iv, m)
    # trace
    d, _ = nd.dos_moments_op(g, op, m, nz, 5, interval=iv)
    coef = nd.dos_fn_coeffs(fn, p, iv, m)
    tr = nd.dos_fn_trace(g, coef, d).item()
    d_ref = oracle.kpm_operator(ref, z, m, op, iv)
    tr_ref = oracle.trace_fn(d_ref, coef_ref, ref.n, n - ref.n)
    bound = ref.n * np.sum(np.abs(coef_ref) * _tol_d(m)) + 1e-12 * abs(tr_ref)
    assert abs(tr - tr_ref) <= bound
    # diagonal
    c, _, _ = nd.ldos_moments_op(g, op, m, nz, 5, interval=iv)
    diag = nd.dos_fn_diag(c, coef).cpu().numpy()
    _, c_ref = oracle.ldos_operator(ref, z, m, op, iv)
    diag_ref = oracle.diag_fn(c_ref, coef_ref)
    bound = np.abs(coef_ref) @ _tol_c(m) + (m + 2) * U32 * (np.abs(c_ref) @ np.abs(coef_ref))
    assert np.all(np.abs(diag - diag_ref) <= bound)


def test_estrada_index_and_subgraph_centrality_end_to_end():
    """matrix_function_trace / _diag (Lanczos interval, moments,
    coefficients, contraction) against the dense exact values: the error is
    the stochastic estimator's, within 6 of its standard deviations
    (Rademacher: Var tr = 2 sum_{i != j} F_ij^2 / Nz; Var F_kk = sum_{j != k}
    F_kj^2 / Nz), plus isolated nodes counted exactly."""
    src, dst, n = sg.erdos_renyi(1500, 0.004, 8)
    n_total = n + 7  # seven nodes without edges
    ref = oracle.build_csr(src, dst, n_total)
    g = _graph(src, dst, n_total)
    nz, m = 64, 80
    f = np.linalg.eigh(oracle.operator_matrix(ref, "adjacency").toarray())
    fm = (f[1] * np.exp(f[0])) @ f[1].T
    off2 = fm * fm - np.diag(np.diag(fm) ** 2)
    ee, iv = nd.matrix_function_trace(g, "adjacency", "exp", 1.0, M=m, Nz=nz, seed=3)
    lam = f[0]
    assert iv[0] <= lam.min() and iv[1] >= lam.max()
    g_abs = np.abs(oracle.cheb_coeffs("exp", 1.0, iv, m))
    exact = oracle.exact_fn_trace(ref, "adjacency", "exp", 1.0, n_isolated=n_total - ref.n)
    sd = np.sqrt(2.0 * off2.sum() / nz)
    assert abs(ee - exact) <= 6 * sd + ref.n * np.sum(g_abs * _tol_d(m))
    sc, iv2 = nd.matrix_function_diag(g, "adjacency", "exp", 1.0, M=m, Nz=nz, seed=3)
    assert iv2 == iv
    sd_k = np.sqrt(off2.sum(axis=1) / nz)
    assert np.all(np.abs(sc.cpu().numpy() - np.diag(fm)) <= 6 * sd_k + np.sum(g_abs * _tol_c(m)))


def test_function_errors():
    g = _graph(*GRAPHS["er2000"])
    with pytest.raises(ValueError):
        nd.dos_fn_coeffs("nope", 1.0, (-1.0, 1.0), 10)
    with pytest.raises(nd.DosError) as e:
        nd.dos_fn_coeffs("resolvent", 0.5, (-1.0, 3.0), 10)  # pole at x = 2
    assert e.value.status == nd.DOS_EINVAL
    with pytest.raises(nd.DosError) as e:
        nd.dos_fn_coeffs("exp", 1.0, (2.0, 2.0), 10)
    assert e.value.status == nd.DOS_EINVAL
    with pytest.raises(ValueError):
        nd.ldos_moments_op(g, "nope", 10, 4, 1)
    c = torch.empty((10, g.n), dtype=torch.float32, device="cuda")
    iv = (nd._binding.C.c_double * 2)()
    assert nd.lib().ldos_moments_op(g.handle, 9, 0.0, 0.0, 10, 4, 1, c.data_ptr(), None, iv, None) == nd.DOS_EINVAL
