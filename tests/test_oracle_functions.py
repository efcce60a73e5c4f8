"""Oracle pins for traces and diagonals of matrix functions from (L)DOS
moments (§6; Eq. (5), (10)-(12)): Chebyshev coefficients against the Bessel
and geometric closed forms, the Estrada index, subgraph and resolvent
centralities of K_n and stars in closed form, and identity probes giving the
exact diagonal of exp(A) (CPU only)."""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.special import iv

import oracle
import synthgraphs as sg


@pytest.mark.parametrize("p,interval", [(1.0, (-5.0, 7.0)), (-0.3, (0.0, 20.0)), (2.5, (-1.0, 1.0))])
def test_exp_coefficients_are_bessel(p, interval):
    # exp(p (c + r x)) = e^{pc} [I_0(pr) + 2 sum_k I_k(pr) T_k(x)]
    a, b = interval
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    m = 40
    g = oracle.cheb_coeffs("exp", p, interval, m)
    want = np.exp(p * c) * iv(np.arange(m), p * r) * np.where(np.arange(m) == 0, 1.0, 2.0)
    assert np.abs(g - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("p,interval", [(0.05, (-5.0, 7.0)), (-0.1, (0.0, 6.0))])
def test_resolvent_coefficients_are_geometric(p, interval):
    # 1 / (alpha - beta x) = (1 + 2 sum_k rho^k T_k(x)) / sqrt(alpha^2 - beta^2),
    # rho = (alpha - sqrt(alpha^2 - beta^2)) / beta  (|beta| < alpha)
    a, b = interval
    c, r = 0.5 * (a + b), 0.5 * (b - a)
    alpha, beta = 1.0 - p * c, p * r
    s = np.sqrt(alpha * alpha - beta * beta)
    rho = (alpha - s) / beta
    m = 30
    want = np.where(np.arange(m) == 0, 1.0, 2.0 * rho ** np.arange(m)) / s
    g = oracle.cheb_coeffs("resolvent", p, interval, m)
    assert np.abs(g - want).max() <= 1e-13 * np.abs(want).max()


def test_closed_form_traces_and_diagonals():
    n, s = 8, 6
    kn = oracle.build_csr(*sg.complete(n))
    assert oracle.exact_fn_trace(kn, "adjacency", "exp", 1.0) == pytest.approx(
        np.exp(n - 1.0) + (n - 1) * np.exp(-1.0), rel=1e-13)
    star = oracle.build_csr(*sg.star(s))
    rs = np.sqrt(s)
    assert oracle.exact_fn_trace(star, "adjacency", "exp", 1.0) == pytest.approx(
        np.exp(rs) + np.exp(-rs) + (s - 1), rel=1e-13)
    center = int(np.argmax(np.diff(star.row_ptr)))
    leaf = [k for k in range(star.n) if k != center]
    sc = oracle.exact_fn_diag(star, "adjacency", "exp", 1.0)
    assert sc[center] == pytest.approx(np.cosh(rs), rel=1e-13)
    assert np.allclose(sc[leaf], 1.0 + (np.cosh(rs) - 1.0) / s, rtol=1e-13)
    p = 0.3
    rc = oracle.exact_fn_diag(star, "adjacency", "resolvent", p)
    assert rc[center] == pytest.approx(1.0 / (1.0 - p * p * s), rel=1e-13)
    assert np.allclose(rc[leaf], 1.0 + p * p / (1.0 - p * p * s), rtol=1e-13)
    # the heat kernel trace of L: sum exp(-t lambda), lambda in {0, 1 x (s-1), s+1}
    t = 0.7
    assert oracle.exact_fn_trace(star, "laplacian", "exp", -t) == pytest.approx(
        1.0 + (s - 1) * np.exp(-t) + np.exp(-t * (s + 1)), rel=1e-13)


@pytest.mark.parametrize("op,fn,p", [("adjacency", "exp", 1.0), ("adjacency", "exp", 0.5),
                                     ("adjacency", "resolvent", 0.04), ("laplacian", "exp", -0.2)])
def test_identity_probes_give_the_exact_diagonal_and_trace(op, fn, p):
    """N unit probes make Eq. (12) exact: N C[k, m] = T_m(X~)_kk; with enough
    moments the Chebyshev sums match the dense eigendecomposition (and
    scipy's expm for exp(p A))."""
    g = oracle.build_csr(*sg.erdos_renyi(150, 0.06, 4))
    interval = oracle.gershgorin_interval(g, op)
    m = 80
    d, cm = oracle.ldos_operator(g, np.eye(g.n), m, op, interval)
    coef = oracle.cheb_coeffs(fn, p, interval, m)
    diag = oracle.diag_fn(g.n * cm, coef)
    exact = oracle.exact_fn_diag(g, op, fn, p)
    assert np.abs(diag - exact).max() <= 1e-10 * np.abs(exact).max()
    if fn == "exp":
        assert np.allclose(exact, np.diag(expm(p * oracle.operator_matrix(g, op).toarray())), rtol=1e-12)
    # the sum of g_m d_m cancels: sum |g_m| is ~e^{p r} (here up to e^15)
    # against a trace of ~e^{lambda_max}, so allow 1e-9
    tr = oracle.trace_fn(g.n * d, coef, g.n, n_isolated=3)
    assert tr == pytest.approx(oracle.exact_fn_trace(g, op, fn, p, n_isolated=3), rel=1e-9)


def test_ldos_operator_moments_average_to_kpm_operator():
    g = oracle.build_csr(*sg.barabasi_albert(200, 3, 5))
    z = oracle.probes(3, g.old_id, 8)
    for op in ("adjacency", "laplacian"):
        iv_ = oracle.gershgorin_interval(g, op)
        d, cm = oracle.ldos_operator(g, z, 30, op, iv_)
        assert np.abs(d - oracle.kpm_operator(g, z, 30, op, iv_)).max() <= 1e-12
        assert np.all(cm[:, 0] == 1.0)
