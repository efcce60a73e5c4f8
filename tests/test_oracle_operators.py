"""Oracle pins for KPM on the adjacency and Laplacian matrices (Eq. (5)
shift-and-scale): closed-form spectra, Gershgorin containment, identity
probes (CPU only)."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg


def _spec(g, op):
    return np.linalg.eigvalsh(oracle.operator_matrix(g, op).toarray())


def test_closed_form_spectra():
    n = 7
    g = oracle.build_csr(*sg.complete(n))
    assert np.allclose(_spec(g, "adjacency"), [-1.0] * (n - 1) + [n - 1.0], atol=1e-12)
    assert np.allclose(_spec(g, "laplacian"), [0.0] + [float(n)] * (n - 1), atol=1e-12)
    g = oracle.build_csr(*sg.cycle(9))
    assert np.allclose(_spec(g, "adjacency"), np.sort(2 * np.cos(2 * np.pi * np.arange(9) / 9)), atol=1e-12)
    assert np.allclose(_spec(g, "laplacian"), np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(9) / 9)), atol=1e-12)
    k = 5  # star K_{1,k}: adjacency +-sqrt(k), 0 x (k-1); Laplacian 0, 1 x (k-1), k+1
    g = oracle.build_csr(*sg.star(k))
    assert np.allclose(_spec(g, "adjacency"), [-np.sqrt(k)] + [0.0] * (k - 1) + [np.sqrt(k)], atol=1e-12)
    assert np.allclose(_spec(g, "laplacian"), [0.0] + [1.0] * (k - 1) + [k + 1.0], atol=1e-12)


@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
def test_gershgorin_interval_contains_the_spectrum(op):
    g = oracle.build_csr(*sg.chung_lu(400, 2.3, 6.0, 3))
    a, b = oracle.gershgorin_interval(g, op)
    lam = _spec(g, op)
    assert lam.min() >= a - 1e-12 and lam.max() <= b + 1e-12
    d = oracle.exact_operator_moments(g, op, (a, b), 30)
    assert d[0] == pytest.approx(1.0) and np.all(np.abs(d) <= 1.0 + 1e-12)


@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
def test_identity_probes_give_exact_moments(op):
    g = oracle.build_csr(*sg.erdos_renyi(120, 0.06, 5))
    interval = oracle.gershgorin_interval(g, op)
    # N unit probes: sum_j e_j^T T_m(X~) e_j = tr T_m(X~); the estimator divides by N Nz = N^2
    d = oracle.kpm_operator(g, np.eye(g.n), 25, op, interval) * g.n
    assert np.abs(d - oracle.exact_operator_moments(g, op, interval, 25)).max() <= 1e-11


def test_first_moments_are_traces():
    # d_1 = tr((X - c) / r) / N: for A, tr A = 0; for L, tr L = sum of degrees
    g = oracle.build_csr(*sg.barabasi_albert(200, 3, 7))
    for op in ("adjacency", "laplacian"):
        a, b = oracle.gershgorin_interval(g, op)
        c, r = 0.5 * (a + b), 0.5 * (b - a)
        tr = 0.0 if op == "adjacency" else float(np.diff(g.row_ptr).sum())
        d = oracle.exact_operator_moments(g, op, (a, b), 2)
        assert d[1] == pytest.approx((tr / g.n - c) / r, abs=1e-12)
