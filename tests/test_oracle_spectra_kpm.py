"""Oracle pins: exact moments against closed-form spectra, and the sparse
KPM recurrences against the exact moments (CPU only)."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg


def _t(m, x):
    return np.cos(m * np.arccos(np.clip(x, -1.0, 1.0)))


M = 40


def _moments_of(points, weights=None):
    points = np.asarray(points, float)
    w = np.full(points.size, 1.0 / points.size) if weights is None else np.asarray(weights, float)
    return np.array([(w * _t(m, points)).sum() for m in range(M)])


def test_complete_graph_closed_form():
    n = 12
    g = oracle.build_csr(*sg.complete(n))
    lam, _ = oracle.exact_eigs(g)
    # normalized adjacency of K_n: eigenvalue 1 once, -1/(n-1) with multiplicity n-1
    expect = np.array([1.0] + [-1.0 / (n - 1)] * (n - 1))
    assert np.allclose(np.sort(lam), np.sort(expect), atol=1e-12)
    assert np.allclose(oracle.exact_moments(lam, M), _moments_of(expect), atol=1e-12)


@pytest.mark.parametrize("n", [7, 10])
def test_cycle_closed_form(n):
    g = oracle.build_csr(*sg.cycle(n))
    lam, _ = oracle.exact_eigs(g)
    expect = np.cos(2 * np.pi * np.arange(n) / n)
    assert np.allclose(np.sort(lam), np.sort(expect), atol=1e-12)
    assert np.allclose(oracle.exact_moments(lam, M), _moments_of(expect), atol=1e-12)


def test_star_and_complete_bipartite_closed_form():
    g = oracle.build_csr(*sg.star(9))
    lam, _ = oracle.exact_eigs(g)
    assert np.allclose(np.sort(lam), [-1.0] + [0.0] * 8 + [1.0], atol=1e-12)
    g = oracle.build_csr(*sg.complete_bipartite(3, 5))
    lam, _ = oracle.exact_eigs(g)
    assert np.allclose(np.sort(lam), [-1.0] + [0.0] * 6 + [1.0], atol=1e-12)


def test_bipartite_odd_moments_vanish():
    # a path is bipartite: spectrum symmetric about 0, odd moments 0
    g = oracle.build_csr(*sg.path(31))
    lam, _ = oracle.exact_eigs(g)
    d = oracle.exact_moments(lam, M)
    assert np.abs(d[1::2]).max() < 1e-13
    # path P_n normalized adjacency eigenvalues: cos(pi k/(n-1)), k = 0..n-1
    expect = np.cos(np.pi * np.arange(31) / 30)
    assert np.allclose(np.sort(lam), np.sort(expect), atol=1e-12)


def test_trace_identities_t1_t2():
    src, dst, n = sg.chung_lu(400, 2.5, 8.0, 21)
    g = oracle.build_csr(src, dst, n)
    lam, _ = oracle.exact_eigs(g)
    d = oracle.exact_moments(lam, 3)
    assert abs(d[1]) < 1e-13  # tr T_1(H) = tr H = 0 (no self-loops)
    # tr T_2(H) = 2 sum_ij A_ij / (d_i d_j) - N, summed straight from the CSR
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    s2 = np.sum(1.0 / (g.deg[rows].astype(float) * g.deg[g.col].astype(float)))
    assert abs(d[2] * g.n - (2.0 * s2 - g.n)) < 1e-9


def test_exact_ldos_sums_to_dos_and_matches_matrix_polynomial():
    src, dst, n = sg.erdos_renyi(60, 0.1, 5)
    g = oracle.build_csr(src, dst, n)
    lam, q = oracle.exact_eigs(g)
    c = oracle.exact_ldos(lam, q, 12)
    d = oracle.exact_moments(lam, 12)
    assert np.allclose(c.mean(axis=0), d, atol=1e-13)
    h = oracle.dense_h(g)
    # T_3(H) = 4H^3 - 3H directly from matrix powers
    t3 = 4 * h @ h @ h - 3 * h
    assert np.allclose(np.diag(t3), c[:, 3], atol=1e-12)


def test_kpm_direct_with_identity_probes_is_exact_trace():
    src, dst, n = sg.chung_lu(150, 2.3, 6.0, 8)
    g = oracle.build_csr(src, dst, n)
    lam, q = oracle.exact_eigs(g)
    z = np.eye(g.n)
    mu, c = oracle.kpm_direct(g, z, 30, ldos=True)
    assert np.allclose(mu / g.n, oracle.exact_moments(lam, 30), atol=1e-11)
    # with Z = I, C[k, m] = T_m(H)_kk / N
    assert np.allclose(c * g.n, oracle.exact_ldos(lam, q, 30), atol=1e-11)


def test_kpm_direct_random_probes_match_eigen_form():
    src, dst, n = sg.erdos_renyi(120, 0.06, 9)
    g = oracle.build_csr(src, dst, n)
    lam, q = oracle.exact_eigs(g)
    z = oracle.probes(3, g.old_id, 7)
    mu, c = oracle.kpm_direct(g, z, 25, ldos=True)
    w = q.T @ z  # probe weights in the eigenbasis
    t = oracle.cheb_values(lam, 25)
    mu_ref = t @ (w * w).sum(axis=1)
    assert np.allclose(mu, mu_ref, rtol=1e-11, atol=1e-9)
    # per-node: (1/Nz) sum_j z_kj (Q T_m(Lambda) Q^T z_j)_k
    for m in (0, 1, 5, 24):
        tz = q @ (t[m][:, None] * w)
        assert np.allclose(c[:, m], (z * tz).sum(axis=1) / z.shape[1], atol=1e-11)


@pytest.mark.parametrize("m_count", [2, 3, 50, 51])
def test_doubled_equals_direct(m_count):
    src, dst, n = sg.chung_lu(800, 2.5, 10.0, 12)
    g = oracle.build_csr(src, dst, n)
    z = oracle.probes(11, g.old_id, 5)
    mu_d, _ = oracle.kpm_direct(g, z, m_count)
    mu_2 = oracle.kpm_doubled(g, z, m_count)
    assert np.allclose(mu_2, mu_d, rtol=1e-10, atol=1e-8)
    assert mu_d[0] == g.n * 5  # Rademacher: ||z||^2 = N per probe


def test_hutchinson_mean_converges_to_exact():
    src, dst, n = sg.erdos_renyi(200, 0.04, 2)
    g = oracle.build_csr(src, dst, n)
    lam, _ = oracle.exact_eigs(g)
    d_ex = oracle.exact_moments(lam, 10)
    est = []
    for seed in range(40):
        z = oracle.probes(1000 + seed, g.old_id, 10)
        mu, _ = oracle.kpm_direct(g, z, 10)
        est.append(mu / (g.n * 10))
    est = np.array(est)
    se = est.std(axis=0, ddof=1) / np.sqrt(len(est))
    err = np.abs(est.mean(axis=0) - d_ex)
    assert np.all(err[1:] <= 5 * se[1:] + 1e-12)
    # error of a single estimate shrinks like 1/sqrt(N Nz): Nz=40 vs Nz=10
    z40 = oracle.probes(77, g.old_id, 40)
    mu40, _ = oracle.kpm_direct(g, z40, 10)
    assert np.abs(mu40 / (g.n * 40) - d_ex)[1:].mean() < 2.5 * se[1:].mean() * np.sqrt(40) / 2
