"""Oracle pins for the Gauss quadrature / Lanczos estimator (§3.2): Gauss
exactness against the KPM moments of the same probes, closed-form rules on
K_n and C_n, unit weights, and the PDOS of unit probes (CPU only)."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg


def _kpm(g, z, m):
    mu, _ = oracle.kpm_direct(g, z, m)
    return mu / (g.n * z.shape[1])


@pytest.mark.parametrize("m_steps", [1, 5, 12])
def test_gauss_rule_is_exact_up_to_degree_2m_minus_1(m_steps):
    for src, dst, n in (sg.erdos_renyi(400, 0.03, 3), sg.barabasi_albert(300, 3, 4)):
        g = oracle.build_csr(src, dst, n)
        z = oracle.probes(7, g.old_id, 5)
        a, b, st = oracle.lanczos(g, z, m_steps)
        assert np.all(st == m_steps)
        m = 2 * m_steps + 4
        d = oracle.gql_moments(a, b, st, m)
        dk = _kpm(g, z, m)
        k = 2 * m_steps
        assert np.abs(d[:k] - dk[:k]).max() <= 1e-12
        # the degree bound is tight: degree 2M is not integrated exactly
        assert np.abs(d[k] - dk[k]) > 1e-8


def test_weights_are_unit_and_nodes_inside_the_spectrum():
    g = oracle.build_csr(*sg.chung_lu(500, 2.5, 6.0, 5))
    z = oracle.probes(3, g.old_id, 4)
    a, b, st = oracle.lanczos(g, z, 20)
    lam, _ = oracle.exact_eigs(g)
    for tau, w in oracle.gauss_rules(a, b, st):
        assert abs(w.sum() - 1.0) <= 1e-12 and np.all(w >= 0)
        assert tau.min() >= lam.min() - 1e-10 and tau.max() <= lam.max() + 1e-10
    h = oracle.gql_histogram(a, b, st, 40)
    assert abs(h.sum() - 1.0) <= 1e-12


def test_complete_graph_two_node_rule():
    # K_n: spectrum {1, -1/(n-1)}; a generic probe's Krylov space has
    # dimension 2, so Lanczos stops after two steps with the exact rule:
    # weight (sum z)^2 / (n ||z||^2) at 1 (eigenvector 1/sqrt(n)), the rest at -1/(n-1)
    n = 9
    g = oracle.build_csr(*sg.complete(n))
    z = oracle.probes(11, g.old_id, 3)
    a, b, st = oracle.lanczos(g, z, 6)
    assert np.all(st == 2)
    for j, (tau, w) in enumerate(oracle.gauss_rules(a, b, st)):
        w1 = z[:, j].sum() ** 2 / (n * (z[:, j] @ z[:, j]))
        assert np.allclose(np.sort(tau), [-1.0 / (n - 1), 1.0], atol=1e-12)
        assert abs(w[np.argmax(tau)] - w1) <= 1e-12


def test_cycle_unit_probe_gives_the_pdos():
    # C_8 from e_0: eigenvalues cos(2 pi k / 8), each Fourier mode has |q_k(0)|^2 = 1/8;
    # the distinct values 1, +-1/sqrt 2, 0, -1 carry weights 1/8, 2/8, 2/8, 2/8, 1/8
    g = oracle.build_csr(*sg.cycle(8))
    z = np.zeros((8, 1))
    z[0, 0] = 1.0
    a, b, st = oracle.lanczos(g, z, 10)
    assert st[0] == 5
    tau, w = oracle.gauss_rules(a, b, st)[0]
    r = 1.0 / np.sqrt(2.0)
    assert np.allclose(tau, [-1.0, -r, 0.0, r, 1.0], atol=1e-12)
    assert np.allclose(w, [1 / 8, 2 / 8, 2 / 8, 2 / 8, 1 / 8], atol=1e-12)


def test_unit_probe_moments_match_exact_pdos():
    g = oracle.build_csr(*sg.erdos_renyi(150, 0.05, 9))
    lam, q = oracle.exact_eigs(g)
    k, m_steps = 17, 6
    z = np.zeros((g.n, 1))
    z[k, 0] = 1.0
    a, b, st = oracle.lanczos(g, z, m_steps)
    d = oracle.gql_moments(a, b, st, 2 * m_steps, norms2=[1.0], n=1)
    exact = oracle.exact_ldos(lam, q, 2 * m_steps)[k]
    assert np.abs(d - exact).max() <= 1e-12
