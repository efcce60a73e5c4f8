"""Oracle pins: twin-motif classes, probe projection, Jackson damping and the
spectral histogram (CPU only)."""
import numpy as np
import pytest
from scipy import integrate

import oracle
import synthgraphs as sg


def _p_matrix(class_id):
    ids = np.unique(class_id)
    p = np.zeros((class_id.size, ids.size))
    for k, c in enumerate(ids):
        mem = class_id == c
        p[mem, k] = 1.0 / np.sqrt(mem.sum())
    return p


def test_star_is_one_twin_class():
    g = oracle.build_csr(*sg.star(6))
    cid, removed = oracle.twin_classes(g)
    assert removed == 5
    assert list(cid) == [0, 1, 1, 1, 1, 1, 1]


def test_complete_bipartite_two_classes():
    g = oracle.build_csr(*sg.complete_bipartite(3, 4))
    cid, removed = oracle.twin_classes(g)
    assert removed == 3 + 4 - 2
    assert list(cid) == [0, 0, 0, 3, 3, 3, 3]


def test_adjacent_nodes_are_never_twins():
    # in K_n every pair is adjacent; open neighbourhoods all differ
    g = oracle.build_csr(*sg.complete(5))
    cid, removed = oracle.twin_classes(g)
    assert removed == 0 and list(cid) == list(range(5))


def test_twins_remove_zero_eigenvalues_and_projection_spectrum():
    src, dst, n = sg.chung_lu(300, 2.3, 4.0, 31)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 20, 32)
    g = oracle.build_csr(src, dst, n)
    cid, removed = oracle.twin_classes(g)
    assert removed >= 20
    lam, _ = oracle.exact_eigs(g)
    assert np.sum(np.abs(lam) < 1e-9) >= removed
    p = _p_matrix(cid)
    assert np.allclose(p.T @ p, np.eye(p.shape[1]), atol=1e-12)
    hr = p.T @ oracle.dense_h(g) @ p
    lam_r = np.linalg.eigvalsh(hr)
    # spec(P^T H P) = spec(H) minus `removed` copies of 0
    zeros = np.nonzero(np.abs(lam) < 1e-9)[0]
    keep = np.ones(lam.size, bool)
    keep[zeros[:removed]] = False
    assert lam_r.size == g.n - removed
    assert np.allclose(np.sort(lam_r), np.sort(lam[keep]), atol=1e-9)


def test_projection_is_class_mean_and_matches_ppt():
    src, dst, n = sg.star(4)
    src = np.concatenate([src, [5, 5]])
    dst = np.concatenate([dst, [6, 7]])
    g = oracle.build_csr(src, dst, 8)
    cid, _ = oracle.twin_classes(g)
    z = oracle.probes(5, g.old_id, 9)
    zr = oracle.project_probes(z, cid)
    p = _p_matrix(cid)
    assert np.allclose(zr, p @ (p.T @ z), atol=1e-14)
    assert np.allclose(oracle.project_probes(zr, cid), zr)


def test_filtered_moments_estimate_reduced_trace():
    src, dst, n = sg.chung_lu(250, 2.4, 5.0, 41)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 15, 42)
    g = oracle.build_csr(src, dst, n)
    cid, removed = oracle.twin_classes(g)
    r = g.n - removed
    p = _p_matrix(cid)
    lam_r = np.linalg.eigvalsh(p.T @ oracle.dense_h(g) @ p)
    d_r = oracle.exact_moments(lam_r, 8)
    # identity-like probes: columns of P P^T give tr(P^T T_m(H) P) exactly
    z = p @ p.T
    mu, _ = oracle.kpm_direct(g, z, 8)
    assert np.allclose(mu / r, d_r, atol=1e-11)


def test_jackson_coefficients_properties():
    for m in (2, 10, 100, 500):
        g = oracle.jackson(m)
        assert abs(g[0] - 1.0) < 1e-15
        assert abs(g[1] - np.cos(np.pi / (m + 1))) < 1e-14
        assert np.all(np.diff(g) < 0) and g[-1] > 0
    # the damped kernel K(x, y) = g_0 + 2 sum g_m T_m(x) T_m(y) is nonnegative
    g = oracle.jackson(40)
    x = np.cos(np.linspace(0, np.pi, 301))
    t = oracle.cheb_values(x, 40)
    k = g[0] + 2.0 * np.einsum("m,mi,mj->ij", g[1:], t[1:], t[1:])
    assert k.min() > -1e-10


@pytest.mark.parametrize("m", [0, 1, 2, 7, 30])
def test_bin_integrals_against_quadrature(m):
    nb = 10
    i_cf = oracle.bin_integrals(m + 1, nb)[m]
    e = oracle.bin_edges(nb)
    for b in range(nb):
        a, c = e[b], e[b + 1]
        f = lambda x: np.cos(m * np.arccos(x)) / np.pi  # noqa: E731
        if b == 0:
            val, _ = integrate.quad(lambda x: f(x) / np.sqrt(1 - x), a, c, weight="alg", wvar=(-0.5, 0.0))
        elif b == nb - 1:
            val, _ = integrate.quad(lambda x: f(x) / np.sqrt(1 + x), a, c, weight="alg", wvar=(0.0, -0.5))
        else:
            val, _ = integrate.quad(lambda x: f(x) / np.sqrt(1 - x * x), a, c)
        assert abs(val - i_cf[b]) < 1e-9


def test_histogram_unit_mass_and_positive_with_exact_moments():
    src, dst, n = sg.barabasi_albert(400, 3, 6)
    g = oracle.build_csr(src, dst, n)
    lam, _ = oracle.exact_eigs(g)
    for mm in (20, 100, 300):
        d = oracle.exact_moments(lam, mm)
        h = oracle.histogram(d, 50)
        assert abs(h.sum() - 1.0) < 1e-12
        assert h.min() > -1e-12
    # without damping the sum is still d_0 but Gibbs ringing can go negative
    h0 = oracle.histogram(oracle.exact_moments(lam, 100), 50, kernel="none")
    assert abs(h0.sum() - 1.0) < 1e-12


def test_histogram_independent_evaluation():
    # h_b = (1/N) sum_i integral_bin K_M(x, lambda_i) w(x) dx, evaluated by quadrature
    src, dst, n = sg.erdos_renyi(40, 0.15, 3)
    g = oracle.build_csr(src, dst, n)
    lam, _ = oracle.exact_eigs(g)
    mm, nb = 12, 8
    h = oracle.histogram(oracle.exact_moments(lam, mm), nb)
    gj = oracle.jackson(mm)
    e = oracle.bin_edges(nb)

    def dens(theta):  # density in theta = arccos x, where dx / (pi sqrt(1-x^2)) = dtheta / pi
        x = np.cos(theta)
        s = 0.0
        for lm in lam:
            tl = np.cos(np.arange(mm) * np.arccos(np.clip(lm, -1, 1)))
            tx = np.cos(np.arange(mm) * theta)
            s += gj[0] + 2.0 * np.dot(gj[1:] * tl[1:], tx[1:])
        return s / (lam.size * np.pi) + 0.0 * x

    for b in range(nb):
        val, _ = integrate.quad(dens, np.arccos(e[b + 1]), np.arccos(e[b]), limit=200)
        assert abs(val - h[b]) < 1e-9


def test_point_mass_histogram_edges():
    h = oracle.point_mass_histogram([0.0, -1.0, 1.0, 0.3], [1, 1, 1, 1], 4)
    # 0.0 is an interior edge of 4 bins over [-1, 1]: split between bins 1 and 2
    assert np.allclose(h, [1.0, 0.5, 0.5 + 1.0, 1.0])
    h = oracle.point_mass_histogram([0.0], [1.0], 5)
    assert np.allclose(h, [0, 0, 1, 0, 0])


def test_jackson_error_decreases_with_moments():
    src, dst, n = sg.chung_lu(600, 2.5, 6.0, 14)
    g = oracle.build_csr(src, dst, n)
    lam, _ = oracle.exact_eigs(g)
    cid, removed = oracle.twin_classes(g)
    h_ex = oracle.exact_histogram(lam, 20)
    errs = [oracle.l1(oracle.histogram(oracle.exact_moments(lam, mm), 20), h_ex) for mm in (25, 100, 400)]
    assert errs[0] > errs[1] > errs[2]


def test_filtered_density_recovers_spectrum_better():
    # the lambda = 0 spike of twin leaves, filtered and added back as a point mass,
    # lowers the L1 error at a fixed moment count (§3.4, Fig. 4)
    src, dst, n = sg.chung_lu(500, 2.3, 4.0, 51)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 60, 52)
    g = oracle.build_csr(src, dst, n)
    lam, _ = oracle.exact_eigs(g)
    cid, removed = oracle.twin_classes(g)
    r = g.n - removed
    p = _p_matrix(cid)
    lam_r = np.linalg.eigvalsh(p.T @ oracle.dense_h(g) @ p)
    nb, mm = 40, 60
    h_ex = oracle.exact_histogram(lam, nb)
    h_plain = oracle.histogram(oracle.exact_moments(lam, mm), nb)
    h_filt = (r / g.n) * oracle.histogram(oracle.exact_moments(lam_r, mm), nb)
    h_filt += oracle.point_mass_histogram([0.0], [removed / g.n], nb)
    assert abs(h_filt.sum() - 1.0) < 1e-12
    assert oracle.l1(h_filt, h_ex) < oracle.l1(h_plain, h_ex)


# ---- closed twins (lambda = -1/d) -------------------------------------------
def _remove_eigs(lam, spikes, tol=1e-9):
    """spec(H) minus `count` copies of each spike value."""
    keep = np.ones(lam.size, bool)
    for x, c in spikes:
        hit = np.nonzero(np.abs(lam - x) < tol)[0]
        assert hit.size >= c, (x, c, hit.size)
        keep[hit[:c]] = False
    return lam[keep]


def test_complete_graph_is_one_closed_class():
    # K_n: spectrum {1, -1/(n-1) x (n-1)}, every node a closed twin of every other
    for n in (2, 3, 7):
        g = oracle.build_csr(*sg.complete(n))
        cid, removed, spikes = oracle.closed_twin_classes(g)
        assert np.all(cid == 0) and removed == n - 1 and spikes == {n - 1: n - 1}
        lam, _ = oracle.exact_eigs(g)
        assert np.sum(np.abs(lam + 1.0 / (n - 1)) < 1e-9) == n - 1


def test_windmill_pairs_give_minus_half():
    g = oracle.build_csr(*sg.windmill(5))
    cid, removed, spikes = oracle.motif_classes(g)
    assert removed == 5 and spikes == [(-0.5, 5)]
    assert list(cid) == [0, 1, 1, 3, 3, 5, 5, 7, 7, 9, 9]
    # spectrum {-1/2 x (k+1), 1/2 x (k-1), 1}: k of the -1/2 are localized on
    # the twin pairs, one lives on the symmetric part and must stay
    lam, _ = oracle.exact_eigs(g)
    assert np.sum(np.abs(lam + 0.5) < 1e-9) == 6
    p = _p_matrix(cid)
    lam_r = np.linalg.eigvalsh(p.T @ oracle.dense_h(g) @ p)
    assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)
    assert np.sum(np.abs(lam_r + 0.5) < 1e-9) == 1


def test_star_leaves_are_open_not_closed_twins():
    g = oracle.build_csr(*sg.star(6))
    assert oracle.closed_twin_classes(g)[1] == 0
    assert oracle.motif_classes(g)[2] == [(0.0, 5)]


def test_open_and_closed_filter_projection_spectrum():
    src, dst, n = sg.chung_lu(300, 2.3, 4.0, 51)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 15, 52)
    src, dst, n = sg.add_triangle_twins(src, dst, n, 12, 53)
    g = oracle.build_csr(src, dst, n)
    cid, removed, spikes = oracle.motif_classes(g)
    sp = dict(spikes)
    assert sp[-0.5] >= 12 and sp[0.0] >= 15 and removed == sum(sp.values())
    lam, _ = oracle.exact_eigs(g)
    p = _p_matrix(cid)
    h = oracle.dense_h(g)
    # the class-constant subspace is invariant: P P^T commutes with H
    ppt = p @ p.T
    assert np.allclose(ppt @ h, h @ ppt, atol=1e-12)
    lam_r = np.linalg.eigvalsh(p.T @ h @ p)
    assert lam_r.size == g.n - removed
    assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


def test_closed_filter_on_graph_without_motifs_is_identity():
    g = oracle.build_csr(*sg.cycle(9))
    cid, removed, spikes = oracle.motif_classes(g)
    assert removed == 0 and spikes == [] and np.array_equal(cid, np.arange(9))


# ---- pendant twins (lambda = +-1/sqrt d: pendant 2-paths, the +-1/2 motif) -----
R2 = 1.0 / np.sqrt(2.0)


def test_path_p5_has_one_pendant_pair():
    # P5 = a2-a1-u-b1-b2: normalized adjacency eigenvalues cos(pi k / 4)
    g = oracle.build_csr(*sg.path(5))
    cid, removed, pairs = oracle.pendant_twin_classes(g)
    assert removed == 2 and pairs == {2: 1}
    lam, _ = oracle.exact_eigs(g)
    assert np.allclose(np.sort(lam), np.sort(np.cos(np.pi * np.arange(5) / 4)), atol=1e-12)
    _, _, spikes = oracle.motif_classes(g, pendant_twins=True)
    assert spikes == [(-R2, 1), (R2, 1)]


def test_spider_pendant_classes_and_projection():
    for legs in (2, 3, 5):
        g = oracle.build_csr(*sg.spider(legs))
        cid, removed, spikes = oracle.motif_classes(g, pendant_twins=True)
        assert removed == 2 * (legs - 1) and spikes == [(-R2, legs - 1), (R2, legs - 1)]
        lam, _ = oracle.exact_eigs(g)
        p = _p_matrix(cid)
        h = oracle.dense_h(g)
        assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
        lam_r = np.linalg.eigvalsh(p.T @ h @ p)
        assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


def test_tree_with_all_three_relations_disjoint():
    # a Barabasi-Albert tree (m = 1) plus twin leaves and triangles
    src, dst, n = sg.barabasi_albert(400, 1, 61)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 10, 62)
    src, dst, n = sg.add_triangle_twins(src, dst, n, 10, 63)
    g = oracle.build_csr(src, dst, n)
    cid, removed, spikes = oracle.motif_classes(g, pendant_twins=True)
    sp = dict(spikes)
    assert sp[R2] == sp[-R2] >= 1 and sp[-0.5] >= 10 and sp[0.0] >= 10
    lam, _ = oracle.exact_eigs(g)
    p = _p_matrix(cid)
    h = oracle.dense_h(g)
    assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
    lam_r = np.linalg.eigvalsh(p.T @ h @ p)
    assert lam_r.size == g.n - removed
    assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


def test_pendant_twins_of_degree_four_give_plus_minus_half():
    # Fig. 3's second +-1/2 example: nodes 0 and 1 share the neighbours 2, 3, 4
    # and each carries one leaf (5 on 0, 6 on 1); the shared nodes hang on a
    # small cycle so nothing else is symmetric
    src = [0, 0, 0, 1, 1, 1, 0, 1, 2, 3, 4, 7, 8]
    dst = [2, 3, 4, 2, 3, 4, 5, 6, 7, 8, 9, 8, 9]
    g = oracle.build_csr(np.array(src), np.array(dst), 10)
    cid, removed, pairs = oracle.pendant_twin_classes(g)
    assert removed == 2 and pairs == {4: 1}
    assert cid[1] == 0 and cid[6] == 5
    cid, removed, spikes = oracle.motif_classes(g, pendant_twins=True)
    assert (-0.5, 1) in spikes and (0.5, 1) in spikes
    lam, _ = oracle.exact_eigs(g)
    p = _p_matrix(cid)
    h = oracle.dense_h(g)
    assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
    lam_r = np.linalg.eigvalsh(p.T @ h @ p)
    assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


def test_random_graph_with_pendant_twins_of_mixed_degree():
    src, dst, n = sg.chung_lu(300, 2.4, 6.0, 81)
    for k, seed in ((1, 82), (2, 83), (3, 84)):
        src, dst, n = sg.add_pendant_twins(src, dst, n, 4, k, seed)
    g = oracle.build_csr(src, dst, n)
    _, _, pairs = oracle.pendant_twin_classes(g)
    # later groups may take an earlier group's leaf as a common neighbour and
    # so break that pair; most survive
    assert all(pairs.get(d, 0) >= 2 for d in (2, 3, 4))
    cid, removed, spikes = oracle.motif_classes(g, pendant_twins=True)
    lam, _ = oracle.exact_eigs(g)
    p = _p_matrix(cid)
    h = oracle.dense_h(g)
    assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
    lam_r = np.linalg.eigvalsh(p.T @ h @ p)
    assert lam_r.size == g.n - removed
    assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


# ---- parallel paths between two hosts (lambda = +-1/2) -------------------------
def test_theta_graph_parallel_paths():
    # theta graph: hosts 0 and 1 joined by k paths 0 - a - b - 1 (k = 2 is the
    # 6-cycle: no host of degree >= 3, nothing is filtered)
    src, dst = [0, 2, 3, 0, 4, 5], [2, 3, 1, 4, 5, 1]
    assert oracle.parallel_path_classes(oracle.build_csr(np.array(src), np.array(dst), 6))[1] == 0
    for k in (3, 5):
        src, dst = [], []
        for t in range(k):
            a, b = 2 + 2 * t, 3 + 2 * t
            src += [0, a, b]
            dst += [a, b, 1]
        g = oracle.build_csr(np.array(src), np.array(dst), 2 + 2 * k)
        cid, removed, pairs = oracle.parallel_path_classes(g)
        assert removed == 2 * (k - 1) and pairs == k - 1
        cid, removed, spikes = oracle.motif_classes(g, parallel_paths=True)
        lam, _ = oracle.exact_eigs(g)
        p = _p_matrix(cid)
        h = oracle.dense_h(g)
        assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
        lam_r = np.linalg.eigvalsh(p.T @ h @ p)
        assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


def test_all_motifs_together():
    src, dst, n = sg.chung_lu(400, 2.4, 6.0, 91)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 8, 92)
    src, dst, n = sg.add_triangle_twins(src, dst, n, 8, 93)
    src, dst, n = sg.add_pendant_twins(src, dst, n, 4, 3, 94)
    src, dst, n = sg.add_parallel_paths(src, dst, n, 4, 3, 95)
    g = oracle.build_csr(src, dst, n)
    _, _, pairs = oracle.parallel_path_classes(g)
    assert pairs >= 8
    cid, removed, spikes = oracle.motif_classes(g, pendant_twins=True, parallel_paths=True)
    lam, _ = oracle.exact_eigs(g)
    p = _p_matrix(cid)
    h = oracle.dense_h(g)
    assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
    lam_r = np.linalg.eigvalsh(p.T @ h @ p)
    assert lam_r.size == g.n - removed
    assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


@pytest.mark.parametrize("seed", [1, 2])
def test_motif_filters_on_watts_strogatz_and_ba_tree(seed):
    """The synthetic models of the paper's small-world and BA examples (§5.3):
    Watts-Strogatz with twin leaves and triangle twins, and the BA tree (m = 1),
    where pendant twins abound.  All relations together keep the projection
    exact: P P^T commutes with H, spec(P^T H P) is spec(H) without the spikes."""
    for src, dst, n in (sg.add_triangle_twins(*sg.add_twin_leaves(*sg.watts_strogatz(300, 2, 0.3, seed), 10, seed),
                                              10, seed + 1),
                        sg.barabasi_albert(300, 1, seed)):
        g = oracle.build_csr(src, dst, n)
        cid, removed, spikes = oracle.motif_classes(g, pendant_twins=True, parallel_paths=True)
        assert removed > 0
        lam, _ = oracle.exact_eigs(g)
        p = _p_matrix(cid)
        h = oracle.dense_h(g)
        assert np.allclose(p @ p.T @ h, h @ p @ p.T, atol=1e-12)
        lam_r = np.linalg.eigvalsh(p.T @ h @ p)
        assert lam_r.size == g.n - removed
        assert np.allclose(np.sort(lam_r), np.sort(_remove_eigs(lam, spikes)), atol=1e-9)


def test_watts_strogatz_generator():
    src, dst, n = sg.watts_strogatz(200, 3, 0.0, 5)  # the lattice itself
    deg = np.bincount(np.concatenate([src, dst]), minlength=n)
    assert np.all(deg == 6) and src.size == 600
    src, dst, n = sg.watts_strogatz(200, 3, 0.5, 5)  # rewiring keeps the edge count, no loops
    assert src.size == 600 and np.all(src != dst) and np.all(src < dst)
    assert len(set(zip(src.tolist(), dst.tolist()))) == 600
