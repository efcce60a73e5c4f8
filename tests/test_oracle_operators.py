"""Oracle pins for KPM on the adjacency and Laplacian matrices (Eq. (5)
shift-and-scale): closed-form spectra, Gershgorin containment, identity
probes, and the Lanczos spectral interval (exact on K_n and stars, where a
probe's Krylov space is exhausted; containing the dense spectrum after as few
as 3 steps; much tighter than Gershgorin on graphs with hubs) (CPU only)."""
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


OPS = ["adjacency", "laplacian", "normalized_adjacency", "normalized_laplacian"]


def _spec_any(g, op):
    if op in ("adjacency", "laplacian"):
        return _spec(g, op)
    lam = np.linalg.eigvalsh(oracle.dense_h(g))
    return lam if op == "normalized_adjacency" else np.sort(1.0 - lam)


def test_lanczos_on_a_matrix_matches_the_dense_tridiagonal_spectrum():
    # K_n: a probe with sum z != 0 reaches both eigenspaces (the constant
    # vector and its complement), so Lanczos stops after two steps with the
    # Ritz values n - 1, -1 (A) or 0, n (D - A); a probe with sum z = 0 lies
    # in one eigenspace and stops after one step at -1 (A) or n (D - A)
    n = 8
    g = oracle.build_csr(*sg.complete(n))
    z = oracle.probes(5, g.old_id, 3)
    sums = z.sum(axis=0)
    assert np.any(sums != 0) and np.any(sums == 0)
    for op, want, rest in (("adjacency", [-1.0, n - 1.0], -1.0), ("laplacian", [0.0, float(n)], float(n))):
        a, b, st = oracle.lanczos(g, z, 6, x=oracle.operator_matrix(g, op))
        for j in range(3):
            if sums[j] == 0:
                assert st[j] == 1 and a[j, 0] == pytest.approx(rest, abs=1e-12)
                continue
            assert st[j] == 2
            theta = np.linalg.eigvalsh(np.diag(a[j, :2]) + np.diag(b[j, :1], 1) + np.diag(b[j, :1], -1))
            assert np.allclose(theta, want, atol=1e-12)


@pytest.mark.parametrize("bound", ["residual", "ritz"])
@pytest.mark.parametrize("pad", [0.0, 0.1])
def test_spectral_interval_closed_forms(pad, bound):
    n, k = 8, 6
    kn, star = oracle.build_csr(*sg.complete(n)), oracle.build_csr(*sg.star(k))
    r = np.sqrt(k)
    cases = [
        (kn, "adjacency", (-1.0, n - 1.0), (False, False)),
        (kn, "laplacian", (0.0, float(n)), (True, False)),
        (kn, "normalized_adjacency", (-1.0 / (n - 1), 1.0), (False, True)),
        (kn, "normalized_laplacian", (0.0, n / (n - 1.0)), (True, False)),
        (star, "adjacency", (-r, r), (False, False)),
        (star, "laplacian", (0.0, k + 1.0), (True, False)),
    ]
    for g, op, (lo, hi), (fix_lo, fix_hi) in cases:
        z = oracle.probes(9, g.old_id, 4)
        a, b = oracle.spectral_interval(g, op, z, 10, pad=pad, bound=bound)
        w = hi - lo
        want_lo = lo if fix_lo else lo - pad * w
        want_hi = hi if fix_hi else hi + pad * w
        g_lo, g_hi = oracle.gershgorin_interval(g, op) if op in ("adjacency", "laplacian") else (-1.0, 2.0)
        assert a == pytest.approx(max(want_lo, g_lo), abs=1e-10), (op, a)
        assert b == pytest.approx(min(want_hi, g_hi), abs=1e-10), (op, b)


HUBBY = {
    "ba": sg.barabasi_albert(400, 3, 4),
    "cl": sg.chung_lu(600, 2.5, 6.0, 5),
    "er": sg.erdos_renyi(300, 0.03, 3),
    "grid": sg.grid2d(10, 12),
    "cl_heavy": sg.chung_lu(2000, 2.1, 6.0, 11),
}


@pytest.mark.parametrize("op", OPS)
def test_residual_interval_contains_the_spectrum_after_few_steps(op):
    for src, dst, n in HUBBY.values():
        g = oracle.build_csr(src, dst, n)
        lam = _spec_any(g, op)
        for m_steps, nz in ((3, 4), (10, 4), (30, 4), (30, 16)):
            a, b = oracle.spectral_interval(g, op, oracle.probes(7, g.old_id, nz), m_steps, pad=0.0)
            assert a <= lam.min() + 1e-12 and b >= lam.max() - 1e-12, (op, m_steps, a, b, lam.min(), lam.max())


@pytest.mark.parametrize("op", OPS)
def test_ritz_interval_is_the_spectrum_once_converged(op):
    """After 30 steps on 4 probes the extreme Ritz values have converged: the
    Ritz interval contains the spectrum (pad 0) and exceeds it by < 1%."""
    for src, dst, n in HUBBY.values():
        g = oracle.build_csr(src, dst, n)
        lam = _spec_any(g, op)
        w = lam.max() - lam.min()
        a, b = oracle.spectral_interval(g, op, oracle.probes(7, g.old_id, 4), 30, pad=0.0, bound="ritz")
        assert a <= lam.min() + 1e-12 and b >= lam.max() - 1e-12, (op, a, b, lam.min(), lam.max())
        assert lam.min() - a <= 0.01 * w and b - lam.max() <= 0.01 * w


def test_ritz_interval_is_too_narrow_before_convergence():
    """The Ritz residual is a bound only near convergence: after 3 steps on 4
    probes it misses an end, which the plain residual norm covers."""
    g = oracle.build_csr(*HUBBY["cl"])
    lam = _spec(g, "adjacency")
    z = oracle.probes(7, g.old_id, 4)
    a, b = oracle.spectral_interval(g, "adjacency", z, 3, pad=0.0, bound="ritz")
    assert a > lam.min() or b < lam.max()
    a, b = oracle.spectral_interval(g, "adjacency", z, 3, pad=0.0)
    assert a < lam.min() and b > lam.max()


def test_spectral_interval_is_tight_on_hub_graphs():
    """Gershgorin's d_max is far above the spectral radius (~sqrt(d_max) for a
    hub) on a heavy-tailed graph; the Lanczos intervals stay within a small
    factor of the spectrum's width."""
    g = oracle.build_csr(*HUBBY["cl_heavy"])
    z = oracle.probes(3, g.old_id, 8)
    lam = _spec(g, "adjacency")
    w = lam.max() - lam.min()
    ga, gb = oracle.gershgorin_interval(g, "adjacency")
    a, b = oracle.spectral_interval(g, "adjacency", z, 30)
    assert b - a <= 2.0 * w and b - a <= 0.3 * (gb - ga)
    a, b = oracle.spectral_interval(g, "adjacency", z, 30, bound="ritz")
    assert b - a <= 1.03 * w and b - a <= 0.15 * (gb - ga)
    lam = _spec(g, "laplacian")
    ga, gb = oracle.gershgorin_interval(g, "laplacian")
    a, b = oracle.spectral_interval(g, "laplacian", z, 30, bound="ritz")
    assert b - a <= 1.03 * (lam.max() - lam.min()) and b - a <= 0.55 * (gb - ga)


def _p_matrix(class_id):
    ids = np.unique(class_id)
    p = np.zeros((class_id.size, ids.size))
    for k, c in enumerate(ids):
        mem = class_id == c
        p[mem, k] = 1.0 / np.sqrt(mem.sum())
    return p


def _without(lam, spikes, tol=1e-9):
    keep = np.ones(lam.size, bool)
    for x, c in spikes:
        hit = np.nonzero(np.abs(lam - x) < tol)[0]
        assert hit.size >= c, (x, c, hit.size)
        keep[hit[:c]] = False
    return lam[keep]


def test_motif_spikes_closed_forms():
    n, s = 7, 5
    kn, star = oracle.build_csr(*sg.complete(n)), oracle.build_csr(*sg.star(s))
    # K_n: closed twins of degree n - 1; spec A = {n - 1, -1 x (n - 1)}, spec L = {0, n x (n - 1)}
    assert oracle.motif_spikes(kn, "adjacency") == [(-1.0, n - 1)]
    assert oracle.motif_spikes(kn, "laplacian") == [(float(n), n - 1)]
    # star: open twins of degree 1; A: 0 x (s - 1), L: 1 x (s - 1)
    assert oracle.motif_spikes(star, "adjacency") == [(0.0, s - 1)]
    assert oracle.motif_spikes(star, "laplacian") == [(1.0, s - 1)]
    # P5 (pendant twins of degree 2): spec A = 2 cos(pi k / 6) holds +-1, spec L = 2 - 2 cos(pi k / 5)
    # holds (3 +- sqrt 5) / 2
    p5 = oracle.build_csr(*sg.path(5))
    sa = oracle.motif_spikes(p5, "adjacency", open_twins=False, closed_twins=False, pendant_twins=True)
    sl = oracle.motif_spikes(p5, "laplacian", open_twins=False, closed_twins=False, pendant_twins=True)
    assert sa == [(-1.0, 1), (1.0, 1)]
    assert np.allclose([x for x, _ in sl], [(3 - np.sqrt(5)) / 2, (3 + np.sqrt(5)) / 2], atol=1e-14)
    lam_l = np.sort(2 - 2 * np.cos(np.pi * np.arange(5) / 5))
    assert np.allclose(np.sort(_spec(p5, "laplacian")), lam_l, atol=1e-12)


@pytest.mark.parametrize("op", ["adjacency", "laplacian", "normalized_adjacency", "normalized_laplacian"])
def test_motif_spikes_complete_the_projected_spectrum(op):
    """All four motifs at once: the class-mean projection commutes with X
    and spec(X) = spec(P^T X P) plus the spikes, for every operator."""
    src, dst, n = sg.chung_lu(400, 2.4, 6.0, 91)
    src, dst, n = sg.add_twin_leaves(src, dst, n, 8, 92)
    src, dst, n = sg.add_triangle_twins(src, dst, n, 8, 93)
    src, dst, n = sg.add_pendant_twins(src, dst, n, 4, 3, 94)
    src, dst, n = sg.add_parallel_paths(src, dst, n, 4, 3, 95)
    g = oracle.build_csr(src, dst, n)
    cid, removed, _ = oracle.motif_classes(g, pendant_twins=True, parallel_paths=True)
    spikes = oracle.motif_spikes(g, op, pendant_twins=True, parallel_paths=True)
    assert sum(c for _, c in spikes) == removed
    if op in ("adjacency", "laplacian"):
        x = oracle.operator_matrix(g, op).toarray()
    else:
        x = oracle.dense_h(g)
        if op == "normalized_laplacian":
            x = np.eye(g.n) - x
    p = _p_matrix(cid)
    assert np.allclose(p @ p.T @ x, x @ p @ p.T, atol=1e-12)
    lam = np.linalg.eigvalsh(x)
    lam_r = np.linalg.eigvalsh(p.T @ x @ p)
    assert np.allclose(np.sort(lam_r), np.sort(_without(lam, spikes)), atol=1e-8)
