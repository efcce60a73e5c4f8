"""KPM on the adjacency and Laplacian matrices (Eq. (5) shift and scale) on
the GPU against the FP64 oracle on the same probes; the normalised Laplacian
and the normalised adjacency as special cases; Lanczos on A and D - A and the
spectral interval from its Ritz values."""
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


# steps before the FP32 and FP64 runs part ways: on the hub graph Lanczos
# captures the hub's eigenvector within a few steps, orthogonality is lost at
# once and later coefficients depend on the rounding (both runs stay valid
# Lanczos runs on nearby problems; their moments agree, see below)
COEF_STEPS = {"er2000": 10, "ba": 10, "hub": 3}


@pytest.mark.parametrize("name", ["er2000", "ba", "hub"])
@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
@pytest.mark.parametrize("nz", [1, 5, 16])
def test_lanczos_op_coefficients_match_oracle(name, op, nz):
    """FP32 vectors against the FP64 oracle, relative to the operator's scale
    (max |alpha|, beta ~ ||X||): a few float32 roundings per step; alpha_0 =
    z^T X z / N sums integers, scaled by the float32 1 / ||z||, to ~1e-7."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m = COEF_STEPS[name]
    a, b, st = nd.dos_lanczos_op(g, op, m, nz, 19)
    z = oracle.probes(19, ref.old_id, nz)
    ar, br, sr = oracle.lanczos(ref, z, m, x=oracle.operator_matrix(ref, op))
    scale = max(np.abs(ar).max(), br.max())
    assert np.array_equal(st.cpu().numpy(), sr)
    assert np.abs(a.cpu().numpy() - ar).max() <= 1e-4 * scale
    assert np.abs(b.cpu().numpy() - br).max() <= 1e-4 * scale
    assert np.abs(a.cpu().numpy()[:, 0] - ar[:, 0]).max() <= 1e-6 * scale


@pytest.mark.parametrize("name", ["er2000", "ba", "hub"])
@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
def test_lanczos_op_rules_are_exact_against_kpm(name, op):
    """Gauss exactness on X~ = (X - c) / r: the rules of the mapped
    tridiagonal (alpha - c) / r, beta / r reproduce the oracle's KPM moments of
    the same probes up to degree 2M - 1, even where the coefficients
    themselves have parted ways with the FP64 run."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m, nz = 20, 16
    iv = oracle.gershgorin_interval(ref, op)
    c, r = 0.5 * (iv[0] + iv[1]), 0.5 * (iv[1] - iv[0])
    a, b, st = nd.dos_lanczos_op(g, op, m, nz, 23)
    d = nd.dos_gql_moments(((a - c) / r).contiguous(), (b / r).contiguous(), st, 2 * m).cpu().numpy()
    d_ref = oracle.kpm_operator(ref, oracle.probes(23, ref.old_id, nz), 2 * m, op, iv)
    assert np.all(np.abs(d - d_ref) <= _tol(2 * m))


@pytest.mark.parametrize("bound", ["residual", "ritz"])
def test_ritz_bounds_kernel_on_oracle_coefficients(bound):
    """The FP64 bound stage (bisection for the extreme Ritz values, backward
    recurrence for |s_M|) on the oracle's own coefficients.  After 40 steps
    the extreme Ritz value has ghost copies (lost orthogonality): its
    eigenvector within the cluster, hence beta_M |s_M|, is ill-conditioned
    and two eigensolvers agree on it to ~1e-8 of the scale only."""
    src, dst, n = GRAPHS["hub"]
    ref = oracle.build_csr(src, dst, n)
    for op in ("adjacency", "laplacian"):
        ar, br, sr = oracle.lanczos(ref, oracle.probes(3, ref.old_id, 6), 40, x=oracle.operator_matrix(ref, op))
        want = oracle.ritz_bounds(ar, br, sr, bound)
        got = nd.dos_ritz_bounds(torch.from_numpy(ar).cuda(), torch.from_numpy(br).cuda(),
                                 torch.from_numpy(sr.astype(np.int32)).cuda(), bound).cpu().numpy()
        scale = max(np.abs(ar).max(), br.max())
        assert np.abs(got - want).max() <= (1e-12 if bound == "residual" else 2e-8) * scale


def test_lanczos_op_h_is_dos_lanczos():
    g = _graph(*GRAPHS["ba"])
    a0, b0, s0 = nd.dos_lanczos(g, 12, 8, 4)
    a1, b1, s1 = nd.dos_lanczos_op(g, "normalized_adjacency", 12, 8, 4)
    assert torch.equal(a0, a1) and torch.equal(b0, b1) and torch.equal(s0, s1)


def test_lanczos_op_stops_on_complete_graph():
    """K_n: a probe with sum z != 0 spans two eigenspaces (2 steps), one with
    sum z = 0 one (1 step); the interval is then exact."""
    n = 40
    src, dst, _ = sg.complete(n)
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    z = oracle.probes(2, ref.old_id, 32)
    for op, spec in (("adjacency", (-1.0, n - 1.0)), ("laplacian", (0.0, float(n)))):
        _, _, st = nd.dos_lanczos_op(g, op, 6, 32, 2)
        _, _, sr = oracle.lanczos(ref, z, 6, x=oracle.operator_matrix(ref, op))
        assert np.array_equal(st.cpu().numpy(), sr) and set(sr.tolist()) == {1, 2}
        for bound in ("residual", "ritz"):
            lo, hi = nd.dos_spectral_interval(g, op, 6, 32, 2, bound=bound, pad=0.0)
            assert abs(lo - spec[0]) <= 1e-5 * n and abs(hi - spec[1]) <= 1e-5 * n


_SPECTRA = {}


def _spectrum(name, op):
    if (name, op) not in _SPECTRA:
        ref = oracle.build_csr(*GRAPHS[name])
        if op in ("adjacency", "laplacian"):
            lam = np.linalg.eigvalsh(oracle.operator_matrix(ref, op).toarray())
        else:
            lam = np.linalg.eigvalsh(oracle.dense_h(ref))
            lam = lam if op == "normalized_adjacency" else 1.0 - lam
        _SPECTRA[(name, op)] = (lam.min(), lam.max())
    return _SPECTRA[(name, op)]


@pytest.mark.parametrize("name", ["er2000", "ba", "hub"])
@pytest.mark.parametrize("op", ["adjacency", "laplacian", "normalized_adjacency", "normalized_laplacian"])
@pytest.mark.parametrize("bound", ["residual", "ritz"])
def test_spectral_interval_holds_the_spectrum(name, op, bound):
    """Both bounds hold the dense spectrum; the Ritz interval (converged
    extreme Ritz values) matches the oracle's to 1e-3 of its width; the
    residual interval depends on beta_M, which FP32 and FP64 runs reach by
    different roundings after orthogonality is lost, so it is checked for
    containment and for staying inside Gershgorin only."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    m, nz = 30, 8
    lo, hi = nd.dos_spectral_interval(g, op, m, nz, 13, bound=bound, pad=0.01)
    lam_lo, lam_hi = _spectrum(name, op)
    assert lo <= lam_lo and hi >= lam_hi
    if op in ("adjacency", "laplacian"):
        ga, gb = oracle.gershgorin_interval(ref, op)
        assert ga <= lo and hi <= gb
    if bound == "ritz":
        rlo, rhi = oracle.spectral_interval(ref, op, oracle.probes(13, ref.old_id, nz), m, pad=0.01, bound=bound)
        w = rhi - rlo
        assert abs(lo - rlo) <= 1e-3 * w and abs(hi - rhi) <= 1e-3 * w


@pytest.mark.parametrize("op", ["adjacency", "laplacian"])
def test_moments_on_the_lanczos_interval(op):
    """KPM on the hub graph with the Ritz interval: parity with the oracle on
    the same interval, and far finer resolution than Gershgorin's."""
    src, dst, n = GRAPHS["hub"]
    ref = oracle.build_csr(src, dst, n)
    g = _graph(src, dst, n)
    iv = nd.dos_spectral_interval(g, op, 40, 8, 5, bound="ritz")
    ga, gb = oracle.gershgorin_interval(ref, op)
    assert iv[1] - iv[0] <= 0.6 * (gb - ga)
    m, nz = 60, 24
    d, iv2 = nd.dos_moments_op(g, op, m, nz, 31, interval=iv)
    assert iv2 == iv
    d_ref = oracle.kpm_operator(ref, oracle.probes(31, ref.old_id, nz), m, op, iv)
    assert np.all(np.abs(d.cpu().numpy() - d_ref) <= _tol(m))


def test_spectral_interval_errors():
    g = _graph(*GRAPHS["er2000"])
    with pytest.raises(ValueError):
        nd.dos_spectral_interval(g, "nope")
    with pytest.raises(ValueError):
        nd.dos_spectral_interval(g, "adjacency", bound="nope")
    with pytest.raises(nd.DosError) as e:
        nd.dos_spectral_interval(g, "adjacency", pad=-1.0)
    assert e.value.status == nd.DOS_EINVAL
    with pytest.raises(nd.DosError) as e:
        nd.dos_lanczos_op(g, "normalized_laplacian", 5, 4, 1)
    assert e.value.status == nd.DOS_EINVAL
    iv = (nd._binding.C.c_double * 2)()
    assert nd.lib().dos_spectral_interval(g.handle, 1, 10, 4, 1, 5, 0.01, iv, None) == nd.DOS_EINVAL
