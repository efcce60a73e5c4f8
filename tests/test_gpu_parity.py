"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
identical seeded inputs.

Tolerances:
* CSR, degrees, 1/sqrt(d), old ids, twin classes: bit-exact.
* FP32 DOS moments: |d_gpu - d_oracle| <= 1e-5 absolute on the normalised
  moments (|d_m| <= d_0 = 1), identical probes.
* FP32 per-node (LDOS) moments C[k, m]: <= 1e-4 absolute for M <= 100.  Each
  step rounds every entry with relative error ~6e-8 and the Chebyshev
  recurrence carries an error made at step s into step m with a factor
  |U_{m-s}| <= m - s + 1, so per-entry errors accumulate like a random walk,
  ~ eps * m^1.5 / sqrt(3) ~ 3.5e-5 at m = 100 before the 1/Nz average; the
  bound keeps a margin for the maximum over N * M entries.
* Density from the same moments: 1e-12 (FP64 on both sides).
"""
import numpy as np
import pytest
import torch

import oracle
import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")

TOL_D = 1e-5
TOL_C = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()
    yield
    nd.dos_set_plan(0, 0)


def _gpu_graph(src, dst, n, host=False):
    s = torch.from_numpy(np.ascontiguousarray(src, np.int64))
    d = torch.from_numpy(np.ascontiguousarray(dst, np.int64))
    if not host:
        s, d = s.cuda(), d.cuda()
    return nd.dos_build_csr(s, d, n)


def _graphs():
    yield "er2000", sg.erdos_renyi(2000, 0.005, 1)
    s, d, n = sg.chung_lu(6000, 2.5, 12.0, 7)
    yield "cl_twins", sg.add_twin_leaves(s, d, n, 300, 8)
    # a hub of degree 3000 exercises the CTA-per-row path
    s, d, n = sg.erdos_renyi(4000, 0.003, 2)
    hub = np.zeros(3000, np.int64)
    leaves = 1 + np.arange(3000, dtype=np.int64)
    yield "hub", (np.concatenate([s, hub, [5, 5, 9]]), np.concatenate([d, leaves, [5, 9, 5]]), n)
    yield "ba", sg.barabasi_albert(3000, 4, 3)


GRAPHS = dict(_graphs())


@pytest.mark.parametrize("name", list(GRAPHS))
def test_csr_bit_exact(name):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    info = g.info()
    assert (info["n"], info["nnz"], info["n_isolated"], info["n_original"]) == (ref.n, ref.nnz, ref.n_isolated, n)
    ex = {k: v.cpu().numpy() for k, v in nd.dos_graph_export(g).items()}
    assert np.array_equal(ex["row_ptr"], ref.row_ptr)
    assert np.array_equal(ex["col"], ref.col)
    assert np.array_equal(ex["deg"], ref.deg)
    assert np.array_equal(ex["inv_sqrt_deg"], ref.s64)
    assert np.array_equal(ex["inv_sqrt_deg32"], ref.s32)
    assert np.array_equal(ex["old_id"], ref.old_id)


def test_csr_from_host_buffers_and_edge_cases():
    src = np.array([0, 1, 1, 3, 3, 5, 2, 0, 6])
    dst = np.array([1, 0, 1, 5, 5, 3, 2, 6, 0])
    ref = oracle.build_csr(src, dst, 9)
    g = _gpu_graph(src, dst, 9, host=True)
    ex = nd.dos_graph_export(g)
    assert np.array_equal(ex["col"].cpu().numpy(), ref.col)
    assert g.info()["n_isolated"] == ref.n_isolated == 4  # nodes 2 (self-loop only), 4, 7, 8
    # no edges at all
    g0 = _gpu_graph(np.zeros(0, np.int64), np.zeros(0, np.int64), 7)
    assert g0.info() == {"n": 0, "nnz": 0, "n_isolated": 7, "n_original": 7}
    with pytest.raises(nd.DosError):
        nd.dos_moments(g0, 10, 4, 1)
    # only self-loops
    g1 = _gpu_graph(np.array([3, 3]), np.array([3, 3]), 4)
    assert g1.info()["nnz"] == 0


@pytest.mark.parametrize("name", ["cl_twins", "hub"])
def test_csr_from_pinned_host_buffers(name):
    """Page-locked host edge lists are read in place (no device copy): the CSR
    is still bit-exact, also from a slice that starts inside the buffer."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    s = torch.from_numpy(np.concatenate([[7], src]).astype(np.int64)).pin_memory()
    d = torch.from_numpy(np.concatenate([[7], dst]).astype(np.int64)).pin_memory()
    g = nd.dos_build_csr(s[1:], d[1:], n)
    ex = nd.dos_graph_export(g)
    assert np.array_equal(ex["row_ptr"].cpu().numpy(), ref.row_ptr)
    assert np.array_equal(ex["col"].cpu().numpy(), ref.col)
    assert np.array_equal(ex["old_id"].cpu().numpy(), ref.old_id)


def test_invalid_ids_are_rejected():
    with pytest.raises(nd.DosError) as e:
        _gpu_graph(np.array([0, 7]), np.array([1, 2]), 5)
    assert e.value.status == nd.DOS_EINVAL
    with pytest.raises(nd.DosError):
        _gpu_graph(np.array([-1]), np.array([1]), 5)


def _dos_ref(ref, seed, nz, m, filt=None):
    z = oracle.probes(seed, ref.old_id, nz)
    r = ref.n
    if filt is not None:
        cid, removed = filt
        z = oracle.project_probes(z, cid)
        r = ref.n - removed
    return oracle.kpm_doubled(ref, z, m) / (r * nz)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("m,nz", [(100, 20), (31, 37), (2, 1), (1, 5)])
def test_dos_moments_fp32(name, m, nz):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    d = nd.dos_moments(g, m, nz, 11).cpu().numpy()
    d_ref = _dos_ref(ref, 11, nz, m)
    assert abs(d[0] - 1.0) < 1e-12
    assert np.abs(d - d_ref).max() <= TOL_D


PLANS = [(t, c) for t in (4, 8, 16, 32, 64) for c in (0, 1)]


@pytest.mark.parametrize("t,p", PLANS)
def test_every_kernel_variant_fp32(t, p):
    src, dst, n = GRAPHS["hub"]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    nd.dos_set_plan(t, p)
    try:
        plan = nd.dos_get_plan(g, 70)
        assert plan["tile_width"] == t and (p == 0 or plan["ctas_per_sm"] <= p)
        d = nd.dos_moments(g, 24, 70, 5).cpu().numpy()
        c, dl = nd.ldos_moments(g, 12, 70, 5)
    finally:
        nd.dos_set_plan(0, 0)
    assert np.abs(d - _dos_ref(ref, 5, 70, 24)).max() <= TOL_D
    z = oracle.probes(5, ref.old_id, 70)
    mu, cref = oracle.kpm_direct(ref, z, 12, ldos=True)
    assert np.abs(c.cpu().numpy().T - cref).max() <= TOL_C
    assert np.abs(dl.cpu().numpy() - mu / (ref.n * 70)).max() <= TOL_D


@pytest.mark.parametrize("name", ["er2000", "cl_twins", "hub"])
def test_ldos_fp32(name):
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    m, nz = 100, 20
    c, dl = nd.ldos_moments(g, m, nz, 3)
    z = oracle.probes(3, ref.old_id, nz)
    mu, cref = oracle.kpm_direct(ref, z, m, ldos=True)
    c = c.cpu().numpy()
    assert c.shape == (m, ref.n)
    assert np.all(c[0] == 1.0)
    assert np.abs(c.T - cref).max() <= TOL_C
    assert np.abs(dl.cpu().numpy() - mu / (ref.n * nz)).max() <= TOL_D
    # the doubled DOS path and the direct LDOS path estimate the same moments
    d = nd.dos_moments(g, m, nz, 3).cpu().numpy()
    assert np.abs(d - dl.cpu().numpy()).max() <= 2 * TOL_D


def test_twin_filter_bit_exact_and_filtered_moments():
    src, dst, n = GRAPHS["cl_twins"]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    f = nd.dos_motif_filter(g)
    cid_ref, removed = oracle.twin_classes(ref)
    cid = nd.dos_filter_export(f).cpu().numpy()
    assert np.array_equal(cid, cid_ref)
    info = f.info()
    assert info["removed"] == removed and info["r"] == ref.n - removed
    assert info["n_classes"] == int(np.sum(np.bincount(cid_ref, minlength=ref.n) >= 2))
    d = nd.dos_moments(g, 60, 16, 9, filter=f).cpu().numpy()
    d_ref = _dos_ref(ref, 9, 16, 60, filt=(cid_ref, removed))
    assert np.abs(d - d_ref).max() <= TOL_D


def test_twin_filter_star_and_bipartite():
    for (s, d, n), expect in [(sg.star(50), 49), (sg.complete_bipartite(6, 9), 13)]:
        ref = oracle.build_csr(s, d, n)
        g = _gpu_graph(s, d, n)
        f = nd.dos_motif_filter(g)
        assert f.info()["removed"] == expect
        assert np.array_equal(nd.dos_filter_export(f).cpu().numpy(), oracle.twin_classes(ref)[0])


@pytest.mark.parametrize("kernel", ["jackson", "none"])
@pytest.mark.parametrize("m,b", [(100, 200), (7, 5), (1, 3), (500, 50)])
def test_density_matches_oracle(kernel, m, b):
    rng = np.random.default_rng(m * 1000 + b)
    d = rng.uniform(-1, 1, m)
    d[0] = 1.0
    h = nd.dos_density(torch.from_numpy(d).cuda(), b, kernel=kernel).cpu().numpy()
    assert np.abs(h - oracle.histogram(d, b, kernel=kernel)).max() <= 1e-12


def test_density_spikes_and_scale():
    d = np.zeros(10)
    d[0] = 1.0
    spikes = [(0.0, 0.25), (-1.0, 0.1), (0.33, 0.05)]
    h = nd.dos_density_raw(torch.from_numpy(d).cuda(), 4, scale=0.6, spikes=spikes).cpu().numpy()
    ref = 0.6 * oracle.histogram(d, 4) + oracle.point_mass_histogram([s[0] for s in spikes], [s[1] for s in spikes], 4)
    assert np.abs(h - ref).max() <= 1e-12


def test_filtered_density_assembly():
    src, dst, n = GRAPHS["cl_twins"]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    f = nd.dos_motif_filter(g)
    d = nd.dos_moments(g, 80, 16, 4, filter=f)
    h = nd.density_with_spikes(d, g, 50, filter=f).cpu().numpy()
    cid, removed = oracle.twin_classes(ref)
    n_total = ref.n + ref.n_isolated
    d_ref = _dos_ref(ref, 4, 16, 80, filt=(cid, removed))
    h_ref = (ref.n - removed) / n_total * oracle.histogram(d_ref, 50)
    h_ref += oracle.point_mass_histogram([0.0], [(removed + ref.n_isolated) / n_total], 50)
    assert abs(h.sum() - 1.0) < 1e-3
    assert np.abs(h - h_ref).max() <= 1e-5


def test_argument_errors():
    src, dst, n = GRAPHS["er2000"]
    g = _gpu_graph(src, dst, n)
    for bad in [dict(M=0, Nz=4), dict(M=4, Nz=0), dict(M=4, Nz=70000)]:
        with pytest.raises(nd.DosError) as e:
            nd.dos_moments(g, bad["M"], bad["Nz"], 1, d_out=torch.empty(max(1, bad["M"]), dtype=torch.float64,
                                                                           device="cuda"))
        assert e.value.status == nd.DOS_EINVAL
    with pytest.raises(nd.DosError):
        nd.dos_density(torch.zeros(4, dtype=torch.float64, device="cuda"), 0)
    # a filter from another graph is refused
    g2 = _gpu_graph(*sg.star(5))
    f2 = nd.dos_motif_filter(g2)
    with pytest.raises(nd.DosError):
        nd.dos_moments(g, 4, 4, 1, filter=f2)


def test_kernels_are_counted():
    src, dst, n = GRAPHS["er2000"]
    g = _gpu_graph(src, dst, n)
    before = nd.dos_launch_count()
    nd.dos_moments(g, 40, 8, 1)
    torch.cuda.synchronize()
    # init + 20 steps + reduction + moments
    assert nd.dos_launch_count() - before >= 23


def test_all_rows_heavy_complete_graph():
    # K_2100: every degree is 2099 >= the heavy threshold, so no light chunks;
    # spectrum {1, -1/(n-1) x (n-1)} gives the moments in closed form
    n = 2100
    src, dst, _ = sg.complete(n)
    g = _gpu_graph(src, dst, n)
    d = nd.dos_moments(g, 12, 8, 3).cpu().numpy()
    ref = oracle.build_csr(src, dst, n)
    assert np.abs(d - _dos_ref(ref, 3, 8, 12)).max() <= TOL_D
    lam = np.array([1.0] + [-1.0 / (n - 1)] * (n - 1))
    exact = np.array([np.mean(np.cos(m * np.arccos(lam))) for m in range(12)])
    # a stochastic estimate: error ~ 1/sqrt(N Nz) per moment
    assert np.abs(d - exact).max() < 0.05
    assert nd.dos_device_status() == 0


# ---- closed twins (lambda = -1/d) --------------------------------------------
def _closed_graphs():
    yield "windmill", sg.windmill(7)
    yield "k12", sg.complete(12)
    s, d, n = sg.chung_lu(6000, 2.5, 6.0, 17)
    s, d, n = sg.add_twin_leaves(s, d, n, 200, 18)
    yield "cl_both", sg.add_triangle_twins(s, d, n, 300, 19)
    yield "ba_tri", sg.add_triangle_twins(*sg.barabasi_albert(4000, 2, 20), 150, 21)


CLOSED = dict(_closed_graphs())


@pytest.mark.parametrize("name", list(CLOSED))
def test_closed_twin_filter_bit_exact_and_moments(name):
    src, dst, n = CLOSED[name]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    f = nd.dos_motif_filter_ex(g, ("open", "closed"))
    cid_ref, removed, spikes = oracle.motif_classes(ref)
    assert np.array_equal(nd.dos_filter_export(f).cpu().numpy(), cid_ref)
    assert f.info()["removed"] == removed and f.info()["r"] == ref.n - removed
    assert nd.dos_filter_spikes(f) == spikes
    # closed only
    fc = nd.dos_motif_filter_ex(g, ("closed",))
    cc, rc, sc = oracle.motif_classes(ref, open_twins=False)
    assert np.array_equal(nd.dos_filter_export(fc).cpu().numpy(), cc)
    assert fc.info()["removed"] == rc and nd.dos_filter_spikes(fc) == sc
    # filtered moments on the projected probes
    m, nz = 40, 24
    d = nd.dos_moments(g, m, nz, 13, filter=f).cpu().numpy()
    z = oracle.project_probes(oracle.probes(13, ref.old_id, nz), cid_ref)
    d_ref = oracle.kpm_doubled(ref, z, m) / ((ref.n - removed) * nz)
    assert np.abs(d - d_ref).max() <= TOL_D
    # the assembled density: (r/N) KPM(d^r) + a point mass per removed eigenvalue
    b = 40
    h = nd.density_with_spikes(torch.from_numpy(d).cuda(), g, b, filter=f).cpu().numpy()
    n_tot = ref.n + ref.n_isolated
    pts = [x for x, _ in spikes] + [0.0]
    wts = [c / n_tot for _, c in spikes] + [ref.n_isolated / n_tot]
    want = (ref.n - removed) / n_tot * oracle.histogram(d, b) + oracle.point_mass_histogram(pts, wts, b)
    assert np.abs(h - want).max() <= 1e-12


def test_motif_filter_ex_rejects_bad_sets():
    g = _gpu_graph(*sg.windmill(3))
    for bad in (0, 16, 31, 1 << 20):
        with pytest.raises(nd.DosError) as e:
            out = nd._binding.C.c_void_p()
            nd._binding._check(nd.lib().dos_motif_filter_ex(g.handle, bad, None, nd._binding.C.byref(out)))
        assert e.value.status == nd.DOS_EINVAL


# ---- pendant twins (lambda = +-1/sqrt d) ----------------------------------------
def _pendant_graphs():
    yield "p5", sg.path(5)
    yield "spider6", sg.spider(6)
    yield "fig3_deg4", (np.array([0, 0, 0, 1, 1, 1, 0, 1, 2, 3, 4, 7, 8]),
                        np.array([2, 3, 4, 2, 3, 4, 5, 6, 7, 8, 9, 8, 9]), 10)
    s, d, n = sg.chung_lu(5000, 2.4, 6.0, 81)
    for k, seed in ((1, 82), (2, 83), (3, 84), (7, 85)):
        s, d, n = sg.add_pendant_twins(s, d, n, 40, k, seed)
    yield "cl_pendant_mixed", (s, d, n)
    s, d, n = sg.barabasi_albert(5000, 1, 71)
    s, d, n = sg.add_twin_leaves(s, d, n, 100, 72)
    yield "ba_tree_all", sg.add_triangle_twins(s, d, n, 100, 73)
    yield "cl_sparse", sg.chung_lu(8000, 2.3, 2.5, 74)


PENDANT = dict(_pendant_graphs())


@pytest.mark.parametrize("name", list(PENDANT))
def test_pendant_twin_filter_bit_exact_and_moments(name):
    src, dst, n = PENDANT[name]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    f = nd.dos_motif_filter_ex(g, ("open", "closed", "pendant"))
    cid_ref, removed, spikes = oracle.motif_classes(ref, pendant_twins=True)
    assert np.array_equal(nd.dos_filter_export(f).cpu().numpy(), cid_ref)
    assert f.info()["removed"] == removed
    assert nd.dos_filter_spikes(f) == spikes
    m, nz = 30, 16
    d = nd.dos_moments(g, m, nz, 21, filter=f).cpu().numpy()
    z = oracle.project_probes(oracle.probes(21, ref.old_id, nz), cid_ref)
    d_ref = oracle.kpm_doubled(ref, z, m) / ((ref.n - removed) * nz)
    assert np.abs(d - d_ref).max() <= TOL_D
    b = 60
    h = nd.density_with_spikes(torch.from_numpy(d).cuda(), g, b, filter=f).cpu().numpy()
    n_tot = ref.n + ref.n_isolated
    pts = [x for x, _ in spikes] + [0.0]
    wts = [c / n_tot for _, c in spikes] + [ref.n_isolated / n_tot]
    want = (ref.n - removed) / n_tot * oracle.histogram(d, b) + oracle.point_mass_histogram(pts, wts, b)
    assert np.abs(h - want).max() <= 1e-12


# ---- parallel paths between two hosts (lambda = +-1/2), all motifs together ----
def _theta(k):
    src, dst = [], []
    for t in range(k):
        a, b = 2 + 2 * t, 3 + 2 * t
        src += [0, a, b]
        dst += [a, b, 1]
    return np.array(src, np.int64), np.array(dst, np.int64), 2 + 2 * k


def _all_motifs():
    s, d, n = sg.chung_lu(6000, 2.4, 6.0, 91)
    s, d, n = sg.add_twin_leaves(s, d, n, 100, 92)
    s, d, n = sg.add_triangle_twins(s, d, n, 100, 93)
    s, d, n = sg.add_pendant_twins(s, d, n, 40, 3, 94)
    return sg.add_parallel_paths(s, d, n, 40, 3, 95)


ALL = {"theta5": _theta(5), "cycle6": sg.cycle(6), "all_motifs": _all_motifs()}


@pytest.mark.parametrize("name", list(ALL))
def test_all_motif_filters_bit_exact_and_moments(name):
    src, dst, n = ALL[name]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    f = nd.dos_motif_filter_ex(g, ("open", "closed", "pendant", "parallel"))
    cid_ref, removed, spikes = oracle.motif_classes(ref, pendant_twins=True, parallel_paths=True)
    assert np.array_equal(nd.dos_filter_export(f).cpu().numpy(), cid_ref)
    assert f.info()["removed"] == removed
    assert nd.dos_filter_spikes(f) == [(float(x), c) for x, c in spikes]
    m, nz = 30, 16
    d = nd.dos_moments(g, m, nz, 27, filter=f).cpu().numpy()
    z = oracle.project_probes(oracle.probes(27, ref.old_id, nz), cid_ref)
    d_ref = oracle.kpm_doubled(ref, z, m) / ((ref.n - removed) * nz)
    assert np.abs(d - d_ref).max() <= TOL_D


@pytest.mark.parametrize("t,nz", [(16, 70), (64, 70), (64, 50)])
def test_ldos_layouts_equal_and_reproducible(t, nz):
    """ldos_moments_ex: the node-major N x M matrix is the transpose of the
    moment-major one bit for bit, repeated runs agree bit for bit (several
    probe tiles are summed in a fixed order), and both match the oracle."""
    src, dst, n = GRAPHS["hub"]
    ref = oracle.build_csr(src, dst, n)
    g = _gpu_graph(src, dst, n)
    m, seed = 37, 8
    nd.dos_set_plan(t, 0)
    try:
        assert nd.dos_get_plan(g, nz)["tiles"] == -(-nz // t)
        c_mm, d_mm = nd.ldos_moments(g, m, nz, seed)
        c_mm2, _ = nd.ldos_moments(g, m, nz, seed)
        c_nm, d_nm = nd.ldos_moments(g, m, nz, seed, layout="node")
    finally:
        nd.dos_set_plan(0, 0)
    c_mm, c_mm2, c_nm = c_mm.cpu().numpy(), c_mm2.cpu().numpy(), c_nm.cpu().numpy()
    assert c_nm.shape == (ref.n, m)
    assert np.array_equal(c_mm, c_mm2)
    assert np.array_equal(c_nm, c_mm.T)
    assert np.array_equal(d_mm.cpu().numpy(), d_nm.cpu().numpy())
    z = oracle.probes(seed, ref.old_id, nz)
    _, cref = oracle.kpm_direct(ref, z, m, ldos=True)
    assert np.abs(c_nm - cref).max() <= TOL_C


@pytest.mark.parametrize("name", list(GRAPHS))
def test_class_row_order_matches_oracle(name):
    """DOS_ORDER_BY_CLASS only relabels the kernels' rows (degree classes kept
    apart, node numbering inside a class): the exported CSR, DOS and LDOS
    moments and the twin filter match the oracle as with the default order,
    and the filtered moments of the two orders agree."""
    src, dst, n = GRAPHS[name]
    ref = oracle.build_csr(src, dst, n)
    g = nd.dos_build_csr(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n, order="class")
    ex = {k: v.cpu().numpy() for k, v in nd.dos_graph_export(g).items()}
    assert np.array_equal(ex["row_ptr"], ref.row_ptr) and np.array_equal(ex["col"], ref.col)
    d = nd.dos_moments(g, 60, 20, 11).cpu().numpy()
    assert np.abs(d - _dos_ref(ref, 11, 20, 60)).max() <= TOL_D
    c, dl = nd.ldos_moments(g, 40, 20, 3)
    z = oracle.probes(3, ref.old_id, 20)
    mu, cref = oracle.kpm_direct(ref, z, 40, ldos=True)
    assert np.abs(c.cpu().numpy().T - cref).max() <= TOL_C
    assert np.abs(dl.cpu().numpy() - mu / (ref.n * 20)).max() <= TOL_D
    f = nd.dos_motif_filter(g)
    cid_ref, removed = oracle.twin_classes(ref)
    assert np.array_equal(nd.dos_filter_export(f).cpu().numpy(), cid_ref)
    g_deg = _gpu_graph(src, dst, n)
    d_cls = nd.dos_moments(g, 40, 16, 9, filter=f).cpu().numpy()
    d_deg = nd.dos_moments(g_deg, 40, 16, 9, filter=nd.dos_motif_filter(g_deg)).cpu().numpy()
    assert np.abs(d_cls - d_deg).max() <= 2 * TOL_D


def test_class_row_order_flag_checks():
    import ctypes

    s = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    t = torch.tensor([1, 2], dtype=torch.int64, device="cuda")
    out = ctypes.c_void_p()
    off = (ctypes.c_int64 * 2)(0, 3)
    st = nd.lib().dos_build_csr_batched(ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(t.data_ptr()), 2, off, 1,
                                        nd.DOS_ORDER_BY_CLASS, None, ctypes.byref(out))
    assert st == nd.DOS_EINVAL and not out.value
    st = nd.lib().dos_build_csr(ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(t.data_ptr()), 2, 3, 8, None,
                                ctypes.byref(out))
    assert st == nd.DOS_EINVAL and not out.value
    with pytest.raises(ValueError):
        nd.dos_build_csr(s, t, 3, order="bfs")
