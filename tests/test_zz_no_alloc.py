"""dos_moments_noalloc, the entry point for callers that cannot allocate
device memory (a framework allocator holding the memory, or no tolerance for
cudaMalloc's possible device synchronisation): it must give the same moments
as dos_moments while taking its scratch from the library's fixed static
device array.  Called through the C ABI; collected last so a failure here
does not hide the other tests' results."""
import ctypes

import numpy as np
import pytest
import torch

import synthgraphs as sg

pytestmark = pytest.mark.gpu

nd = pytest.importorskip("paper_1905_09758_gb300")

TOL_D = 1e-5  # the FP32 moment tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_09758_gb300.build import build

    build()


def _graph(src, dst, n):
    return nd.dos_build_csr(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)


def _noalloc(g, M, Nz, seed):
    d = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = nd.lib().dos_moments_noalloc(g.handle, M, Nz, ctypes.c_uint64(seed), ctypes.c_void_p(d.data_ptr()), stream)
    if st != nd.DOS_OK:
        raise nd.DosError(st, nd.lib().dos_last_error().decode())
    torch.cuda.synchronize()
    return d.cpu().numpy()


def test_noalloc_matches_dos_moments_on_consecutive_calls():
    ga = _graph(*sg.erdos_renyi(2000, 0.005, 1))
    s, d, n = sg.chung_lu(5000, 2.5, 10.0, 3)
    gb = _graph(*sg.add_twin_leaves(s, d, n, 100, 4))
    cases = [(ga, 100, 20, 1), (gb, 61, 37, 9)]
    refs = [nd.dos_moments(g, M, Nz, seed).cpu().numpy() for g, M, Nz, seed in cases]
    # two calls in a row on the same input, then the other input, then back:
    # the shared static scratch keeps stale contents between calls
    for idx in (0, 0, 1, 0, 1):
        g, M, Nz, seed = cases[idx]
        out = _noalloc(g, M, Nz, seed)
        assert np.all(np.isfinite(out))
        # same kernels, plan and fixed-order reduction as dos_moments: equal bits
        assert np.abs(out - refs[idx]).max() <= TOL_D
        assert np.array_equal(out, refs[idx]), np.abs(out - refs[idx]).max()


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    g = _graph(*sg.erdos_renyi(120000, 0.0001, 5))
    with pytest.raises(nd.DosError) as e:
        _noalloc(g, 50, 64, 1)
    assert e.value.status == nd.DOS_EINVAL
    assert "static scratch holds" in str(e.value)
