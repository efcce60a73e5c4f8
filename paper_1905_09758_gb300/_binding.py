"""ctypes binding of libnetdos.so (include/netdos.h).

Argument marshalling only: every computation runs in the CUDA library.  Torch
is used for device memory and the current CUDA stream.  There is no fallback:
if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnetdos.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "netdos.h")

DOS_OK, DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA, DOS_ETIMEOUT, DOS_EOVERFLOW = range(6)
PREC = {"fp32": 0, "bf16": 1, "fp16": 2}
KERNEL = {"none": 0, "jackson": 1}
LAYOUT = {"moment": 0, "node": 1}
DOS_INPUT_HOST = 1
DOS_ORDER_BY_CLASS = 2
MOTIF = {"open": 1, "closed": 2, "pendant": 4, "parallel": 8}
OPERATOR = {"normalized_adjacency": 0, "adjacency": 1, "laplacian": 2, "normalized_laplacian": 3}

_STATUS_NAMES = {
    DOS_EINVAL: "DOS_EINVAL",
    DOS_ENOMEM: "DOS_ENOMEM",
    DOS_ECUDA: "DOS_ECUDA",
    DOS_ETIMEOUT: "DOS_ETIMEOUT",
    DOS_EOVERFLOW: "DOS_EOVERFLOW",
}


class DosError(RuntimeError):
    """A netdos call returned a status other than DOS_OK."""

    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp, _i64, _i32, _u32, _u64, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_uint32, C.c_uint64, C.c_double
_P64 = C.POINTER(C.c_int64)
_PI = C.POINTER(C.c_int)

_SIGNATURES = {
    "dos_version": ([], _i32),
    "dos_last_error": ([], C.c_char_p),
    "dos_build_csr": ([_vp, _vp, _i64, _i64, _u32, _vp, C.POINTER(_vp)], _i32),
    "dos_graph_info": ([_vp, _P64, _P64, _P64, _P64], _i32),
    "dos_graph_export": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "dos_graph_destroy": ([_vp], None),
    "dos_motif_filter": ([_vp, _vp, C.POINTER(_vp)], _i32),
    "dos_motif_filter_ex": ([_vp, _u32, _vp, C.POINTER(_vp)], _i32),
    "dos_filter_spikes": ([_vp, _vp, _i32, _PI], _i32),
    "dos_filter_info": ([_vp, _P64, _P64, _P64], _i32),
    "dos_filter_export": ([_vp, _vp, _vp], _i32),
    "dos_filter_destroy": ([_vp], None),
    "dos_moments": ([_vp, _vp, _i32, _i32, _u64, _i32, _vp, _vp], _i32),
    "ldos_moments": ([_vp, _i32, _i32, _u64, _i32, _vp, _vp, _vp], _i32),
    "ldos_moments_ex": ([_vp, _i32, _i32, _u64, _i32, _i32, _vp, _vp, _vp], _i32),
    "dos_moments_noalloc": ([_vp, _i32, _i32, _u64, _vp, _vp], _i32),
    "dos_density": ([_vp, _i32, _i32, _i32, _vp, _vp, _u32, _vp, _vp], _i32),
    "dos_density_weights": ([_vp, _vp, _u32, C.POINTER(C.c_double), _vp, _i32, _PI], _i32),
    "dos_density_raw": ([_vp, _i32, _i32, _i32, _dbl, _vp, _i32, _vp, _vp], _i32),
    "dos_device_status": ([_vp, C.POINTER(C.c_int)], _i32),
    "dos_launch_count": ([], _i64),
    "dos_profile_enable": ([_i32], _i32),
    "dos_profile_read": ([C.POINTER(C.c_double), _P64, _i32], _i32),
    "dos_set_plan": ([_i32, _i32], _i32),
    "dos_build_csr_batched": ([_vp, _vp, _i64, _vp, _i64, _u32, _vp, C.POINTER(_vp)], _i32),
    "dos_batch_info": ([_vp, _P64, _vp, _vp], _i32),
    "dos_moments_batched": ([_vp, _i32, _i32, _u64, _i32, _vp, _vp], _i32),
    "dos_autotune": ([_vp, _i32, _i32, _vp, _PI, _PI], _i32),
    "dos_get_plan": ([_vp, _i32, _i32, _PI, _PI, _PI, _PI], _i32),
    "dos_density_batched": ([_vp, _i32, _i64, _i32, _i32, _vp, _vp], _i32),
    "dos_mlp_create": ([_i32, _PI, _u64, C.POINTER(_vp)], _i32),
    "dos_mlp_destroy": ([_vp], None),
    "dos_mlp_param_count": ([_vp, _P64], _i32),
    "dos_mlp_get_params": ([_vp, _vp, _vp], _i32),
    "dos_mlp_set_params": ([_vp, _vp, _vp], _i32),
    "dos_test_fail_alloc": ([_i64], _i32),
    "dos_mlp_get_state": ([_vp, _vp, _vp, _vp, C.POINTER(_i64), _vp], _i32),
    "dos_mlp_set_state": ([_vp, _vp, _vp, _vp, _i64, _vp], _i32),
    "dos_mlp_forward": ([_vp, _vp, _i32, _vp, _vp], _i32),
    "dos_mlp_loss_grad": ([_vp, _vp, _vp, _i32, _vp, _vp, _vp], _i32),
    "dos_mlp_train_step": ([_vp, _vp, _vp, _vp, _i32, C.c_float, _vp, _vp], _i32),
    "dos_mlp_features": ([_vp, _i32, _vp, _i32, _i32, _vp, _i64, _vp, _vp], _i32),
    "dos_graph_stats": ([_vp, _i32, _vp, _vp], _i32),
    "dos_hist_normalize": ([_vp, _i32, _i64, _vp, _vp], _i32),
    "dos_hist_assemble": ([_vp, _i32, _i64, _dbl, _vp, _i32, _vp, _vp], _i32),
    "dos_lanczos": ([_vp, _i32, _i32, _u64, _vp, _vp, _vp, _vp], _i32),
    "dos_lanczos_op": ([_vp, _i32, _i32, _i32, _u64, _vp, _vp, _vp, _vp], _i32),
    "ldos_moments_op": ([_vp, _i32, _dbl, _dbl, _i32, _i32, _u64, _vp, _vp, _vp, _vp], _i32),
    "dos_fn_coeffs": ([_i32, _dbl, _dbl, _dbl, _i32, _vp, _vp], _i32),
    "dos_fn_trace": ([_vp, _vp, _vp, _i32, _vp, _vp], _i32),
    "dos_fn_diag": ([_vp, _i64, _i32, _vp, _vp, _vp], _i32),
    "dos_ritz_bounds": ([_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp], _i32),
    "dos_spectral_interval": ([_vp, _i32, _i32, _i32, _u64, _i32, _dbl, _vp, _vp], _i32),
    "dos_pdos_nd": ([_vp, _i32, _i32, _dbl, _vp, _P64, _vp], _i32),
    "dos_moments_op": ([_vp, _i32, _dbl, _dbl, _i32, _i32, _u64, _i32, _vp, _vp, _vp], _i32),
    "dos_gauss_rules": ([_vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp], _i32),
    "dos_gql_moments": ([_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp], _i32),
    "dos_gql_histogram": ([_vp, _vp, _i32, _i32, _i32, _vp, _vp], _i32),
}


def lib():
    """Load libnetdos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_1905_09758_gb300.build.build() "
                "(there is no non-CUDA implementation)"
            )
        handle = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(handle, name)
            f.argtypes = args
            f.restype = res
        _lib = handle
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/netdos.h."""
    txt = open(HEADER_PATH).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b((?:dos|ldos)_[a-z0-9_]+)\s*\(", txt)))


def _check(status: int):
    if status != DOS_OK:
        msg = lib().dos_last_error()
        raise DosError(status, msg.decode() if msg else "")


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _need_cuda(t: torch.Tensor, dtype, name: str, numel: int | None = None):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements")


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
class Graph:
    """Owned dos_graph_t handle."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        n, nnz, iso, orig = (C.c_int64() for _ in range(4))
        _check(lib().dos_graph_info(self._h, C.byref(n), C.byref(nnz), C.byref(iso), C.byref(orig)))
        return {"n": n.value, "nnz": nnz.value, "n_isolated": iso.value, "n_original": orig.value}

    @property
    def n(self) -> int:
        return self.info()["n"]

    def close(self):
        if self._h is not None and self._h.value:
            lib().dos_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Filter:
    """Owned dos_filter_t handle (keeps its graph alive)."""

    def __init__(self, handle: int, graph: Graph):
        self._h = C.c_void_p(handle)
        self.graph = graph

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        rem, ncl, r = (C.c_int64() for _ in range(3))
        _check(lib().dos_filter_info(self._h, C.byref(rem), C.byref(ncl), C.byref(r)))
        return {"removed": rem.value, "n_classes": ncl.value, "r": r.value}

    def close(self):
        if self._h is not None and self._h.value:
            lib().dos_filter_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Owned dos_mlp_t handle (density-reconstruction network)."""

    def __init__(self, handle: int, sizes):
        self._h = C.c_void_p(handle)
        self.sizes = [int(x) for x in sizes]

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().dos_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def dos_version() -> int:
    return lib().dos_version()


def dos_build_csr(src: torch.Tensor, dst: torch.Tensor, n_nodes: int, stream=None, order: str = "degree") -> Graph:
    """Edge list (int64 tensors, CUDA or host) -> Graph.  Host tensors are copied by the library.
    order "degree": the step kernels' rows by descending degree; "class": by
    degree class only, keeping the node numbering inside a class."""
    if order not in ("degree", "class"):
        raise ValueError("order must be 'degree' or 'class'")
    if src.dtype != torch.int64 or dst.dtype != torch.int64 or src.shape != dst.shape:
        raise ValueError("src and dst must be int64 tensors of equal shape")
    src, dst = src.contiguous(), dst.contiguous()
    if src.is_cuda != dst.is_cuda:
        raise ValueError("src and dst must be on the same device")
    flags = (0 if src.is_cuda else DOS_INPUT_HOST) | (DOS_ORDER_BY_CLASS if order == "class" else 0)
    out = C.c_void_p()
    _check(lib().dos_build_csr(_ptr(src), _ptr(dst), src.numel(), int(n_nodes), flags, _stream(stream),
                               C.byref(out)))
    return Graph(out.value)


def dos_build_csr_batched(src: torch.Tensor, dst: torch.Tensor, node_offset, stream=None) -> Graph:
    """A batch of graphs: graph g owns original ids [node_offset[g], node_offset[g+1])."""
    if src.dtype != torch.int64 or dst.dtype != torch.int64 or src.shape != dst.shape:
        raise ValueError("src and dst must be int64 tensors of equal shape")
    src, dst = src.contiguous(), dst.contiguous()
    flags = 0 if src.is_cuda else DOS_INPUT_HOST
    off = (C.c_int64 * len(node_offset))(*[int(x) for x in node_offset])
    out = C.c_void_p()
    _check(lib().dos_build_csr_batched(_ptr(src), _ptr(dst), src.numel(), off, len(node_offset) - 1, flags,
                                       _stream(stream), C.byref(out)))
    return Graph(out.value)


def dos_batch_info(g: Graph) -> dict:
    ng = C.c_int64()
    _check(lib().dos_batch_info(g.handle, C.byref(ng), None, None))
    gn = (C.c_int64 * max(1, ng.value))()
    gi = (C.c_int64 * max(1, ng.value))()
    _check(lib().dos_batch_info(g.handle, None, gn, gi))
    return {"n_graphs": ng.value, "graph_n": list(gn)[: ng.value], "graph_isolated": list(gi)[: ng.value]}


def dos_moments_batched(g: Graph, M: int, Nz: int, seed: int, prec: str = "fp32",
                        d_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per-graph DOS moments of a batch: float64 CUDA tensor (n_graphs, M)."""
    ng = dos_batch_info(g)["n_graphs"]
    if d_out is None:
        d_out = torch.empty((ng, M), dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _need_cuda(d_out, torch.float64, "d_out", ng * M)
    _check(lib().dos_moments_batched(g.handle, int(M), int(Nz), int(seed) & (2**64 - 1), PREC[prec], _ptr(d_out),
                                     _stream(stream)))
    return d_out


def dos_autotune(g: Graph, Nz: int, prec: str = "fp32", stream=None) -> dict:
    """Time candidate plans on this graph and keep the fastest; returns it."""
    t, c = C.c_int(), C.c_int()
    _check(lib().dos_autotune(g.handle, int(Nz), PREC[prec], _stream(stream), C.byref(t), C.byref(c)))
    return {"tile_width": t.value, "ctas_per_sm": c.value}


def dos_graph_info(g: Graph) -> dict:
    return g.info()


def dos_graph_export(g: Graph, stream=None) -> dict:
    """CSR arrays (compact ids) as CUDA tensors."""
    info = g.info()
    n, nnz = info["n"], info["nnz"]
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {
        "row_ptr": torch.empty(n + 1, dtype=torch.int64, device=dev),
        "col": torch.empty(nnz, dtype=torch.int32, device=dev),
        "deg": torch.empty(n, dtype=torch.int32, device=dev),
        "inv_sqrt_deg": torch.empty(n, dtype=torch.float64, device=dev),
        "inv_sqrt_deg32": torch.empty(n, dtype=torch.float32, device=dev),
        "old_id": torch.empty(n, dtype=torch.int32, device=dev),
    }
    _check(lib().dos_graph_export(g.handle, *(_ptr(out[k]) for k in
                                              ("row_ptr", "col", "deg", "inv_sqrt_deg", "inv_sqrt_deg32", "old_id")),
                                  _stream(stream)))
    return out


def dos_motif_filter(g: Graph, stream=None) -> Filter:
    """Open-twin (lambda = 0) classes of the graph."""
    out = C.c_void_p()
    _check(lib().dos_motif_filter(g.handle, _stream(stream), C.byref(out)))
    return Filter(out.value, g)


def dos_motif_filter_ex(g: Graph, motifs=("open", "closed"), stream=None) -> Filter:
    """Motif classes for a set of motifs: "open" twins (lambda = 0), "closed"
    twins (lambda = -1/d), "pendant" twins (lambda = +-1/sqrt d), "parallel"
    paths (lambda = +-1/2)."""
    mask = 0
    for m in motifs:
        mask |= MOTIF[m]
    out = C.c_void_p()
    _check(lib().dos_motif_filter_ex(g.handle, mask, _stream(stream), C.byref(out)))
    return Filter(out.value, g)


def dos_filter_spikes(f: Filter) -> list:
    """Removed eigenvalues as [(lambda, count)], ascending lambda."""
    n = C.c_int()
    _check(lib().dos_filter_spikes(f.handle, None, 0, C.byref(n)))
    buf = (C.c_double * max(1, 2 * n.value))()
    _check(lib().dos_filter_spikes(f.handle, buf, n.value, None))
    return [(buf[2 * k], int(buf[2 * k + 1])) for k in range(n.value)]


def dos_filter_info(f: Filter) -> dict:
    return f.info()


def dos_filter_export(f: Filter, stream=None) -> torch.Tensor:
    n = f.graph.n
    cid = torch.empty(n, dtype=torch.int32, device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib().dos_filter_export(f.handle, _ptr(cid), _stream(stream)))
    return cid


def dos_moments(g: Graph, M: int, Nz: int, seed: int, prec: str = "fp32", filter: Filter | None = None,
                d_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """DOS moments d_0..d_{M-1} (float64 CUDA tensor)."""
    if d_out is None:
        d_out = torch.empty(M, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _need_cuda(d_out, torch.float64, "d_out", M)
    _check(lib().dos_moments(g.handle, None if filter is None else filter.handle, int(M), int(Nz),
                             int(seed) & (2**64 - 1), PREC[prec], _ptr(d_out), _stream(stream)))
    return d_out


def dos_moments_noalloc(g: Graph, M: int, Nz: int, seed: int, d_out: torch.Tensor, stream=None) -> torch.Tensor:
    """dos_moments (FP32, no filter) without device allocation; d_out is caller-allocated."""
    _need_cuda(d_out, torch.float64, "d_out", M)
    _check(lib().dos_moments_noalloc(g.handle, int(M), int(Nz), int(seed) & (2**64 - 1), _ptr(d_out),
                                     _stream(stream)))
    return d_out


def ldos_moments(g: Graph, M: int, Nz: int, seed: int, prec: str = "fp32", C_out: torch.Tensor | None = None,
                 d_out: torch.Tensor | None = None, want_d: bool = True, layout: str = "moment", stream=None):
    """Per-node moments C and, if want_d, the DOS moments from the same
    recurrence.  layout "moment": C has shape (M, N), C[m, k] = moment m of
    compact node k; layout "node": shape (N, M), row k = node k's moments."""
    n = g.n
    dev = torch.device("cuda", torch.cuda.current_device())
    if layout not in LAYOUT:
        raise ValueError(f"layout must be one of {sorted(LAYOUT)}")
    if C_out is None:
        C_out = torch.empty((M, n) if layout == "moment" else (n, M), dtype=torch.float32, device=dev)
    _need_cuda(C_out, torch.float32, "C_out", M * n)
    if d_out is None and want_d:
        d_out = torch.empty(M, dtype=torch.float64, device=dev)
    if d_out is not None:
        _need_cuda(d_out, torch.float64, "d_out", M)
    _check(lib().ldos_moments_ex(g.handle, int(M), int(Nz), int(seed) & (2**64 - 1), PREC[prec], LAYOUT[layout],
                                 _ptr(C_out), _ptr(d_out), _stream(stream)))
    return C_out, d_out


DOS_DENSITY_COUNT_ISOLATED = 1


def dos_density(d: torch.Tensor, n_bins: int, kernel: str = "jackson", g: Graph | None = None,
                filter: Filter | None = None, count_isolated: bool = True, hist_out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Damped histogram over n_bins equal bins of [-1, 1] (float64 CUDA tensor).
    Without g and filter: the plain series of d.  With them: the whole graph's
    density (the library weights the series by r / N_total and adds the
    removed eigenvalues and, if count_isolated, the isolated nodes as point
    masses)."""
    _need_cuda(d, torch.float64, "d")
    if hist_out is None:
        hist_out = torch.empty(n_bins, dtype=torch.float64, device=d.device)
    _need_cuda(hist_out, torch.float64, "hist_out", n_bins)
    flags = DOS_DENSITY_COUNT_ISOLATED if count_isolated else 0
    _check(lib().dos_density(_ptr(d), d.numel(), int(n_bins), KERNEL[kernel], None if g is None else g.handle,
                             None if filter is None else filter.handle, flags, _ptr(hist_out), _stream(stream)))
    return hist_out


def dos_density_weights(g: Graph | None, filter: Filter | None = None, count_isolated: bool = True):
    """(scale, [(lambda, mass)]) that dos_density applies for (g, filter)."""
    flags = DOS_DENSITY_COUNT_ISOLATED if count_isolated else 0
    scale, n = C.c_double(), C.c_int()
    hg, hf = (None if g is None else g.handle), (None if filter is None else filter.handle)
    _check(lib().dos_density_weights(hg, hf, flags, C.byref(scale), None, 0, C.byref(n)))
    buf = (C.c_double * max(1, 2 * n.value))()
    _check(lib().dos_density_weights(hg, hf, flags, C.byref(scale), buf, n.value, C.byref(n)))
    return scale.value, [(buf[2 * k], buf[2 * k + 1]) for k in range(n.value)]


def dos_density_raw(d: torch.Tensor, n_bins: int, kernel: str = "jackson", scale: float = 1.0, spikes=(),
                    hist_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dos_density with an explicit series weight and point masses (lambda, mass)."""
    _need_cuda(d, torch.float64, "d")
    if hist_out is None:
        hist_out = torch.empty(n_bins, dtype=torch.float64, device=d.device)
    _need_cuda(hist_out, torch.float64, "hist_out", n_bins)
    sp = [float(x) for pair in spikes for x in pair]
    arr = (C.c_double * max(1, len(sp)))(*sp)
    _check(lib().dos_density_raw(_ptr(d), d.numel(), int(n_bins), KERNEL[kernel], float(scale),
                                 arr if sp else None, len(sp) // 2, _ptr(hist_out), _stream(stream)))
    return hist_out


def dos_device_status(stream=None) -> int:
    """Device error word (0 = no bounded wait gave up); raises DosError(DOS_ETIMEOUT) otherwise."""
    st = C.c_int()
    _check(lib().dos_device_status(_stream(stream), C.byref(st)))
    return st.value


def dos_launch_count() -> int:
    return int(lib().dos_launch_count())


def dos_test_fail_alloc(after: int):
    """Make the library's device allocation after `after` more successful ones
    fail with DOS_ENOMEM (once); a negative value disarms."""
    _check(lib().dos_test_fail_alloc(int(after)))


def dos_profile_enable(on: bool = True):
    _check(lib().dos_profile_enable(1 if on else 0))


def dos_profile_read(reset: bool = True):
    """(total ms, launches) of the Chebyshev step kernels since the last reset."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().dos_profile_read(C.byref(ms), C.byref(n), 1 if reset else 0))
    return ms.value, n.value


def dos_set_plan(tile_width: int = 0, ctas_per_sm: int = 0):
    """Force the probe tile width (4..64) and light-kernel CTAs per SM; 0 = automatic."""
    _check(lib().dos_set_plan(int(tile_width), int(ctas_per_sm)))


def dos_get_plan(g: Graph, Nz: int, prec: str = "fp32") -> dict:
    t, p, tiles, gx = (C.c_int() for _ in range(4))
    _check(lib().dos_get_plan(g.handle, int(Nz), PREC[prec], C.byref(t), C.byref(p), C.byref(tiles), C.byref(gx)))
    return {"tile_width": t.value, "ctas_per_sm": p.value, "tiles": tiles.value, "grid_x": gx.value}


# ---------------------------------------------------------------------------
# whole-graph densities (the library does the assembly)
# ---------------------------------------------------------------------------
def density_with_spikes(d: torch.Tensor, g: Graph, n_bins: int, filter: Filter | None = None,
                        count_isolated: bool = True, kernel: str = "jackson", stream=None) -> torch.Tensor:
    """Histogram of the whole graph from moments d of the (filtered) operator
    (§3.4): dos_density with the graph and the filter."""
    return dos_density(d, n_bins, kernel=kernel, g=g, filter=filter, count_isolated=count_isolated, stream=stream)


def filtered_scale_and_spikes(g: Graph, filter: Filter | None = None, count_isolated: bool = True):
    """(r / N_total, [(lambda, count / N_total)]) from the library (dos_density_weights)."""
    return dos_density_weights(g, filter, count_isolated)


# ---------------------------------------------------------------------------
# batched density and the density-reconstruction network
# ---------------------------------------------------------------------------
def dos_density_batched(d: torch.Tensor, n_bins: int, kernel: str = "jackson",
                        hist_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per-graph histograms (n_graphs, n_bins) from moments d (n_graphs, M), float64 CUDA."""
    _need_cuda(d, torch.float64, "d")
    ng, M = d.shape
    if hist_out is None:
        hist_out = torch.empty((ng, n_bins), dtype=torch.float64, device=d.device)
    _need_cuda(hist_out, torch.float64, "hist_out", ng * n_bins)
    _check(lib().dos_density_batched(_ptr(d), int(M), int(ng), int(n_bins), KERNEL[kernel], _ptr(hist_out),
                                     _stream(stream)))
    return hist_out


def dos_mlp_create(sizes, seed: int = 0) -> Mlp:
    """Network sizes[0] -> ... -> sizes[-1] (ReLU hidden layers, softmax output)."""
    arr = (C.c_int * len(sizes))(*[int(x) for x in sizes])
    out = C.c_void_p()
    _check(lib().dos_mlp_create(len(sizes) - 1, arr, int(seed) & (2**64 - 1), C.byref(out)))
    return Mlp(out.value, sizes)


def dos_mlp_destroy(net: Mlp):
    net.close()


def dos_mlp_param_count(net: Mlp) -> int:
    n = C.c_int64()
    _check(lib().dos_mlp_param_count(net.handle, C.byref(n)))
    return n.value


def _dev():
    return torch.device("cuda", torch.cuda.current_device())


def dos_mlp_get_params(net: Mlp, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n = dos_mlp_param_count(net)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=_dev())
    _need_cuda(out, torch.float32, "out", n)
    _check(lib().dos_mlp_get_params(net.handle, _ptr(out), _stream(stream)))
    return out


def dos_mlp_set_params(net: Mlp, params: torch.Tensor, stream=None):
    _need_cuda(params, torch.float32, "params", dos_mlp_param_count(net))
    _check(lib().dos_mlp_set_params(net.handle, _ptr(params), _stream(stream)))


def dos_mlp_get_state(net: Mlp, stream=None) -> dict:
    """Training state: {"params", "m", "v"} (float32 CUDA tensors) and "step"."""
    n = dos_mlp_param_count(net)
    st = {k: torch.empty(n, dtype=torch.float32, device=_dev()) for k in ("params", "m", "v")}
    step = C.c_int64()
    _check(lib().dos_mlp_get_state(net.handle, _ptr(st["params"]), _ptr(st["m"]), _ptr(st["v"]), C.byref(step),
                                   _stream(stream)))
    st["step"] = step.value
    return st


def dos_mlp_set_state(net: Mlp, state: dict, stream=None):
    """Load a state from dos_mlp_get_state (tensors on any device)."""
    n = dos_mlp_param_count(net)
    t = {k: torch.as_tensor(state[k], dtype=torch.float32).to(_dev()).contiguous() for k in ("params", "m", "v")}
    for k, v in t.items():
        _need_cuda(v, torch.float32, k, n)
    _check(lib().dos_mlp_set_state(net.handle, _ptr(t["params"]), _ptr(t["m"]), _ptr(t["v"]), int(state["step"]),
                                   _stream(stream)))
    torch.cuda.synchronize()  # the copies have read t before it is released


def dos_mlp_forward(net: Mlp, x: torch.Tensor, probs: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Softmax output (rows, sizes[-1]) for features x (rows, sizes[0])."""
    _need_cuda(x, torch.float32, "x")
    rows = x.shape[0]
    if x.numel() != rows * net.sizes[0]:
        raise ValueError("x must have shape (rows, sizes[0])")
    if probs is None:
        probs = torch.empty((rows, net.sizes[-1]), dtype=torch.float32, device=x.device)
    _need_cuda(probs, torch.float32, "probs", rows * net.sizes[-1])
    _check(lib().dos_mlp_forward(net.handle, _ptr(x), int(rows), _ptr(probs), _stream(stream)))
    return probs


def dos_mlp_loss_grad(net: Mlp, x: torch.Tensor, t: torch.Tensor, stream=None):
    """(loss float32[1], flat gradient float32[param_count]) on the device."""
    _need_cuda(x, torch.float32, "x")
    _need_cuda(t, torch.float32, "t")
    rows = x.shape[0]
    if x.numel() != rows * net.sizes[0] or t.numel() != rows * net.sizes[-1]:
        raise ValueError("x and t must have shapes (rows, sizes[0]) and (rows, sizes[-1])")
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    grad = torch.empty(dos_mlp_param_count(net), dtype=torch.float32, device=x.device)
    _check(lib().dos_mlp_loss_grad(net.handle, _ptr(x), _ptr(t), int(rows), _ptr(loss), _ptr(grad),
                                   _stream(stream)))
    return loss, grad


def dos_mlp_train_step(net: Mlp, x: torch.Tensor, t: torch.Tensor, lr: float, idx: torch.Tensor | None = None,
                       loss: torch.Tensor | None = None, stream=None) -> torch.Tensor | None:
    """One Adam step on rows idx (int32 CUDA tensor; None = all rows of x)."""
    _need_cuda(x, torch.float32, "x")
    _need_cuda(t, torch.float32, "t")
    n_rows = x.shape[0]
    if x.numel() != n_rows * net.sizes[0] or t.numel() != n_rows * net.sizes[-1]:
        raise ValueError("x and t must have shapes (rows, sizes[0]) and (rows, sizes[-1])")
    if idx is not None:
        _need_cuda(idx, torch.int32, "idx")
        rows = idx.numel()
    else:
        rows = n_rows
    if loss is not None:
        _need_cuda(loss, torch.float32, "loss", 1)
    _check(lib().dos_mlp_train_step(net.handle, _ptr(x), _ptr(t), _ptr(idx), int(rows), float(lr), _ptr(loss),
                                    _stream(stream)))
    return loss


def dos_mlp_features(hist: torch.Tensor, d: torch.Tensor, K: int, stats: torch.Tensor | None = None,
                     x_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Feature rows [n_bins * hist, d_1 .. d_{K-1}] (+ 4 degree / noise entries
    with stats of shape (n_graphs, 4)), float32 (n_graphs, F)."""
    _need_cuda(hist, torch.float64, "hist")
    _need_cuda(d, torch.float64, "d")
    ng, B = hist.shape
    if d.shape[0] != ng or d.shape[1] < K:
        raise ValueError("d must have shape (n_graphs, >= K)")
    if stats is not None:
        _need_cuda(stats, torch.float64, "stats", 4 * ng)
    F = B + K - 1 + (4 if stats is not None else 0)
    if x_out is None:
        x_out = torch.empty((ng, F), dtype=torch.float32, device=hist.device)
    _need_cuda(x_out, torch.float32, "x_out", ng * F)
    _check(lib().dos_mlp_features(_ptr(hist), int(B), _ptr(d), int(d.shape[1]), int(K), _ptr(stats), int(ng),
                                  _ptr(x_out), _stream(stream)))
    return x_out


def dos_graph_stats(g: Graph, Nz: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """(mean degree, mean squared degree, largest degree, N * Nz), float64 CUDA (4,)."""
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _need_cuda(out, torch.float64, "out", 4)
    _check(lib().dos_graph_stats(g.handle, int(Nz), _ptr(out), _stream(stream)))
    return out


def dos_hist_normalize(hist: torch.Tensor, t_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Clip negative bins and renormalise each row to sum 1 (float32 targets)."""
    _need_cuda(hist, torch.float64, "hist")
    ng, B = hist.shape
    if t_out is None:
        t_out = torch.empty((ng, B), dtype=torch.float32, device=hist.device)
    _need_cuda(t_out, torch.float32, "t_out", ng * B)
    _check(lib().dos_hist_normalize(_ptr(hist), int(B), int(ng), _ptr(t_out), _stream(stream)))
    return t_out


def dos_hist_assemble(probs: torch.Tensor, scale: float = 1.0, spikes=(), hist_out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """float64 histograms scale * probs + point masses (spikes: (lambda, mass) pairs)."""
    _need_cuda(probs, torch.float32, "probs")
    rows, B = probs.shape
    if hist_out is None:
        hist_out = torch.empty((rows, B), dtype=torch.float64, device=probs.device)
    _need_cuda(hist_out, torch.float64, "hist_out", rows * B)
    sp = [float(x) for pair in spikes for x in pair]
    arr = (C.c_double * max(1, len(sp)))(*sp)
    _check(lib().dos_hist_assemble(_ptr(probs), int(B), int(rows), float(scale), arr if sp else None, len(sp) // 2,
                                   _ptr(hist_out), _stream(stream)))
    return hist_out


# ---------------------------------------------------------------------------
# Gauss quadrature and Lanczos (§3.2)
# ---------------------------------------------------------------------------
def dos_lanczos(g: Graph, M: int, Nz: int, seed: int, stream=None):
    """Lanczos coefficients of each probe: alpha, beta float64 (Nz, M) and steps int32 (Nz,), CUDA."""
    dev = torch.device("cuda", torch.cuda.current_device())
    alpha = torch.empty((Nz, M), dtype=torch.float64, device=dev)
    beta = torch.empty((Nz, M), dtype=torch.float64, device=dev)
    steps = torch.empty(Nz, dtype=torch.int32, device=dev)
    _check(lib().dos_lanczos(g.handle, int(M), int(Nz), int(seed) & (2**64 - 1), _ptr(alpha), _ptr(beta),
                             _ptr(steps), _stream(stream)))
    return alpha, beta, steps


def dos_lanczos_op(g: Graph, op: str, M: int, Nz: int, seed: int, stream=None):
    """dos_lanczos on op = "normalized_adjacency", "adjacency" or "laplacian"."""
    if op not in OPERATOR:
        raise ValueError(f"unknown operator {op!r}; one of {sorted(OPERATOR)}")
    dev = torch.device("cuda", torch.cuda.current_device())
    alpha = torch.empty((Nz, M), dtype=torch.float64, device=dev)
    beta = torch.empty((Nz, M), dtype=torch.float64, device=dev)
    steps = torch.empty(Nz, dtype=torch.int32, device=dev)
    _check(lib().dos_lanczos_op(g.handle, OPERATOR[op], int(M), int(Nz), int(seed) & (2**64 - 1), _ptr(alpha),
                                _ptr(beta), _ptr(steps), _stream(stream)))
    return alpha, beta, steps


BOUND = {"residual": 0, "ritz": 1}


def dos_spectral_interval(g: Graph, op: str, M: int = 30, Nz: int = 16, seed: int = 1, bound: str = "residual",
                          pad: float = 0.01, stream=None):
    """(a, b) holding the spectrum of the operator: extreme Ritz values widened
    by beta_M ("residual") or by the Ritz pair's residual ("ritz"), then by
    pad (b - a) at each end."""
    if op not in OPERATOR:
        raise ValueError(f"unknown operator {op!r}; one of {sorted(OPERATOR)}")
    if bound not in BOUND:
        raise ValueError(f"unknown bound {bound!r}; one of {sorted(BOUND)}")
    iv = (C.c_double * 2)()
    _check(lib().dos_spectral_interval(g.handle, OPERATOR[op], int(M), int(Nz), int(seed) & (2**64 - 1),
                                       BOUND[bound], float(pad), iv, _stream(stream)))
    return iv[0], iv[1]


def dos_ritz_bounds(alpha, beta, steps, bound: str = "residual", stream=None) -> torch.Tensor:
    """Per probe [theta_min - r, theta_max + r], float64 CUDA (Nz, 2)."""
    if bound not in BOUND:
        raise ValueError(f"unknown bound {bound!r}; one of {sorted(BOUND)}")
    nz, m = _lanczos_args(alpha, beta, steps)
    out = torch.empty((nz, 2), dtype=torch.float64, device=alpha.device)
    _check(lib().dos_ritz_bounds(_ptr(alpha), _ptr(beta), _ptr(steps), m, nz, BOUND[bound], _ptr(out),
                                 _stream(stream)))
    return out


def _lanczos_args(alpha, beta, steps):
    _need_cuda(alpha, torch.float64, "alpha")
    _need_cuda(beta, torch.float64, "beta", alpha.numel())
    _need_cuda(steps, torch.int32, "steps", alpha.shape[0])
    return alpha.shape[0], alpha.shape[1]


def dos_gauss_rules(alpha, beta, steps, stream=None):
    """Nodes and weights (Nz, M) of each probe's Gauss rule (0 past its steps)."""
    nz, m = _lanczos_args(alpha, beta, steps)
    nodes = torch.empty((nz, m), dtype=torch.float64, device=alpha.device)
    weights = torch.empty((nz, m), dtype=torch.float64, device=alpha.device)
    _check(lib().dos_gauss_rules(_ptr(alpha), _ptr(beta), _ptr(steps), m, nz, _ptr(nodes), _ptr(weights),
                                 _stream(stream)))
    return nodes, weights


def dos_gql_moments(alpha, beta, steps, m_count: int, stream=None) -> torch.Tensor:
    """Chebyshev moments of the probe-averaged Gauss rules (float64 CUDA, m_count)."""
    nz, m = _lanczos_args(alpha, beta, steps)
    d = torch.empty(m_count, dtype=torch.float64, device=alpha.device)
    _check(lib().dos_gql_moments(_ptr(alpha), _ptr(beta), _ptr(steps), m, nz, int(m_count), _ptr(d),
                                 _stream(stream)))
    return d


def dos_gql_histogram(nodes, weights, n_bins: int, stream=None) -> torch.Tensor:
    """Bin masses of the probe-averaged Gauss rules (float64 CUDA, n_bins)."""
    _need_cuda(nodes, torch.float64, "nodes")
    _need_cuda(weights, torch.float64, "weights", nodes.numel())
    nz, m = nodes.shape
    h = torch.empty(n_bins, dtype=torch.float64, device=nodes.device)
    _check(lib().dos_gql_histogram(_ptr(nodes), _ptr(weights), m, nz, int(n_bins), _ptr(h), _stream(stream)))
    return h


# ---------------------------------------------------------------------------
# other graph operators (Eq. (5) shift and scale)
# ---------------------------------------------------------------------------
def dos_moments_op(g: Graph, op: str, M: int, Nz: int, seed: int, prec: str = "fp32", interval=None,
                   d_out: torch.Tensor | None = None, stream=None):
    """DOS moments of (X - c) / r for X = "adjacency", "laplacian",
    "normalized_laplacian" or "normalized_adjacency"; interval [a, b] (None:
    Gershgorin for A and D - A).  Returns (d float64 CUDA (M,), (a, b))."""
    if op not in OPERATOR:
        raise ValueError(f"unknown operator {op!r}; one of {sorted(OPERATOR)}")
    if d_out is None:
        d_out = torch.empty(M, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _need_cuda(d_out, torch.float64, "d_out", M)
    lo, hi = (0.0, 0.0) if interval is None else (float(interval[0]), float(interval[1]))
    iv = (C.c_double * 2)()
    _check(lib().dos_moments_op(g.handle, OPERATOR[op], lo, hi, int(M), int(Nz), int(seed) & (2**64 - 1), PREC[prec],
                                _ptr(d_out), iv, _stream(stream)))
    return d_out, (iv[0], iv[1])


def ldos_moments_op(g: Graph, op: str, M: int, Nz: int, seed: int, interval=None,
                    C_out: torch.Tensor | None = None, d_out: torch.Tensor | None = None, stream=None):
    """LDOS moments C (float32 (M, N)) of (X - c) / r and the DOS moments
    (float64 (M,)); returns (C, d, (a, b))."""
    if op not in OPERATOR:
        raise ValueError(f"unknown operator {op!r}; one of {sorted(OPERATOR)}")
    n = g.n
    dev = torch.device("cuda", torch.cuda.current_device())
    if C_out is None:
        C_out = torch.empty((M, n), dtype=torch.float32, device=dev)
    _need_cuda(C_out, torch.float32, "C_out", M * n)
    if d_out is None:
        d_out = torch.empty(M, dtype=torch.float64, device=dev)
    _need_cuda(d_out, torch.float64, "d_out", M)
    lo, hi = (0.0, 0.0) if interval is None else (float(interval[0]), float(interval[1]))
    iv = (C.c_double * 2)()
    _check(lib().ldos_moments_op(g.handle, OPERATOR[op], lo, hi, int(M), int(Nz), int(seed) & (2**64 - 1),
                                 _ptr(C_out), _ptr(d_out), iv, _stream(stream)))
    return C_out, d_out, (iv[0], iv[1])


# ---------------------------------------------------------------------------
# traces and diagonals of matrix functions (§6)
# ---------------------------------------------------------------------------
FUNCTION = {"exp": 0, "resolvent": 1}


def dos_fn_coeffs(fn: str, p: float, interval, M: int, stream=None) -> torch.Tensor:
    """Chebyshev coefficients (float64 CUDA (M,)) of exp(p x) or 1 / (1 - p x) on the interval."""
    if fn not in FUNCTION:
        raise ValueError(f"unknown function {fn!r}; one of {sorted(FUNCTION)}")
    coef = torch.empty(M, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib().dos_fn_coeffs(FUNCTION[fn], float(p), float(interval[0]), float(interval[1]), int(M), _ptr(coef),
                               _stream(stream)))
    return coef


def dos_fn_trace(g: Graph, coef: torch.Tensor, d: torch.Tensor, stream=None) -> torch.Tensor:
    """tr f(X) (float64 CUDA (1,)) from DOS moments d and coefficients coef on the same interval."""
    _need_cuda(coef, torch.float64, "coef")
    _need_cuda(d, torch.float64, "d", coef.numel())
    out = torch.empty(1, dtype=torch.float64, device=coef.device)
    _check(lib().dos_fn_trace(g.handle, _ptr(coef), _ptr(d), coef.numel(), _ptr(out), _stream(stream)))
    return out


def dos_fn_diag(C_moments: torch.Tensor, coef: torch.Tensor, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """f(X)_kk (float64 CUDA (N,)) from LDOS moments (float32 (M, N)) and coefficients."""
    _need_cuda(C_moments, torch.float32, "C_moments")
    m, n = C_moments.shape
    _need_cuda(coef, torch.float64, "coef", m)
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=C_moments.device)
    _need_cuda(out, torch.float64, "out", n)
    _check(lib().dos_fn_diag(_ptr(C_moments), int(n), int(m), _ptr(coef), _ptr(out), _stream(stream)))
    return out


def matrix_function_trace(g: Graph, op: str, fn: str, p: float, M: int = 100, Nz: int = 32, seed: int = 1,
                          interval=None, stream=None):
    """tr f(X) of op ("adjacency", "laplacian", ...) by KPM: the interval
    (Lanczos Ritz bounds unless given), DOS moments, coefficients, trace.
    Returns (trace, (a, b)).  exp with p = 1 on A: the Estrada index."""
    if interval is None:
        interval = dos_spectral_interval(g, op, 30, 8, seed + 1, bound="ritz", stream=stream)
    d, iv = dos_moments_op(g, op, M, Nz, seed, interval=interval, stream=stream)
    coef = dos_fn_coeffs(fn, p, iv, M, stream=stream)
    return float(dos_fn_trace(g, coef, d, stream=stream).item()), iv


def matrix_function_diag(g: Graph, op: str, fn: str, p: float, M: int = 100, Nz: int = 32, seed: int = 1,
                         interval=None, stream=None):
    """f(X)_kk of every node with edges (float64 CUDA (N,), compact ids) from
    LDOS moments: exp with p = 1 on A gives subgraph centrality, resolvent
    with p < 1 / lambda_max resolvent centrality.  Returns (diag, (a, b))."""
    if interval is None:
        interval = dos_spectral_interval(g, op, 30, 8, seed + 1, bound="ritz", stream=stream)
    cm, _, iv = ldos_moments_op(g, op, M, Nz, seed, interval=interval, stream=stream)
    coef = dos_fn_coeffs(fn, p, iv, M, stream=stream)
    return dos_fn_diag(cm, coef, stream=stream), iv


# ---------------------------------------------------------------------------
# nested dissection (§3.3, Algorithm 1)
# ---------------------------------------------------------------------------
def dos_pdos_nd(g: Graph, M: int, leaf_size: int = 64, max_entries: float = 1e9, C_out: torch.Tensor | None = None,
                stream=None):
    """Exact PDOS moments C (M, N) float32 CUDA, C[m, k] = T_m(H)_kk, and the
    partition statistics."""
    n = g.n
    if C_out is None:
        C_out = torch.empty((M, n), dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    _need_cuda(C_out, torch.float32, "C_out", M * n)
    st = (C.c_int64 * 4)()
    _check(lib().dos_pdos_nd(g.handle, int(M), int(leaf_size), float(max_entries), _ptr(C_out), st, _stream(stream)))
    return C_out, {"tree_nodes": st[0], "depth_levels": st[1], "block_entries": st[2], "max_separator": st[3]}
