"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/netdos.h declares (CPU only: no compute call is made)."""
import ctypes
import shutil

import pytest

import paper_1905_09758_gb300 as nd
from paper_1905_09758_gb300 import _binding
from paper_1905_09758_gb300.build import LIB, build


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return build()


def test_header_declares_the_boundary():
    names = nd.header_functions()
    for must in ("dos_build_csr", "dos_moments", "ldos_moments", "dos_density", "dos_motif_filter",
                 "dos_graph_export", "dos_last_error"):
        assert must in names


def test_every_declaration_cites_its_passage():
    """Each declaration's comment (or the comment of the section it opens a
    group in) names the passage that defines the operation, or says that it
    is not in the paper (instrumentation, tuning, project additions)."""
    import os
    import re

    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "netdos.h")).read()
    marks = ("§", "Eq.", "Algorithm", "Fig.", "not in the paper", "project addition", "Project addition")
    decl = re.compile(r"/\*((?:(?!\*/).)*)\*/\s*\n(?:int|void|const char\*|int64_t|uint64_t)\s+(\w+)\(", re.S)
    missing = [name for com, name in decl.findall(text) if not any(m in com for m in marks)]
    assert not missing, missing


def test_library_exports_every_declared_symbol(libpath):
    assert libpath == LIB
    handle = ctypes.CDLL(libpath)
    missing = [f for f in nd.header_functions() if not hasattr(handle, f)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(nd.header_functions()) == set(_binding._SIGNATURES)


def test_version_and_error_text_without_gpu(libpath):
    lib = nd.lib()
    assert lib.dos_version() == 100
    # argument validation happens before any CUDA call
    assert lib.dos_moments(None, None, 10, 4, 1, 0, None, None) == nd.DOS_EINVAL
    assert b"NULL" in lib.dos_last_error() or b"null" in lib.dos_last_error()
    assert lib.dos_set_plan(3, 0) == nd.DOS_EINVAL
    assert lib.dos_set_plan(0, -1) == nd.DOS_EINVAL
    assert lib.dos_set_plan(0, 2) == nd.DOS_OK
    assert lib.dos_set_plan(0, 0) == nd.DOS_OK
