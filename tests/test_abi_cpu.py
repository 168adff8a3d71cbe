"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ibm.h")


def _header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z_]+)\s*\(", text)))


def _lib():
    p = os.path.join(ROOT, "paper_2506_14328_gb300", "libibm.so")
    if not os.path.exists(p):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(p)


def test_library_exports_every_header_symbol():
    lib = _lib()
    names = _header_functions()
    assert "ibm_step" in names and "ibm_setup_geometry" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_same_symbols():
    import paper_2506_14328_gb300 as P
    assert sorted(P.EXPORTED) == _header_functions()


def _grid(**kw):
    import paper_2506_14328_gb300 as P
    g = P.ibm_grid_desc()
    g.ndim = kw.get("ndim", 3)
    for d, v in enumerate(kw.get("n", (8, 8, 8))):
        g.n[d] = v
    for d in range(3):
        g.L[d] = 1.0
    bl = kw.get("bc_lo", (0, 1, 0))
    bh = kw.get("bc_hi", (0, 1, 0))
    for d in range(3):
        g.bc_lo[d] = bl[d]
        g.bc_hi[d] = bh[d]
    g.precision = kw.get("precision", 0)
    return g


@pytest.mark.parametrize("kw,status", [
    (dict(ndim=4), -1),
    (dict(n=(8, 1, 8)), -1),
    (dict(ndim=2, n=(8, 8, 4)), -1),
    (dict(precision=7), -1),
    (dict(bc_lo=(1, 1, 0)), -4),
    (dict(bc_lo=(0, 3, 0)), -4),
])
def test_invalid_grids_are_rejected_before_any_cuda_call(kw, status):
    import paper_2506_14328_gb300 as P
    b = ctypes.c_size_t(0)
    st = P.lib.ibm_workspace_bytes(ctypes.byref(_grid(**kw)), ctypes.byref(b))
    assert st == status
    assert P.ibm_last_error() != ""


def test_null_handles_are_rejected():
    import paper_2506_14328_gb300 as P
    assert P.lib.ibm_step(None, 1, 0) == P.IBM_E_INVALID
    assert P.lib.ibm_project(None) == P.IBM_E_INVALID
    P.lib.ibm_destroy(None)
