"""The C ABI library loads and exports every entry point include/aao_rk.h declares
(no compute: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aao_rk.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aao_rk_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_16863_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_lists_the_paths_entry_points():
    names = declared_functions()
    for required in ("aao_rk_setup", "aao_rk_matvec", "aao_rk_precond_apply", "aao_rk_solve",
                     "aao_rk_adjoint_solve", "aao_rk_solve_batched", "aao_rk_destroy", "aao_rk_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_2609_16863_gb300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert bound == set(declared_functions())


def test_struct_layouts_match_header_sizes():
    # sizes follow the C layout rules on every 64-bit target this builds for
    from paper_2609_16863_gb300 import _lib
    assert ctypes.sizeof(_lib.aao_tableau) == 4 + 4 + 8 * 64 + 8 * 8 + 8 * 8
    assert ctypes.sizeof(_lib.aao_info) == 4 + 4 + 8 + 8 + 4 + 4 + 8 * 3 + 4 + 4 + 8 * 128


def test_setup_rejects_bad_arguments_without_gpu(lib):
    # argument validation happens before any device call
    from paper_2609_16863_gb300 import _lib
    L = _lib.load()
    g = _lib.aao_grid()
    g.dim = 4
    t = _lib.aao_tableau()
    t.s = 2
    o = _lib.aao_options()
    L.aao_rk_default_options(ctypes.byref(o))
    h = ctypes.c_void_p()
    st = L.aao_rk_setup(ctypes.byref(g), 0.1, 4, ctypes.byref(t), ctypes.byref(o), ctypes.byref(h))
    assert st == -1 and not h.value
    assert b"dim" in L.aao_rk_last_error()
    g.dim = 2
    g.n[0] = g.n[1] = 8
    g.len[0] = g.len[1] = 1.0
    o.prec_P, o.prec_Pint = 1, 0          # FP32 P with FP64 P_int is not a supported pair
    st = L.aao_rk_setup(ctypes.byref(g), 0.1, 4, ctypes.byref(t), ctypes.byref(o), ctypes.byref(h))
    assert st == -1
