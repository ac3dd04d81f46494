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
    # outer_its, (pad), inner_its_total, rel_res, converged, (pad), 3 times, n_history, (pad),
    # history[128], relaxed_matvecs, (pad)
    assert ctypes.sizeof(_lib.aao_info) == 4 + 4 + 8 + 8 + 4 + 4 + 8 * 3 + 4 + 4 + 8 * 128 + 4 + 4
    # tol, restart, maxit, inner_maxit, (pad), inner_tol, mg_cycles, mg_pre, mg_post, (pad), mg_omega,
    # cheb_steps, prec_P, prec_Pint, ckpt_every, stream, mgrit_m, precond_side, relax_matvec
    assert ctypes.sizeof(_lib.aao_options) == 8 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 4 + 8 + 4 * 4 + 8 + 4 + 4 + 8
    assert _lib.aao_options.precond_side.offset == 84
    assert _lib.aao_options.mgrit_m.offset == 80
    assert _lib.aao_options.relax_matvec.offset == 88


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every field offset and struct size of the ctypes binding equals what a C compiler gives for
    include/aao_rk.h (the header and the binding cannot drift apart)."""
    import shutil
    import subprocess
    from paper_2609_16863_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [_lib.aao_grid, _lib.aao_tableau, _lib.aao_options, _lib.aao_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "aao_rk.h"', 'int main(void) {']
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        for name, *_ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {name}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for st in structs:
        want.append(ctypes.sizeof(st))
        want += [getattr(st, name).offset for name, *_ in st._fields_]
    assert got == want


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


def _valid_setup_args():
    from paper_2609_16863_gb300 import _lib
    L = _lib.load()
    g = _lib.aao_grid()
    g.dim = 2
    g.n[0] = g.n[1] = 8
    g.n[2] = 1
    g.len[0] = g.len[1] = g.len[2] = 1.0
    g.disc = 0
    t = _lib.aao_tableau()
    t.s = 2
    o = _lib.aao_options()
    L.aao_rk_default_options(ctypes.byref(o))
    return L, g, t, o


def _set(obj, field, value):
    if "[" in field:
        name, idx = field[:-1].split("[")
        getattr(obj, name)[int(idx)] = value
    else:
        setattr(obj, field, value)


# (what to change, value, words expected in the error message); every case fails in argument
# validation, before any device call
SETUP_BAD = [
    ("grid.dim", 1, b"dim"), ("grid.dim", 4, b"dim"), ("grid.n[1]", 0, b"grid sizes"),
    ("grid.len[0]", -1.0, b"grid sizes"), ("grid.len[1]", float("nan"), b"grid sizes"),
    ("grid.len[0]", float("inf"), b"grid sizes"),
    ("grid.disc", 7, b"discretisation"), ("q1_kappa", None, b"kappa"),
    ("tau", 0.0, b"tau"), ("tau", float("nan"), b"tau"), ("nt", 0, b"tau"), ("nt", 65535, b"65534"),
    ("tab.s", 0, b"stages"), ("tab.s", 9, b"stages"),
    ("opts.restart", 0, b"restart"), ("opts.restart", 65, b"restart"), ("opts.maxit", -1, b"restart"),
    ("opts.tol", float("nan"), b"restart"), ("opts.tol", -1.0, b"restart"),
    ("opts.inner_maxit", 17, b"inner_maxit"), ("opts.mg_cycles", 0, b"mg_cycles"),
    ("opts.mg_pre", -1, b"mg_pre"), ("opts.mg_post", -1, b"mg_pre"), ("opts.mg_omega", 0.0, b"mg_omega"),
    ("opts.prec_P", 7, b"precision"), ("fp64_fp32", None, b"FP64"), ("bf16_fp32", None, b"16-bit"),
    ("fp16_bf16", None, b"16-bit"), ("null_grid", None, b"null"), ("null_out", None, b"null output"),
    ("opts.mgrit_m", 1, b"mgrit_m"), ("opts.mgrit_m", 5, b"mgrit_m"), ("opts.mgrit_m", -2, b"mgrit_m"),
    ("opts.precond_side", 2, b"precond_side"),
    ("opts.relax_matvec", -1.0, b"relax_matvec"), ("opts.relax_matvec", float("nan"), b"relax_matvec"),
    ("opts.relax_matvec", float("inf"), b"relax_matvec"),
]


@pytest.mark.parametrize("case", ["q1", "left"])
def test_relaxed_product_needs_fd_and_right_preconditioning(lib, case):
    """The FP32 relaxed product is built for finite differences, and its allowance is stated for the
    right-preconditioned residual: other combinations are refused at set-up, before device work."""
    L, g, t, o = _valid_setup_args()
    o.relax_matvec = 1.0
    if case == "q1":
        g.disc = 1
    else:
        o.precond_side = 1
    out = ctypes.c_void_p()
    st = L.aao_rk_setup(ctypes.byref(g), 0.1, 4, ctypes.byref(t), ctypes.byref(o), ctypes.byref(out))
    assert st == -8 and not out.value
    assert b"relax_matvec" in L.aao_rk_last_error()


@pytest.mark.parametrize("what,value,words", SETUP_BAD)
def test_setup_validation_table(lib, what, value, words):
    L, g, t, o = _valid_setup_args()
    tau, nt = 0.1, 4
    gp, out = ctypes.byref(g), ctypes.c_void_p()
    outp = ctypes.byref(out)
    if what == "q1_kappa":
        g.disc = 1
        g.kappa = 0x1000                  # never dereferenced: rejected first
    elif what == "fp64_fp32":
        o.prec_P, o.prec_Pint = 0, 1
    elif what == "bf16_fp32":
        o.prec_P, o.prec_Pint = 2, 1
    elif what == "fp16_bf16":
        o.prec_P, o.prec_Pint = 3, 2
    elif what == "null_grid":
        gp = None
    elif what == "null_out":
        outp = None
    elif what == "tau":
        tau = value
    elif what == "nt":
        nt = value
    else:
        obj, field = what.split(".", 1)
        _set({"grid": g, "tab": t, "opts": o}[obj], field, value)
    st = L.aao_rk_setup(gp, tau, nt, ctypes.byref(t), ctypes.byref(o), outp)
    assert st == -1
    assert not out.value
    assert words in L.aao_rk_last_error(), L.aao_rk_last_error()


NOALLOC_BAD = [
    ("null_grid", b"null"), ("dim", b"dim"), ("kappa", b"constant-coefficient"), ("q1", b"constant-coefficient"),
    ("c", b"c >= 0"), ("cycles", b"cycles"), ("pre", b"pre/post"), ("omega", b"omega"),
    ("size0", b"positive"), ("too_large", b"65536"), ("len0", b"lengths"), ("len_inf", b"lengths"),
    ("len_nan", b"lengths"), ("c_inf", b"finite c"),
]


@pytest.mark.parametrize("what,words", NOALLOC_BAD)
def test_noalloc_validation_table(lib, what, words):
    L, g, _, _ = _valid_setup_args()
    args = dict(c=0.01, cycles=3, pre=2, post=2, omega=0.8)
    gp = ctypes.byref(g)
    if what == "null_grid":
        gp = None
    elif what == "dim":
        g.dim = 1
    elif what == "kappa":
        g.kappa = 0x1000
    elif what == "q1":
        g.disc = 1
    elif what == "c":
        args["c"] = -1.0
    elif what == "cycles":
        args["cycles"] = 0
    elif what == "pre":
        args["pre"] = -1
    elif what == "omega":
        args["omega"] = float("nan")
    elif what == "size0":
        g.n[0] = 0
    elif what == "too_large":
        g.n[0], g.n[1] = 300, 300
    elif what == "len0":
        g.len[0] = 0.0
    elif what == "len_inf":
        g.len[1] = float("inf")
    elif what == "len_nan":
        g.len[0] = float("nan")
    elif what == "c_inf":
        args["c"] = float("inf")
    dummy = ctypes.c_void_p(0x1000)       # never dereferenced: rejected first
    st = L.aao_rk_shifted_solve_noalloc(gp, ctypes.c_double(args["c"]), args["cycles"], args["pre"], args["post"],
                                        ctypes.c_double(args["omega"]), dummy, dummy, None)
    assert st == -1
    assert words in L.aao_rk_last_error(), L.aao_rk_last_error()


def test_batched_validation(lib):
    from paper_2609_16863_gb300 import _lib
    L = _lib.load()
    assert L.aao_rk_solve_batched(0, None, None, None, None, None) == 0     # empty batch: no device work
    assert L.aao_rk_solve_batched(-1, None, None, None, None, None) == -1
    assert L.aao_rk_solve_batched(1, None, None, None, None, None) == -1
    hs = (ctypes.c_void_p * 1)(None)
    vec = (ctypes.c_void_p * 1)(0x1000)
    assert L.aao_rk_solve_batched(1, hs, vec, vec, vec, None) == -1
    assert b"null handle" in L.aao_rk_last_error()


def test_batched_rejects_a_repeated_handle(lib):
    """Handles are not thread-safe; a batch may not name one twice (checked before any device call)."""
    from paper_2609_16863_gb300 import _lib
    L = _lib.load()
    hs = (ctypes.c_void_p * 3)(0x1000, 0x2000, 0x1000)     # never dereferenced: rejected first
    vec = (ctypes.c_void_p * 3)(0x3000, 0x3000, 0x3000)
    assert L.aao_rk_solve_batched(3, hs, vec, vec, vec, None) == -1
    assert b"more than once" in L.aao_rk_last_error()


def test_setup_rejects_library_side_checkpointing(lib):
    L, g, t, o = _valid_setup_args()
    o.ckpt_every = 4
    h = ctypes.c_void_p()
    st = L.aao_rk_setup(ctypes.byref(g), 0.1, 4, ctypes.byref(t), ctypes.byref(o), ctypes.byref(h))
    assert st == -8 and not h.value
    assert b"aao_rk_grad_kappa" in L.aao_rk_last_error()


def test_batched_refuses_while_a_launch_profile_is_open(lib):
    from paper_2609_16863_gb300 import _lib
    L = _lib.load()
    assert L.aao_rk_profile_begin(b"k_cluster_mg") == 0
    try:
        hs = (ctypes.c_void_p * 2)(0x1000, 0x2000)          # never dereferenced: rejected first
        vec = (ctypes.c_void_p * 2)(0x3000, 0x3000)
        assert L.aao_rk_solve_batched(2, hs, vec, vec, vec, None) == -1
        assert b"launch profile" in L.aao_rk_last_error()
    finally:
        L.aao_rk_profile_end(None, None, None)              # closes the profile (no device here)
