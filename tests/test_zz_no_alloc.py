"""The allocation-free shifted solve (aao_rk_shifted_solve_noalloc) against the
handle-based aao_rk_shifted_solve and against the oracle's V-cycles.

The allocation-free entry point is for callers that cannot call cudaMalloc
(pools that forbid it, hosts that only hand out pre-registered buffers,
applications that must not allocate after start-up): all of its scratch lives
in one fixed device array inside the library.  This file runs last so that a
failure here leaves every other test already run; it passes in a fresh process
and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import synth

from gpu_util import dev, host, rel_max, to_dev, torch, zeros

pytestmark = pytest.mark.gpu


def _grid(ns):
    from paper_2609_16863_gb300 import _lib
    g = _lib.aao_grid()
    g.dim = len(ns)
    for a in range(3):
        g.n[a] = ns[a] if a < len(ns) else 1
        g.len[a] = 1.0
    g.disc = 0
    g.kappa = None
    return g


@pytest.mark.parametrize("ns", [(48, 40), (256, 256), (12, 10, 14)])
def test_noalloc_matches_handle_shifted_solve_twice(ns):
    import scipy.sparse as sp
    from oracle.multigrid import Hierarchy
    from oracle.operators import operators
    from paper_2609_16863_gb300 import Solver, _lib, radau_iia
    dev()
    lib = _lib.lib()
    T, nt, s = 1.0, 8, 3
    S = Solver(ns, T, nt, tableau=radau_iia(s), prec_P="fp64", mg_cycles=3, mg_pre=2, mg_post=2, mg_omega=0.8)
    A, _, _ = radau_iia(s)
    c = (T / nt) * A[0, 0]           # shift of stage 1: tau * d_1, d_1 = a_11 (first LDU pivot)
    g = _grid(ns)
    _, K = operators(ns)
    mg = Hierarchy(sp.identity(S.nx, format="csr") + c * K, ns, omega=0.8, nu1=2, nu2=2)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):            # two calls in a row share (and must reset) the scratch
        bh = synth.random_vector(S.nx, 90 + call)
        b = to_dev(bh)
        ref = host(S.shifted_solve(0, b, zeros(S.nx)))
        x = zeros(S.nx)
        st = lib.aao_rk_shifted_solve_noalloc(C.byref(g), c, 3, 2, 2, 0.8, C.c_void_p(b.data_ptr()),
                                             C.c_void_p(x.data_ptr()), C.c_void_p(stream))
        _lib.check(st)
        xh = host(x)
        assert rel_max(xh, ref) <= 1e-12
        assert rel_max(xh, mg.solve(bh, 3)) <= 1e-12


def test_noalloc_rejects_oversize_and_host_buffers():
    from paper_2609_16863_gb300 import _lib
    dev()
    lib = _lib.lib()
    b = zeros(300 * 300)
    x = zeros(300 * 300)
    st = lib.aao_rk_shifted_solve_noalloc(C.byref(_grid((300, 300))), 0.1, 3, 2, 2, 0.8,
                                         C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), None)
    assert st == -1 and b"too large" in lib.aao_rk_last_error()
    hb = np.zeros(64)
    hx = np.zeros(64)
    st = lib.aao_rk_shifted_solve_noalloc(C.byref(_grid((8, 8))), 0.1, 3, 2, 2, 0.8,
                                         C.c_void_p(hb.ctypes.data), C.c_void_p(hx.ctypes.data), None)
    assert st == -1
