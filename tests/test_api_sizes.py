"""The Python binding checks that every vector holds the values the library will touch (the C ABI
takes plain pointers and cannot), before any call: exercised on the CPU against a stand-in for the
library's entry points."""
import numpy as np
import pytest

from paper_2609_16863_gb300 import api


class _FakeLib:
    """Records calls; every entry point succeeds."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append(name)
            return 0
        return fn


def _solver(ns=(5, 4), nt=3, s=2):
    S = api.Solver.__new__(api.Solver)
    S._lib = _FakeLib()
    S.h = 1
    S.n = ns
    S.dim = len(ns)
    S.n_nodes = int(np.prod([v + 2 for v in ns]))
    S.s, S.nt = s, nt
    S.nx = int(np.prod(ns))
    S.n_st = S.nx * (nt + 1 + s * nt)
    S.n_v = (nt + 1) * S.nx
    return S


def _v(n):
    return np.zeros(max(n, 0))


def _calls(S):
    """(method, argument builder from sizes) for every vector entry point."""
    nx, nst, s, nt, nn = S.nx, S.n_st, S.s, S.nt, S.n_nodes
    return [
        ("rhs", lambda d: S.rhs(_v(nx + d[0]), _v(nx + d[1]), _v(nst + d[2]))),
        ("rhs_td", lambda d: S.rhs(_v(nt * s * nx + d[0]), _v(nx + d[1]), _v(nst + d[2]), f_time_dep=True)),
        ("matvec", lambda d: S.matvec(_v(nst + d[0]), _v(nst + d[1]))),
        ("matvec_T", lambda d: S.matvec(_v(nst + d[0]), _v(nst + d[1]), transpose=True)),
        ("precond", lambda d: S.precond_apply(_v(nst + d[0]), _v(nst + d[1]))),
        ("shifted", lambda d: S.shifted_solve(0, _v(nx + d[0]), _v(nx + d[1]))),
        ("pint", lambda d: S.pint_apply(_v(s * nx + d[0]), _v(s * nx + d[1]))),
        ("inner", lambda d: S.inner_solve(2, _v(2 * s * nx + d[0]), _v(2 * s * nx + d[1]))),
        ("solve", lambda d: S.solve(_v(nx + d[0]), _v(nx + d[1]), _v(nst + d[2]))),
        ("solve_rhs", lambda d: S.solve_rhs(_v(nst + d[0]), _v(nst + d[1]))),
        ("adjoint", lambda d: S.adjoint_solve(_v(nst + d[0]), _v(nst + d[1]), x_fwd=_v(nst + d[2]),
                                               grad_f=_v(nx + d[3]), grad_kappa=_v(nn + d[4]))),
        ("grad_kappa", lambda d: S.grad_kappa(_v(nst + d[0]), _v(nst + d[1]), _v(nn + d[2]))),
    ]


NARGS = {"rhs": 3, "rhs_td": 3, "matvec": 2, "matvec_T": 2, "precond": 2, "shifted": 2, "pint": 2, "inner": 2,
         "solve": 3, "solve_rhs": 2, "adjoint": 5, "grad_kappa": 3}


@pytest.mark.parametrize("shape", [((5, 4), 3, 2), ((3, 4, 2), 2, 3)])
def test_exact_and_larger_sizes_pass_short_ones_fail(shape):
    S = _solver(*shape)
    for name, call in _calls(S):
        k = NARGS[name]
        call([0] * k)                                   # exact sizes
        call([3] * k)                                   # larger buffers are allowed
        for i in range(k):                              # any one vector a value short
            d = [0] * k
            d[i] = -1
            before = len(S._lib.calls)
            with pytest.raises(ValueError):
                call(d)
            assert len(S._lib.calls) == before, name    # rejected before the library is called


def test_optional_adjoint_outputs_may_be_absent():
    S = _solver()
    S.adjoint_solve(_v(S.n_st), _v(S.n_st))


def test_batched_sizes(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(api._lib, "lib", lambda: fake)
    A, B = _solver((5, 4), 3, 2), _solver((6, 6), 2, 3)
    api.solve_batched([A, B], [_v(A.nx), _v(B.nx)], [_v(A.nx), _v(B.nx)], [_v(A.n_st), _v(B.n_st)])
    with pytest.raises(ValueError):
        api.solve_batched([A, B], [_v(A.nx), _v(A.nx)], [_v(A.nx), _v(B.nx)], [_v(A.n_st), _v(B.n_st)])
    with pytest.raises(ValueError):
        api.solve_batched([A, B], [_v(A.nx)], [_v(A.nx), _v(B.nx)], [_v(A.n_st), _v(B.n_st)])
    assert fake.calls == ["aao_rk_solve_batched"]


def test_dtype_and_layout_still_checked():
    S = _solver()
    with pytest.raises(TypeError):
        S.shifted_solve(0, np.zeros(S.nx, dtype=np.float32), _v(S.nx))
    with pytest.raises(TypeError):
        S.shifted_solve(0, np.zeros((S.nx, 2))[:, 0], _v(S.nx))
