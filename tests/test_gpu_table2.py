"""The paper's exact-solution problem of Sec. 5.1 (Table 2) solved on the GPU with Q1 elements.

v = exp(t_f - t) cos(pi x1 / 2) cos(pi x2 / 2) + 1 on [-1, 1]^2, t_f = 2; writing v = 1 + w, w has
zero Dirichlet data (oracle.problems).  The right-hand side (M w(0) and the FE load vectors of the
source at the stage times) comes from the oracle's problem assembly and is passed through
aao_rk_solve_rhs; the GPU solve must reach the oracle's direct solution and reproduce its v_error,
which the oracle's own tests pin to Table 2's printed values (Q1: 7-35% above them, at every level).
The outer iteration counts are printed beside Table 2's (context: the paper's AMG is not ours)."""
import os

import numpy as np
import pytest

from oracle.problems import exact_solution_problem
from oracle.sequential import sequential_solve

from gpu_util import dev, host, to_dev, torch, zeros

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_verror.txt")
TABLE = {(int(r[0]), int(r[1])): (float(r[2]), float(r[3]))
         for r in (ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#"))}


@pytest.mark.parametrize("s,l,prec", [(2, 3, "fp64"), (2, 5, "fp64"), (3, 4, "fp64"), (4, 4, "fp64"),
                                      (5, 3, "fp64"), (2, 6, "fp32"), (3, 5, "fp32"), (2, 7, "fp32")])
def test_q1_exact_solution_problem_on_gpu(s, l, prec):
    from paper_2609_16863_gb300 import Solver
    from paper_2609_16863_gb300.tableau import make as tab
    dev()
    P = exact_solution_problem("q1", l, s)
    op = P.op
    itol = 1e-6 if prec == "fp64" else 1e-3
    S = Solver((P.n, P.n), P.tf, op.nt, tableau=tab("radau", s), lens=(2.0, 2.0), disc="q1", prec_P=prec,
               inner_maxit=3, inner_tol=itol, tol=1e-10)
    rhs = P.rhs()
    x, info = S.solve_rhs(to_dev(rhs), zeros(op.n_st))
    x = host(x)
    ref = sequential_solve(op, rhs)
    err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
    e_gpu, e_ref = P.v_error(x), P.v_error(ref)
    print(f"Q1 s={s} l={l} [{prec}]: n_st {op.n_st}, outer its {info.outer_its}, rel err vs direct {err:.2e}, "
          f"v_error {e_gpu:.4e} (oracle {e_ref:.4e}, Table 2 {TABLE[(s, l)][0]:.2e})")
    assert info.converged and err <= 1e-8
    assert abs(e_gpu - e_ref) <= 1e-6 * e_ref
    assert 1.0 <= e_gpu / TABLE[(s, l)][0] <= 1.4
