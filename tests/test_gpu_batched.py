"""Batched uneven solves (aao_rk_solve_batched): every problem of a batch equals its
stand-alone solve bit for bit (same handle, same kernels, deterministic reductions),
and one of them equals the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle.solve import OracleOptions, build, solve as oracle_solve

from gpu_util import dev, host, to_dev, torch, zeros

pytestmark = pytest.mark.gpu


def test_batched_equals_standalone():
    from paper_2609_16863_gb300 import Solver, radau_iia, solve_batched
    dev()
    specs = [((32, 32), 8, 2), ((48, 40), 4, 3), ((20, 24), 16, 2), ((64, 64), 4, 3), ((17, 33), 6, 3),
             ((32, 32), 12, 3)]
    solvers, fs, us = [], [], []
    for p, (ns, nt, s) in enumerate(specs):
        st = torch.cuda.Stream()
        solvers.append(Solver(ns, 1.0, nt, tableau=radau_iia(s), prec_P="fp64", tol=1e-10, stream=st.cuda_stream))
        fs.append(to_dev(synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(4, "f", p))))
        us.append(to_dev(synth.gaussian_random_field(ns, 0.1, 1.0, synth.rng_for(4, "u0", p))))
    xs = [zeros(S.n_st) for S in solvers]
    infos = solve_batched(solvers, fs, us, xs)
    torch.cuda.synchronize()
    for S, f, u, xb, info in zip(solvers, fs, us, xs, infos):
        xa, ia = S.solve(f, u, zeros(S.n_st))
        torch.cuda.synchronize()
        assert info.converged and ia.outer_its == info.outer_its
        assert torch.equal(xa, xb)
    ns, nt, s = specs[1]
    op = build(ns, 1.0, nt, "radau", s)
    ref = oracle_solve(op, ns, op.rhs(host(us[1]), host(fs[1])),
                       OracleOptions(tol=1e-10, inner_maxit=5, inner_tol=1e-6))
    assert np.linalg.norm(host(xs[1]) - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


def test_batched_mixed_precision_and_error_propagation():
    from paper_2609_16863_gb300 import Solver, radau_iia, solve_batched, _lib
    dev()
    specs = [((32, 32), 8, 2), ((40, 40), 8, 3)]
    solvers = [Solver(ns, 1.0, nt, tableau=radau_iia(s), prec_P="fp32", tol=1e-8,
                      stream=torch.cuda.Stream().cuda_stream) for ns, nt, s in specs]
    fs = [to_dev(synth.random_vector(S.nx, 1)) for S in solvers]
    us = [to_dev(synth.random_vector(S.nx, 2)) for S in solvers]
    xs = [zeros(S.n_st) for S in solvers]
    infos = solve_batched(solvers, fs, us, xs)
    assert all(i.converged and i.rel_res <= 1e-8 for i in infos)
    # a problem that cannot converge within maxit reports its status through the batch
    solvers[0].set_tolerances(maxit=1, tol=1e-14)
    with pytest.raises(_lib.AaoError) as e:
        solve_batched(solvers, fs, us, xs)
    assert "problem 0" in str(e.value)
