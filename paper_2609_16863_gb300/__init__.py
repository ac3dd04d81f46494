"""GB300 all-at-once Runge--Kutta heat-equation solver with a mixed-precision
block-triangular preconditioner (hand-written CUDA for sm_103a behind a C ABI).

    from paper_2609_16863_gb300 import Solver, radau_iia
    S = Solver((256, 256), T=1.0, nt=128, tableau=radau_iia(3), prec_P="fp32")
    x, info = S.solve(f, u0, x)          # torch.cuda float64 tensors or numpy arrays
"""
from .tableau import gauss_legendre, radau_iia
from .api import Info, Solver, solve_batched
from .tune import tune_mgrit

__all__ = ["Solver", "Info", "solve_batched", "radau_iia", "gauss_legendre", "tune_mgrit"]
