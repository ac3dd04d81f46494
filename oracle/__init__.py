"""FP64 CPU oracle for the all-at-once Runge--Kutta heat-equation solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call,
link or execute anything in this directory; only the tests, the smoke check
of the build entry point and the CPU-baseline leg of the benchmark use it.

It is a plain, slow, obviously-correct restatement of the method:

* ``tableau``    -- Butcher tableaus (Radau IIA, Gauss--Legendre) by collocation,
                    stability function, LDU factorisation of A_RK (Sec. 2, Sec. 3).
* ``operators``  -- finite-difference stiffness K (constant or face-averaged
                    variable kappa) and mass M = I; Q1 finite-element M and K.
* ``aao``        -- the all-at-once operator of Eq. (system_all_at_once_RK) with
                    the blocks Phi, Psi_1, Psi_2, Theta = I (x) Theta_hat, its
                    transpose, the right-hand side, and a dense Kronecker assembly.
* ``multigrid``  -- Galerkin geometric multigrid V-cycles for M + cK (stands in
                    for the closed HSL_MI20 AMG of Sec. 5).
* ``precond``    -- Rana's stage preconditioner (block LDU reading), inner GMRES
                    for Theta_tilde, the Schur approximation S_tilde of
                    Eq. (AppSchur), the block-triangular P_tilde of Eq. (AppPrec),
                    and their transposes.
* ``mgrit``      -- two-level multigrid reduction in time for S_tilde's time
                    recurrence (the parallel implementation of Sec. 5).
* ``fgmres``     -- restarted right-preconditioned flexible GMRES (Algorithm 1
                    with P_L = I, P_R = P_tilde), and Algorithm 1 with a left
                    (or split) preconditioner.
* ``sequential`` -- sequential RK time stepping with direct stage solves, its
                    adjoint, and forward substitution for any right-hand side.
* ``problems``   -- the paper's exact-solution test problem of Sec. 5.1 with Q1 or
                    Q2 elements (Table 2's DoF, time grids and errors).
* ``adjoint``    -- the adjoint solve and gradients of the tracking functional.
* ``spectral``   -- the exact all-at-once solution for constant-coefficient finite
                    differences, mode by mode in the sine basis (any size).
* ``relaxed``    -- FGMRES with an iteration-dependent (relaxed) product precision:
                    an inexact product accepted while its error bound stays below
                    the inexact-Krylov allowance, which grows as the residual falls
                    (the paper's future-work direction), and the FP32 product with
                    its rigorous rounding bound.
* ``lowprec``    -- P_tilde with its stored vectors rounded to FP32, BF16 or FP16
                    (per-row power-of-two scales) and FP32 arithmetic, the storage
                    emulation of Sec. 4--5 (the paper simulates it with chop).

Parity status per function is stated in each module header.
"""
