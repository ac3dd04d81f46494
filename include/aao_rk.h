/*
 * aao_rk.h -- C ABI of the GB300 all-at-once Runge--Kutta heat-equation solver.
 *
 * The problem (Sec. 2, Eq. heat_equation): v_t - div(kappa grad v) = f on a
 * box Omega in R^d (d = 2, 3), v = 0 on the boundary, v(0) = u0.  An s-stage
 * RK method with tableau (A_RK, b, c) and step tau = T / nt, and a vertex-grid
 * finite-difference (M = I) or Q1 discretisation in space, give the
 * all-at-once system of Eq. (system_all_at_once_RK)
 *
 *     [ Phi    Psi_1 ] [ v ]   [ b ]
 *     [ Psi_2  Theta ] [ V ] = [ f ],
 *
 * solved by restarted flexible GMRES in FP64 (Algorithm 1, P_L = I, or P_R = I) with the
 * block-triangular preconditioner P_tilde of Eq. (AppPrec): Theta_tilde by
 * inner GMRES on Theta_hat preconditioned by Rana's stage sweep (block LDU of
 * A_RK) with multigrid V-cycles for M + tau d_i K, and the Schur approximation
 * S_tilde of Eq. (AppSchur) by forward substitution in time (Sec. 3, Fig. 1).
 *
 * Vector layout (every FP64 vector of length n_st): x = [v_0 .. v_nt ; V_0 ..
 * V_{nt-1}], V_n = [V_{n,1} .. V_{n,s}], every block n_x = prod(n) values in
 * lexicographic order with x fastest.  n_st = n_x (nt + 1 + s nt).
 *
 * Memory: unless stated otherwise a `const double*` / `double*` vector
 * argument may be DEVICE memory (used in place, asynchronously on the
 * handle's stream) or HOST memory (the call then copies through the handle's
 * workspace and returns after the result is back on the host).  The caller
 * owns every pointer it passes; the library never frees them.  A handle owns
 * all of its device workspace and frees it in aao_rk_destroy.  Handles are
 * not thread-safe; calls on one handle are ordered on its stream.
 *
 * Errors: every call returns an aao_status; the text of the last error of the
 * calling thread is returned by aao_rk_last_error().  No call aborts or traps.
 *
 * Profiling and debugging: host NVTX ranges name the phases (aao.fgmres,
 * aao.outer_iteration, aao.orthogonalize, aao.matvec, aao.precond.theta_phase,
 * aao.precond.schur_sweep and the transposed pair) for profilers that record
 * NVTX; aao_rk_profile_begin/end time the launches of chosen kernels.  With
 * the environment variable AAO_POISON_WORKSPACE set (not "0") every device
 * allocation of a handle starts filled with 0xFF bytes (NaN), so a read of
 * workspace before its first write shows in the results.
 */
#ifndef AAO_RK_H
#define AAO_RK_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aao_rk_handle_s* aao_rk_handle;

typedef enum {
    AAO_OK = 0,
    AAO_ERR_ARG = -1,            /* invalid argument (sizes, tableau, options) */
    AAO_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    AAO_ERR_OOM = -3,            /* device allocation failed */
    AAO_ERR_NOT_CONVERGED = -4,  /* maxit reached; x holds the last iterate */
    AAO_ERR_BREAKDOWN = -5,      /* zero pivot in A_RK's LDU or in a Hessenberg solve */
    AAO_ERR_NONFINITE = -6,      /* a residual or Krylov coefficient became NaN/Inf */
    AAO_ERR_TIMEOUT = -7,        /* a bounded device-side wait ran out */
    AAO_ERR_UNSUPPORTED = -8     /* a valid request this build does not implement */
} aao_status;

/* Storage precision of the vectors inside P_tilde (Sec. 4, approaches A1--A5). */
typedef enum { AAO_FP64 = 0, AAO_FP32 = 1, AAO_BF16 = 2, AAO_FP16 = 3 } aao_prec;

typedef enum { AAO_DISC_FD = 0, AAO_DISC_Q1 = 1 } aao_disc;

/* Spatial grid (Sec. 2): vertex grid, interior nodes x_i = i h_a, i = 1..n[a],
 * h_a = len[a] / (n[a] + 1).  kappa: NULL for kappa = 1, else prod(n[a] + 2)
 * nodal values including the boundary nodes (x fastest), host or device; it
 * is copied at set-up.  Variable kappa is defined for disc = AAO_DISC_FD. */
typedef struct {
    int dim;
    int n[3];
    double len[3];
    int disc;
    const double* kappa;
} aao_grid;

/* Butcher tableau (Sec. 2): s <= 8 stages, A row-major s x s (leading
 * dimension s), weights b, nodes c.  A must admit an LDU factorisation
 * without pivoting with positive pivots (true for Radau IIA and Gauss). */
typedef struct {
    int s;
    double A[64];
    double b[8];
    double c[8];
} aao_tableau;

/* Solver options.  Defaults (aao_rk_default_options) follow Sec. 5: restart
 * 20, tol 1e-8, maxit 100, 3 V-cycles, 20 Chebyshev steps; inner GMRES maxit /
 * tol 5 / 1e-6 for an FP64 preconditioner and 3 / 1e-3 otherwise (Sec. 5.2). */
typedef struct {
    double tol;          /* outer: ||b - A x|| <= tol ||b|| (true residual) */
    int restart;         /* outer FGMRES restart length, 1..64 */
    int maxit;           /* outer iteration cap */
    int inner_maxit;     /* inner GMRES iterations per Theta_tilde solve, 1..16; 0 = default */
    double inner_tol;    /* inner early exit |g_{k+1}| <= inner_tol ||r||; < 0 = default */
    int mg_cycles;       /* V-cycles per shifted solve */
    int mg_pre, mg_post; /* damped-Jacobi sweeps before / after the coarse correction */
    double mg_omega;     /* Jacobi damping */
    int cheb_steps;      /* Chebyshev steps for M^{-1} (Q1) */
    int prec_P;          /* aao_prec of Theta_tilde's GMRES and the S_tilde recurrence */
    int prec_Pint;       /* aao_prec of Rana's sweep, the V-cycles and coarse stencils */
    int ckpt_every;      /* must be 0 (else AAO_ERR_UNSUPPORTED): a checkpointed kappa gradient is
                          * summed by the caller over windows of steps recomputed from kept
                          * states, one aao_rk_grad_kappa(accumulate = 1) call per window */
    void* stream;        /* cudaStream_t for every call on the handle; NULL = default stream */
    int mgrit_m;         /* S_tilde's time recurrence: 0 = forward substitution (Eq. AppSchur);
                          * 2 <= m <= nt = one two-level MGRIT iteration with coarsening factor m
                          * and F-relaxation, the coarse step being the same substitution step with
                          * step size m tau (the parallel implementation of Sec. 5).  C-points are
                          * the multiples of m; where m does not divide nt the steps after the last
                          * C-point form a shorter final interval relaxed from it.  P_tilde^T runs
                          * it on the backward recurrence in reversed time */
    int precond_side;    /* 0: right preconditioning, FGMRES with P_R = P_tilde (Algorithm 1 with
                          * P_L = I; the sequential runs of Sec. 5.1); 1: left preconditioning,
                          * P_L = P_tilde and P_R = I (Algorithm 1; the parallel runs of Sec. 5.2),
                          * converged when ||P^{-1} b - P^{-1} A x|| <= tol ||P^{-1} b||, with
                          * rel_res still the true ||b - A x|| / ||b|| */
    double relax_matvec; /* ell >= 0: iteration-dependent precision of the outer product A z_k (the
                          * future-work direction of the paper's introduction, after the inexact-Krylov
                          * bound of Simoncini and Szyld).  0 = every product in FP64.  ell > 0:
                          * iteration k of a cycle first forms A z_k in FP32 with the a-posteriori bound
                          * gamma_32 || |A| |z_k| || on its error, and keeps it when the bound is at most
                          * ell tol ||b|| / (restart |g_k|), |g_k| the current least-squares residual;
                          * else it recomputes A z_k in FP64.  The stopping test stays on the true FP64
                          * residual.  Finite differences with right preconditioning only (else
                          * AAO_ERR_UNSUPPORTED); may be changed by aao_rk_set_options */
} aao_options;

typedef struct {
    int outer_its;             /* FGMRES iterations */
    long long inner_its_total; /* inner GMRES iterations summed over all Theta_tilde solves */
    double rel_res;            /* final true ||b - A x|| / ||b|| */
    int converged;
    double t_theta_ms;         /* time in the Theta_tilde phase of P_tilde applies */
    double t_schur_ms;         /* time in the S_tilde phase of P_tilde applies */
    double t_total_ms;         /* wall time of the call */
    int n_history;
    double history[128];       /* FGMRES least-squares residual / ||b|| per iteration */
    int relaxed_matvecs;       /* outer iterations whose product A z_k was kept in FP32 (relax_matvec) */
} aao_info;

void aao_rk_default_options(aao_options* opts);

/* Build a handle for one problem: operators, Rana shifts tau d_i from the
 * LDU of A_RK (Sec. 3), one multigrid hierarchy per shift with Galerkin
 * coarse stencils, and all workspace.  nt is at most 65534 (time blocks are a
 * launch grid dimension).  Returns AAO_ERR_ARG on bad sizes,
 * AAO_ERR_BREAKDOWN on a non-positive LDU pivot, AAO_ERR_OOM when the
 * workspace does not fit. */
aao_status aao_rk_setup(const aao_grid* grid, double tau, int nt, const aao_tableau* tab,
                        const aao_options* opts, aao_rk_handle* out);
void aao_rk_destroy(aao_rk_handle h);
const char* aao_rk_last_error(void);
/* Number of kernels this library has launched in the process so far (all
 * handles); the difference across a call counts that call's launches. */
long long aao_rk_launch_count(void);
/* Launch profiling (measurement aid, not thread-safe): between begin and end,
 * every launch of a kernel whose name contains kernel_name is bracketed by
 * CUDA events on its stream and credited with the algorithmic bytes its launch
 * site declares (compulsory reads and writes of that launch).  end()
 * synchronises the device and returns the number of such launches, their
 * summed event time and their summed algorithmic bytes. */
aao_status aao_rk_profile_begin(const char* kernel_name);
aao_status aao_rk_profile_end(long long* launches, double* total_ms, double* total_bytes);
/* Per-kernel breakdown of the last completed profile, one line per kernel:
 * "<mangled name>\t<launches>\t<event ms>\t<algorithmic bytes>\n".  The text stays
 * valid until the next aao_rk_profile_end. */
const char* aao_rk_profile_report(void);

/* n_x = prod(n), n_st = n_x (nt + 1 + s nt). */
aao_status aao_rk_sizes(aao_rk_handle h, long long* n_x, long long* n_st);
/* Replace tol / restart / maxit / inner_tol (precisions, multigrid shape,
 * inner_maxit, mgrit_m, precond_side and the stream are fixed at set-up;
 * changing them returns AAO_ERR_ARG). */
aao_status aao_rk_set_options(aao_rk_handle h, const aao_options* opts);

/* rhs = [M u0 ; 0 .. 0 ; M f_{n,i}] (Sec. 2 with zero Dirichlet data).  f has
 * n_x values (constant in time, f_time_dep = 0) or nt*s*n_x values at the
 * stage times t_n + c_i tau (f_time_dep = 1); u0 has n_x values. */
aao_status aao_rk_rhs(aao_rk_handle h, const double* f, int f_time_dep, const double* u0,
                      double* rhs);

/* y = A x and y = A^T x in FP64 (Eq. system_all_at_once_RK), n_st each. */
aao_status aao_rk_matvec(aao_rk_handle h, const double* x, double* y);
/* The FP32 product of the relaxed outer iteration (aao_options.relax_matvec; the paper's
 * future-work direction of an iteration-dependent matvec precision): y = fl32(A x) (transpose:
 * A^T x) with x and every coefficient rounded to FP32 and FP32 arithmetic, and absy = the same
 * expression over absolute coefficients and inputs, so that |y - A x| <= gamma_32 absy entry by
 * entry (gamma_d = d u / (1 - d u), u = 2^-24).  Finite differences only (else
 * AAO_ERR_UNSUPPORTED); x, y, absy are DEVICE arrays of n_st values (else AAO_ERR_ARG). */
aao_status aao_rk_matvec_relaxed(aao_rk_handle h, const double* x, double* y, double* absy, int transpose);
aao_status aao_rk_matvec_transpose(aao_rk_handle h, const double* x, double* y);

/* z = P_tilde^{-1} r (Eq. AppPrec, AppSchur) in the handle's precisions;
 * r and z are FP64, n_st each, and must not alias. */
aao_status aao_rk_precond_apply(aao_rk_handle h, const double* r, double* z);
/* z = P_tilde^{-T} r: backward substitution with S_tilde^T, then
 * Theta_tilde^{-T} (inner GMRES on Theta_hat^T with the backward stage sweep). */
aao_status aao_rk_precond_apply_transpose(aao_rk_handle h, const double* r, double* z);

/* Solve A x = rhs(f, u0) by FGMRES + P_tilde (Algorithm 1).  x (n_st) is the
 * initial guess when x0_given != 0, else ignored; it returns the solution.
 * info may be NULL.  Returns AAO_ERR_NOT_CONVERGED when maxit is reached. */
aao_status aao_rk_solve(aao_rk_handle h, const double* f, int f_time_dep, const double* u0,
                        double* x, int x0_given, aao_info* info);
/* Same with an explicit right-hand side vector of length n_st. */
aao_status aao_rk_solve_rhs(aao_rk_handle h, const double* rhs, double* x, int x0_given,
                            aao_info* info);

/* Adjoint (transposed all-at-once system, solved backward in time):
 * A^T lambda = dJdx by FGMRES preconditioned with P_tilde^T; then, for the
 * constant-in-time source of aao_rk_solve, grad_f = sum_{n,i} M^T lambda_{V,n,i}
 * (n_x values, may be NULL) and grad_kappa_m = -sum_{n,i} lambda_{V,n,i}^T
 * (dK/dkappa_m) W_{n,i}, W_{n,i} = v_n + tau sum_j a_ij V_{n,j}, over the
 * prod(n+2) nodal kappa values (may be NULL; FD only).  x_fwd is the forward
 * solution (n_st).  The source's own regulariser is the caller's to add. */
aao_status aao_rk_adjoint_solve(aao_rk_handle h, const double* dJdx, double* lambda,
                                const double* x_fwd, double* grad_f, double* grad_kappa,
                                aao_info* info);

/* grad_kappa (+)= -sum_{n,i} lambda_{V,n,i}^T (dK/dkappa) W_{n,i} over this handle's
 * nt steps (FD only; device vectors of n_st, n_st and prod(n+2) values).  With
 * accumulate != 0 the result is added to grad_kappa: a gradient over a long
 * horizon can be summed window by window from forward states recomputed from
 * checkpoints (each window a handle with nt = window length). */
aao_status aao_rk_grad_kappa(aao_rk_handle h, const double* lambda, const double* x_fwd, double* grad_kappa,
                             int accumulate);

/* Solve nprob independent problems (each with its own handle, possibly of a
 * different grid, nt and s) in one call.  f[p], u0[p], x[p] as in
 * aao_rk_solve (device memory); infos may be NULL.  Returns the first
 * non-OK status, after every problem has been attempted.  Problems run on up
 * to 64 host threads, largest (space-time unknowns) first; each handle may
 * appear once.  nprob == 0 is a no-op returning AAO_OK; nprob < 0, NULL
 * arrays, a NULL or repeated handle, or an open launch profile
 * (aao_rk_profile_begin) give AAO_ERR_ARG before any device work. */
aao_status aao_rk_solve_batched(int nprob, const aao_rk_handle* hs, const double* const* f,
                                const double* const* u0, double* const* x, aao_info* infos);

/* ---- component entry points (each one piece of P_tilde, FP64 in and out) ---- */

/* x ~= (M + tau d_stage K)^{-1} b by mg_cycles V-cycles from x = 0 (n_x). */
aao_status aao_rk_shifted_solve(aao_rk_handle h, int stage, const double* b, double* x);
/* y = P_int^{-1} r (s n_x), Rana's forward stage sweep (transpose != 0: backward sweep with P_int^T). */
aao_status aao_rk_pint_apply(aao_rk_handle h, const double* r, double* y, int transpose);
/* z_n = Theta_tilde^{-1} r_n for nblocks independent blocks of s n_x values
 * (inner GMRES); its (may be NULL) receives the iterations per block. */
aao_status aao_rk_inner_solve(aao_rk_handle h, int nblocks, const double* r, double* z, int* its);

/* ---- allocation-free variant (no counterpart in the paper) ----
 *
 * x ~= (I + c K)^{-1} b on the constant-coefficient FD grid `grid` by `cycles`
 * V(pre, post)-cycles with Jacobi weight omega, the same multigrid as the
 * handle's shifted solves, computed in FP64.  For callers that cannot allocate
 * device memory (pools that forbid cudaMalloc, hosts that only hand out
 * pre-registered buffers, code that must not allocate after start-up): it
 * needs no handle and calls no allocating routine.  All scratch lives in one
 * fixed 5 MiB device array inside the library, which every GPU that loads the
 * library keeps until the process exits; grids above 65536 points (or whose
 * coarsest level exceeds 256 points) are rejected with AAO_ERR_ARG, as are
 * lengths that are not finite and positive, and a c or omega that is not
 * finite.  b and x are device memory of the current device (n_x values; host
 * pointers and other GPUs' memory are rejected), the work is queued on
 * `stream` (NULL = default stream) and the call returns once it has finished:
 * it reads back the coarsest level's inversion flag and returns
 * AAO_ERR_BREAKDOWN if that operator is not positive definite.  The first call
 * on a device looks up the array's device address, so make it before any
 * stream capture; the address is kept for the process, so do not use this
 * entry point across a cudaDeviceReset.  Every call reuses the same array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  The scratch keeps the last call's contents;
 * each call rebuilds what it reads and clears the flag it reads back. */
aao_status aao_rk_shifted_solve_noalloc(const aao_grid* grid, double c, int cycles, int pre, int post,
                                        double omega, const double* b, double* x, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AAO_RK_H */
