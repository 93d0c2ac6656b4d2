/*
 * lindblad.h -- C ABI of the B300 (sm_103a) Lindblad steady-state / low-spectrum library.
 *
 * Method: Beugnot, Gregory, Robin, Tilloy, "Well-conditioned iterative methods for large
 * open quantum systems".  The Lindbladian L = S + K is split into the no-jump part
 * S(X) = G X + X G^dag, G = -iH - 1/2 sum_j L_j^dag L_j, and the jump part
 * K(X) = sum_j L_j X L_j^dag (Eqs. (2)-(3)).  S is inverted exactly by a Lyapunov solve
 * (App. A.1); Phi = -K S^{-1} is a CPTP map whose fixed point gives the steady state
 * (Theorem 1, Alg. 4), and the no-jump resolvent R_mu^S = (mu - S)^{-1} preconditions the
 * shift-invert solves of the low-lying spectrum (Sec. 3.1, Alg. 2, Alg. 5).
 *
 * Conventions common to every entry point
 *   - Matrices are dense complex128 (two doubles: re, im), row-major, C-contiguous,
 *     leading dimension n.  A stack of d matrices is d*n*n contiguous elements.
 *   - Every pointer argument named *_dev is a DEVICE pointer owned by the caller.
 *     The library never frees caller memory and allocates no device memory of its
 *     own: everything it keeps lives in the caller-provided workspace.  The exceptions
 *     are fixed and documented at their entry points: the 8 MiB scratch array of
 *     lindbladian_apply_noalloc belongs to the library module, and steady_state_batched
 *     creates (and releases) a private stream and a CUDA graph per call.
 *   - `stream` is a cudaStream_t passed as void*.  Calls are stream-ordered.  A call
 *     that returns solver results (steady_state, low_spectrum) synchronises the
 *     stream before returning, because its stopping test is read on the host once
 *     per restart.
 *   - Return value: lb_status.  Negative = no result; 0 = OK; positive = a usable
 *     result with a caveat (e.g. LB_NOT_CONVERGED returns the running best).
 *   - A handle must not be used from two streams at once.
 */
#ifndef LINDBLAD_H_
#define LINDBLAD_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LB_OK = 0,
    LB_NOT_CONVERGED = 1,      /* tolerance not met within the restart cap; best iterate returned */
    LB_S_SINGULAR = 2,         /* Theorem 1 case 1: G has an eigenvalue on iR, S is not invertible;
                                  steady_state returns the pure state |psi><psi| of that eigenvector */
    LB_ILL_CONDITIONED = 3,    /* eigenbasis route refused by the cond(U) gate; Schur route used */
    LB_INVALID_ARG = -1,
    LB_CUDA_ERROR = -2,        /* a CUDA call failed, or a bounded wait of a tensor-core kernel gave up
                                  during the call (every solver and apply entry point checks the
                                  device error word before returning; the result is then not valid) */
    LB_ETA_EXCLUDED = -3,      /* eta * Tr R_mu^S(I) == 1: the Sherman-Morrison preconditioner of
                                  Eq. ShermanMorr / Alg. 2 is undefined */
    LB_WORKSPACE_TOO_SMALL = -4,
    LB_NOT_IMPLEMENTED = -5,
    LB_SOLVER_ERROR = -6       /* a factorisation in set-up failed (info != 0), or the Schur form failed
                                  its backward-error gate (lb_opts.schur_tol) */
} lb_status;

typedef enum {
    LB_PREC_FP64 = 0,   /* every contraction in FP64 on the CUDA cores */
    LB_PREC_MIXED = 1   /* jump-term and Sylvester-update GEMMs on the tensor cores (tcgen05,
                           split-FP16 operands, FP32 accumulate); FP64 residual,
                           FP64 iterative refinement of the steady state */
} lb_precision;

typedef enum { LB_FORM_PHI = 0, LB_FORM_M = 1 } lb_form;   /* Phi = -K S^{-1}; M = -S^{-1} K */

/* phi_apply / jump_apply flags: form in bit 0; coordinates in bit 1; Hermitian input in bit 2 */
#define LB_APPLY_FORM_M   1   /* apply M instead of Phi */
#define LB_APPLY_SCHUR    2   /* X and Y are given in Schur coordinates X~ = Q^dag X Q */
#define LB_APPLY_HERMITIAN 4  /* X is Hermitian (the caller guarantees it): S^{-1} and K preserve Hermiticity
                                 (App. A.1.1), so the jump term's second product is formed on its upper
                                 tiles only and mirrored; the result is exactly Hermitian */

typedef struct {
    double tol;           /* stop when ||L(rho_hat)||_max < tol (absolute, hermitised trace-1 state);
                             default 1e-10 */
    int    krylov_m;      /* Arnoldi cycle length m (default 20) */
    int    max_restarts;  /* N of Alg. 4 / restart cap of Alg. 5 (default 60) */
    int    precision;     /* lb_precision (default LB_PREC_FP64) */
    double eta;           /* deflation coefficient eta (default 1) */
    int    max_refine;    /* mixed precision: refinement steps cap (default 8) */
    int    gmres_m;       /* inner GMRES cycle length (default 40) */
    int    sylv_block;    /* triangular Sylvester block size (default 0 = automatic) */
    double inner_tol;     /* shift-invert inner GMRES relative tolerance (default 1e-10); a solve also
                             stops when one restart cycle reduces its residual by less than 10% */
    int    keep_ritz;     /* p of Alg. 5: Ritz pairs kept at a thick restart (default 0 = auto) */
    int    route;         /* Lyapunov route of the FP64 path (lb_route, default LB_ROUTE_SCHUR); read at
                             set-up */
    double eig_cond_max;  /* cond(U) gate of the eigenbasis route (default 1e3): the route is used only if
                             ||R||_F ||R^{-1}||_F / n <= eig_cond_max, R = Q^dag U */
    double schur_tol;     /* set-up gate on the Schur form (default 1e-12): lindblad_setup fails with
                             LB_SOLVER_ERROR when ||strictly-lower(Q^dag G Q)||_F / ||G||_F exceeds it.  A
                             backward error e makes T the Schur factor of G + E, ||E||_F = e ||G||_F, and the
                             FP64 Phi path then stagnates near ||L rho||_max ~ 2 e ||G||_F ||rho||_2; the
                             refined (mixed) solves absorb it as a preconditioner error */
    int    recycle_k;     /* harmonic Ritz vectors kept by the recycled GMRES (App. A.2; default 8, 0 = plain
                             restarted GMRES); at most 16 and at most gmres_m - 2; read at set-up (workspace) */
    const double* gauge_c;/* nullable host array of d complex shifts (re, im pairs): the gauge of Remark
                             "Non-uniqueness of the decomposition", L~_j = L_j + c_j I and
                             H~ = H + (1/2i) sum_j (c_j^* L~_j - c_j L~_j^dag); read by lindblad_setup only.
                             L is unchanged; the split S~ + K~ (and so Phi, the preconditioners and the
                             Schur form) is that of (H~, L~).  NULL = the split of Eq. (2) */
    const int* batched_tiles; /* nullable host array of LB_TILE_BUCKETS entries: the complex64 GEMM tile
                             shape (0 .. LB_TILE_SHAPES-1, see lindblad_batched_tune) that steady_state_batched
                             uses for an instance of size n, indexed by min((n - 1) / 16, LB_TILE_BUCKETS - 1).
                             NULL = shape 0 (32 x 32) for every size */
} lb_opts;

#define LB_TILE_BUCKETS 16
#define LB_TILE_SHAPES 4

/* Lyapunov route: Bartels-Stewart on the Schur form (App. A.1.1), or the eigenbasis divide of Alg. 1
 * (App. A.1.2) in Schur coordinates, X = R[(R^{-1} Y R^{-dag}) o D]R^dag with D_ij = 1/(s_i + s_j^* - lam)
 * and G = Q T Q^dag = (Q R) diag(s) (Q R)^{-1}; AUTO takes the eigenbasis route when the gate passes. */
typedef enum { LB_ROUTE_SCHUR = 0, LB_ROUTE_EIG = 1, LB_ROUTE_AUTO = 2 } lb_route;

typedef struct {
    int    status;
    int    restarts;          /* Arnoldi cycles run */
    int    phi_applies;       /* Phi (or OP) applications */
    int    gmres_steps;       /* inner GMRES steps (refinement / shift-invert) */
    int    refine_steps;      /* mixed-precision refinement steps */
    double residual_max;      /* ||L(rho_hat)||_max of the returned state (FP64, original basis) */
    double residual_fro;      /* ||L(rho_hat)||_F */
    double ritz_value;        /* Ritz value of Phi selected at the end (steady_state) */
    double schur_backward_err;/* ||strictly-lower(Q^dag G Q)||_F / ||G||_F left out of T */
    double min_abs_re_T;      /* min_i |Re T_ii| (case-1 test of Theorem 1) */
    double setup_ms;          /* lindblad_setup wall time (host clock around the stream) */
    double solve_ms;          /* wall time of the call that filled this struct */
    double cond_eig;          /* ||R||_F ||R^{-1}||_F / n of the eigenbasis (0 if not computed) */
    int    route;             /* Lyapunov route in use (lb_route) */
} lb_info;

typedef struct lb_handle_s* lindblad_handle;

/* Fills *opts with the defaults listed above. */
void lb_default_opts(lb_opts* opts);

/* Device workspace, in bytes, that lindblad_setup needs for (n, d, opts).  Returns 0 for
 * invalid sizes.  The caller allocates it (e.g. a torch uint8 tensor) and keeps it alive
 * until lindblad_destroy. */
size_t lindblad_workspace_bytes(int n, int d, const lb_opts* opts);

/* Set-up, once per Lindbladian (Sec. 1.2 Eq. (3); App. A.1).
 *   H_dev : n x n Hermitian Hamiltonian (device, complex128, row-major)
 *   L_dev : d stacked n x n jump operators (device, d*n*n complex128)
 * Copies H and L into the workspace (with opts->gauge_c, replaced on the device by the gauge-shifted
 * L~_j = L_j + c_j I and H~ = H + (1/2i) sum_j (c_j^* L~_j - c_j L~_j^dag), Remark "Non-uniqueness of
 * the decomposition"; every later call then uses that split), forms G = -iH - 1/2 sum_j L_j^dag L_j with one
 * stacked GEMM, computes the Schur form G = Q T Q^dag (eigenvectors -> QR -> upper
 * triangle of Q^dag G Q), the Schur-coordinate jump operators L~_j = Q^dag L_j Q and the
 * case-1 test of Theorem 1.  With opts->route != LB_ROUTE_SCHUR it also keeps R = Q^dag U and
 * R^{-1} for the eigenbasis route and applies the cond(U) gate.  On success *out receives a handle.
 * Returns LB_OK, or LB_ILL_CONDITIONED (handle valid, Schur route in use) when LB_ROUTE_EIG was
 * requested and the gate refused it.  Errors: LB_INVALID_ARG (n < 2, d < 1, null pointers, a NaN or
 * Inf entry in H or L_j -- checked on the device before any factorisation),
 * LB_WORKSPACE_TOO_SMALL, LB_SOLVER_ERROR (a factorisation failed, or the Schur backward error
 * exceeds opts->schur_tol; info->schur_backward_err then carries the measured value and no handle
 * is returned), LB_CUDA_ERROR.  info (nullable) receives set-up diagnostics. */
lb_status lindblad_setup(const void* H_dev, const void* L_dev, int n, int d,
                         void* workspace_dev, size_t workspace_bytes, void* stream,
                         const lb_opts* opts, lindblad_handle* out, lb_info* info);

/* Y = Phi(X) = -K(S^{-1} X)  (Theorem 1, the map iterated by Alg. 4), or, with
 * LB_APPLY_FORM_M, Y = M(X) = -S^{-1}(K X) (proof of Theorem 1).  X_dev, Y_dev: n x n
 * device complex128; X is not modified; X and Y must not alias.  With LB_APPLY_SCHUR
 * both are in Schur coordinates (what the Arnoldi loop iterates), otherwise in the
 * original basis.  precision: lb_precision.  Errors: LB_INVALID_ARG, LB_S_SINGULAR
 * (case 1: S not invertible), LB_CUDA_ERROR. */
lb_status phi_apply(lindblad_handle h, const void* X_dev, void* Y_dev, int flags,
                    int precision, void* stream);

/* Y = K(X) = sum_j L_j X L_j^dag, the jump part of Eq. (2) (the dominant contraction of every Phi
 * application).  With LB_APPLY_SCHUR, X and Y are in Schur coordinates and L~_j = Q^dag L_j Q is
 * used.  precision: LB_PREC_FP64 (CUDA-core FP64) or LB_PREC_MIXED (tcgen05 split-FP16 GEMMs,
 * FP32 accumulation).  X_dev, Y_dev: n x n device complex128, must not alias. */
lb_status jump_apply(lindblad_handle h, const void* X_dev, void* Y_dev, int flags, int precision,
                     void* stream);

/* X = R_lam^S(Y) = (lam - S)^{-1}(Y), the no-jump resolvent (Sec. 3.1), by Bartels-Stewart
 * on the stored Schur form with T -> T - lam/2 I (App. A.1.1).  lam = 0 gives -S^{-1}.
 * Original-basis device operands.  Errors as phi_apply. */
lb_status resolvent_apply(lindblad_handle h, const void* Y_dev, void* X_dev, double lam,
                          int precision, void* stream);

/* R = L(X) = G X + X G^dag + sum_j L_j X L_j^dag in FP64, original basis (Eq. (1)). */
lb_status lindbladian_apply(lindblad_handle h, const void* X_dev, void* R_dev, void* stream);

/* Steady state by Phi-Arnoldi (Alg. 4): explicitly restarted Arnoldi on Phi in Schur
 * coordinates, Ritz value nearest 1, rho = -S^{-1} xi, hermitise + trace-normalise, stop when
 * ||L(rho_hat)||_max < opts->tol (FP64, original basis).  With LB_PREC_MIXED the cycles run
 * on tensor-core GEMMs and the state is then refined in FP64 (residual-correction steps,
 * each a right-preconditioned GMRES solve of L~_eta delta = -r, Alg. 2/3).
 *   rho_dev : n x n device output (Hermitian, trace 1).
 * Returns LB_OK, LB_NOT_CONVERGED (best state returned), LB_S_SINGULAR (pure steady state of
 * Theorem 1 case 1 returned), or an error. */
lb_status steady_state(lindblad_handle h, void* rho_dev, const lb_opts* opts, lb_info* info,
                       void* stream);

/* Steady state as a preconditioned linear solve (Alg. 3, Sec. 4.1): L~_eta rho = eta I with
 * L~_eta(rho) = L(rho) + eta Tr(rho) I (Eq. steady_state_linear_problem), by GMRES right-preconditioned
 * with P_0 = Precond(., 0, eta) (Alg. 2, Eq. ShermanMorr) and Krylov subspace recycling (App. A.2:
 * opts->recycle_k harmonic Ritz vectors kept across restarts), warm start |0><0|.  After every
 * GMRES cycle (FP64) the iterate is hermitised and trace-normalised and the solve stops when
 * ||L(rho_hat)||_max < opts->tol.  With LB_PREC_MIXED the GMRES cycles run on the tensor cores and
 * each correction is checked against the FP64 residual (residual-correction refinement).
 *   rho_dev : n x n device output (Hermitian, trace 1): the best iterate.
 * Cycle length opts->gmres_m; at most opts->max_restarts corrections (FP64) or opts->max_refine + 4
 * (mixed).  info: restarts = GMRES cycles, gmres_steps = phi_applies = preconditioned operator
 * applications (one Lyapunov solve + one jump term each), refine_steps = FP64 residual corrections.
 * Returns LB_OK, LB_NOT_CONVERGED (best state returned), LB_S_SINGULAR (case 1 of Theorem 1: S not
 * invertible, no result), LB_ETA_EXCLUDED, LB_INVALID_ARG, LB_CUDA_ERROR. */
lb_status steady_state_gmres(lindblad_handle h, void* rho_dev, const lb_opts* opts, lb_info* info, void* stream);

/* Resolvent of the Lindbladian (Corollary "Resolvent of the Lindbladian"; the benchmark of Sec. 3.4):
 * X = R_lam^L(B) = (lam - L)^{-1}(B) for lam > 0, by recycled GMRES right-preconditioned with the
 * no-jump resolvent R_lam^S ((lam - L) R_lam^S = Id - K R_lam^S, Theorem 2: a strict contraction, so
 * the inner solve converges geometrically).  The iterate is hermitised when B is Hermitian and
 * rescaled to its exact trace Tr B / lam; the solve stops when ||(lam - L)(X) - B||_max < opts->tol.
 *   B_dev, X_dev : n x n device complex128 (must not alias).  X is written (no warm start).
 * The recycled subspace is kept in the handle for later solves at the same lam and precision.
 * Returns LB_OK, LB_NOT_CONVERGED (last iterate returned), LB_INVALID_ARG (lam <= 0, null or aliased
 * pointers, a NaN or Inf entry in B), LB_NOT_IMPLEMENTED, LB_CUDA_ERROR. */
lb_status resolvent_solve(lindblad_handle h, double lam, const void* B_dev, void* X_dev, const lb_opts* opts,
                          lb_info* info, void* stream);

/* Implicit Euler time stepping (Eq. resolvent, Sec. 4.3): rho_{k+1} = (Id - dt L)^{-1} rho_k
 * = (1/dt) R_{1/dt}^L rho_k for nsteps steps, each a resolvent solve at lam = 1/dt preconditioned by
 * R_{1/dt}^S (Theorem 2 applies: lam > 0), warm-started from rho_k, with the recycled subspace carried
 * from step to step.  A step stops when ||(1/dt - L)(rho_{k+1}) - rho_k / dt||_max < opts->tol
 * ||rho_k / dt||_max (rho_{k+1} hermitised for Hermitian rho0, trace = Tr rho_k).
 *   rho0_dev : n x n device initial state; rho_dev : n x n device final state (must differ);
 *   traj_dev : nullable, nsteps stacked n x n device states after each step.
 * info: residual_max = the largest relative step residual, gmres_steps / phi_applies / restarts summed.
 * Returns LB_OK, LB_NOT_CONVERGED (a step missed the tolerance; the trajectory continues),
 * LB_INVALID_ARG (dt <= 0, nsteps < 1, a NaN or Inf entry in rho0), LB_NOT_IMPLEMENTED, LB_CUDA_ERROR. */
lb_status implicit_euler(lindblad_handle h, const void* rho0_dev, double dt, int nsteps, void* rho_dev,
                         void* traj_dev, const lb_opts* opts, lb_info* info, void* stream);

/* The k smallest-|lambda| nonzero eigenvalues of L by shift-invert Arnoldi on
 * (mu - L~_eta)^{-1} (Alg. 5), each application a GMRES solve right-preconditioned by
 * Precond(., mu, eta) (Alg. 2), recycled across cycles and across applications (App. A.2); every inner
 * solve's true residual is checked with one explicit application of (mu - L~_eta), and a recycled pair
 * that disagrees with it is dropped.  Thick (Krylov-Schur) restarts keep opts->keep_ritz pairs;
 * stop when max_k ||L v_k - lambda_k v_k||_max / ||v_k||_max < opts->tol.  With LB_PREC_MIXED the inner
 * solves run on the tensor cores while the eigen-residual falls (to 1e-6 or until it stops halving),
 * then the outer iteration restarts explicitly in FP64 from the sum of the k wanted Schur vectors.
 *   evals_host : k complex128 (host memory), sorted by |lambda|, then Re descending.
 *   evecs_dev  : nullable; k stacked n x n device eigenvectors (raw, traceless).
 * Errors: LB_INVALID_ARG (k < 1 or k > m - 2), LB_ETA_EXCLUDED, LB_S_SINGULAR (mu = 0 with
 * S singular: no result is produced, choose mu > 0), LB_NOT_CONVERGED (best estimates returned). */
lb_status low_spectrum(lindblad_handle h, int k, double mu, double eta, void* evals_host,
                       void* evecs_dev, const lb_opts* opts, lb_info* info, void* stream);

/* Adjoint of the steady-state solve, for implicit differentiation (Remark "Differentiating the
 * steady state").  Given the steady state rho (from steady_state) and a Hermitian observable O,
 * solves L~_eta^* w = O (L~_eta^*(w) = G^dag w + w G + sum_j L_j^dag w L_j + eta Tr(w) I) by GMRES
 * right-preconditioned with the adjoint no-jump resolvent (Schur coordinates, reversed-index
 * triangular solve), refined against the FP64 adjoint residual until ||.||_max < opts->tol.
 * Outputs (device, complex128, row-major): w (n x n); gH (n x n, nullable) and gL (d x n x n,
 * nullable), the sensitivities of J = Tr(O rho) with dJ = Re<gH, dH> + sum_j Re<gL_j, dL_j>,
 * <A, B> = Tr(A^dag B):  gH = i (rho w - w rho),  gL_j = -Ws L_j rho + 1/2 L_j (Ws rho + rho Ws),
 * Ws = w + w^dag.  With a gauge set at set-up, gH and gL are the sensitivities with respect to H~ and
 * L~_j taken as independent inputs.  FP64 throughout.  Errors: LB_INVALID_ARG, LB_S_SINGULAR (case 1),
 * LB_NOT_CONVERGED (best w and sensitivities returned). */
lb_status steady_state_adjoint(lindblad_handle h, const void* rho_dev, const void* O_dev, void* w_dev,
                               void* gH_dev, void* gL_dev, const lb_opts* opts, lb_info* info,
                               void* stream);

/* Batched steady states of `count` independent Lindbladians of uneven size sharing the number of
 * jumps d (a parameter sweep), each by Alg. 4 with complex64 contractions and an FP64 anchor, all
 * instances in one set-up launch and one persistent solve launch (a work queue taken in
 * decreasing n), replayed as one CUDA graph on a private stream ordered after `stream`.
 * Per instance: G = -iH - 1/2 sum_j L_j^dag L_j and its complex Schur form G = Q T Q^dag
 * computed on the device in FP64 (Householder-Hessenberg + shifted QR); Phi-Arnoldi cycles of
 * length opts->krylov_m (clipped to [8, 32]) that carry the 5 Schur vectors next nearest 1 across
 * a restart, first in complex64 while the Ritz residual falls, then anchored in FP64: the iterate
 * rho~ = S~^{-1} xi and its image Phi(S~ rho~) = -K~ rho~ are formed in FP64 and every complex64
 * basis vector is used exactly orthogonal to it, so rounding only touches the correction; at
 * most opts->max_restarts cycles per phase, until ||L(rho)||_max < opts->tol in the original
 * basis.  opts->precision, eta and the GMRES / refinement fields are not used.
 *   n        : host array of count sizes, each 2 <= n_i <= 256.
 *   H_dev    : the count Hamiltonians packed back to back (device, complex128, row-major,
 *              instance i at offset sum_{k<i} n_k^2 elements).
 *   L_dev    : the jumps, instance i's d stacked n_i x n_i matrices at offset d sum_{k<i} n_k^2.
 *   rho_dev  : output, packed like H_dev (Hermitian, trace 1; written for every instance whose
 *              set-up status is LB_OK; untouched otherwise).
 *   workspace: device memory of at least lindblad_batched_workspace_bytes(count, n, d, opts)
 *              bytes, 256-byte aligned, owned by the caller; nothing in it needs to be zero.
 *   infos    : nullable host array of count lb_info (status, residual_max, residual_fro of the
 *              last original-basis residual, phi_applies = complex64 Phi applications,
 *              restarts = cycles, refine_steps = FP64-anchored cycles, solve_ms = wall time of
 *              the batch).
 * Synchronises `stream` before returning.  Returns LB_INVALID_ARG (count < 1, d < 1, a size out
 * of range, a null pointer), LB_WORKSPACE_TOO_SMALL, LB_CUDA_ERROR, else the first negative
 * per-instance status (LB_SOLVER_ERROR: the Schur QR iteration stalled), else the first positive
 * one (LB_NOT_CONVERGED; LB_S_SINGULAR for Theorem 1 case 1, reported without solving), else
 * LB_OK. */
size_t lindblad_batched_workspace_bytes(int count, const int* n, int d, const lb_opts* opts);
lb_status steady_state_batched(int count, const int* n, int d, const void* H_dev, const void* L_dev,
                               void* rho_dev, void* workspace, size_t ws_bytes, const lb_opts* opts,
                               lb_info* infos, void* stream);

/* Tile autotuner of the batched engine (the per-instance complex64 GEMMs of the jump term).  For each of
 * the LB_TILE_BUCKETS size buckets (n in (16 b, 16 (b + 1)], the last one open-ended; timed at
 * n = min(16 (b + 1), nmax)) and each of the LB_TILE_SHAPES tile shapes -- 0: 32 x 32 output tile, K step
 * 32, 4 x 1 register tile per thread; 1: 64 x 32, K 16, 4 x 2; 2: 64 x 64, K 16, 4 x 4; 3: 32 x 64, K 16,
 * 2 x 4 -- it times the jump term y = -sum_j L_j Z L_j^dag exactly as the batched solve forms it, one
 * synthetic instance per SM side by side (CUDA events on `stream`), and picks the fastest shape.
 *   workspace : device memory of at least lindblad_batched_tune_workspace_bytes(d, nmax) bytes.
 *   tiles_out : host array of LB_TILE_BUCKETS shapes, for lb_opts.batched_tiles.
 *   us_out    : nullable host array of LB_TILE_BUCKETS x LB_TILE_SHAPES times (microseconds per jump
 *               term per instance, bucket-major).
 * Synchronises `stream`.  Errors: LB_INVALID_ARG (d < 1, nmax outside [2, 256], null workspace or
 * tiles_out), LB_WORKSPACE_TOO_SMALL, LB_CUDA_ERROR.  0 bytes for invalid arguments. */
size_t lindblad_batched_tune_workspace_bytes(int d, int nmax);
lb_status lindblad_batched_tune(int d, int nmax, void* workspace, size_t workspace_bytes, int* tiles_out,
                                float* us_out, void* stream);

/* Largest n accepted by lindbladian_apply_noalloc (its scratch is sized for it). */
#define LB_NOALLOC_NMAX 512

/* R = L(X) = G X + X G^dag + sum_j L_j X L_j^dag in FP64, original basis, straight from H and
 * the jumps: the same result as lindbladian_apply (up to rounding order) but with no handle, no
 * caller workspace and no device allocation of any kind.  The paper has no counterpart: this is
 * plumbing for callers that must not allocate -- a residual monitor inside a latency-bound
 * loop, where cudaMalloc would synchronise the device and stall the other streams, or a process
 * that has already handed all device memory to its own buffers and holds no set-up workspace.
 *   H_dev : n x n Hamiltonian; L_dev : d stacked n x n jumps; X_dev : n x n input; R_dev : n x n
 *           output (all device, complex128, row-major; R must not alias the inputs).
 * Scratch: two n x n complex128 matrices in a file-scope device array of
 * 2 * LB_NOALLOC_NMAX^2 * 16 bytes (8 MiB) that belongs to the library module; every scratch
 * element is written before it is read, so nothing has to start at zero.  The first call on
 * each device looks the array up with cudaGetSymbolAddress (which may load the module); make
 * that first call before any stream capture is begun.  Calls on one device share the array:
 * calls that overlap in time (other streams, other host threads) race, so serialise them.
 * Stream-ordered, no host synchronisation.  Errors: LB_INVALID_ARG (null pointer, n < 2,
 * d < 1), LB_WORKSPACE_TOO_SMALL (n > LB_NOALLOC_NMAX), LB_CUDA_ERROR. */
lb_status lindbladian_apply_noalloc(const void* H_dev, const void* L_dev, int n, int d, const void* X_dev,
                                    void* R_dev, void* stream);

/* Kernel timing (diagnostics, no effect on results).  While enabled, the library records CUDA
 * events on the launching stream around every tensor-core GEMM launch (kernel id 0) and every
 * FP64 GEMM launch of the residual (kernel id 1).  lb_kernel_stats synchronises the stream and
 * returns the launch count, the summed event time in ms and the summed algorithmic flops
 * (8 real flops per complex multiply-add) since the last lb_set_profiling call. */
lb_status lb_set_profiling(lindblad_handle h, int enable);
lb_status lb_kernel_stats(lindblad_handle h, int kernel, int* launches, double* total_ms,
                          double* algorithmic_flops);

/* Test of the bounded waits (failure handling; no effect unless called).  Every mbarrier wait of
 * the handle's tensor-core kernels gives up after wait_ms (0 < wait_ms <= 2000; 0 restores the
 * default of 2000 ms), sets the handle's device error word and lets its warp fall through to the
 * TMEM release, so the kernel ends and the context stays usable.  stall_iteration >= 0 makes the TMA
 * producer of the NEXT jump-term product (1) issue no loads for that iteration of its K loop: the
 * MMA issuer's wait for that stage runs out.  The call that contains that launch then returns
 * LB_CUDA_ERROR (its result is not valid), and the error word is cleared.  stall_iteration = -1
 * sets only the limit.  Errors: LB_INVALID_ARG (null handle, wait_ms outside [0, 2000],
 * stall_iteration < -1). */
lb_status lb_test_bounded_wait(lindblad_handle h, int stall_iteration, double wait_ms);

/* Number of CUDA kernels this library has launched in this process so far (all handles). */
long long lb_launch_count(void);

/* Releases the host-side handle (the workspace stays the caller's). */
void lindblad_destroy(lindblad_handle h);

/* Human-readable name of a status code. */
const char* lb_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif  /* LINDBLAD_H_ */
