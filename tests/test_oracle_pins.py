"""Pins of the CPU oracle to facts fixed outside it: closed forms, values printed in the
paper, invariants the paper proves, and brute force on tiny inputs.  No GPU needed.

Each test names the mistake it is there to catch.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import quad_vec

import lindblad_inputs as gi
from oracle import dense as D
from oracle import krylov as K


def _thermal_closed_form(n, nth):
    x = nth / (1.0 + nth)
    p = (1 - x) * x ** np.arange(n) / (1 - x ** n)
    return np.diag(p).astype(np.complex128)


def _same_multiset(a, b, tol):
    left = list(b)
    for x in a:
        i = int(np.argmin(np.abs(np.array(left) - x)))
        if abs(left.pop(i) - x) > tol:
            return False
    return not left


# ----------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n,nth", [(6, 0.3), (12, 0.8), (20, 2.0)])
def test_thermal_gibbs_steady_state(n, nth):
    """Detailed balance p_{k+1}/p_k = nth/(1+nth) holds exactly for the truncated ladder.
    Catches: dissipator sign/factor mistakes, wrong kron order in vec."""
    H, Ls = gi.thermal_oscillator(n, omega=1.3, kappa=0.7, nth=nth)
    ref = _thermal_closed_form(n, nth)
    rho_lu = D.steady_state_lu(H, Ls)
    rho_svd, _ = D.steady_state_svd(H, Ls)
    assert np.abs(rho_lu - ref).max() < 1e-12
    assert np.abs(rho_svd - ref).max() < 1e-10


def test_thermal_gibbs_haar_rotated():
    """Unitary covariance: rotating (H, L) by W rotates rho_inf to W rho W^dag."""
    n, nth = 10, 0.5
    H, Ls = gi.thermal_oscillator(n, omega=0.9, kappa=0.4, nth=nth)
    W = gi.haar_unitary(n, seed=3)
    Hr, Lr = gi.conjugate_system(H, Ls, W)
    ref = W @ _thermal_closed_form(n, nth) @ W.conj().T
    assert np.abs(D.steady_state_lu(Hr, Lr) - ref).max() < 1e-12


@pytest.mark.parametrize("n", [4, 7])
def test_damped_oscillator_spectrum_exact(n):
    """nth = 0: L is triangular in total excitation, spectrum = {-kappa(p+q)/2 + i omega (q-p)}
    exactly at every truncation.  Catches: commutator sign, the 1/2 of the anticommutator."""
    omega, kappa = 1.7, 0.6
    H, Ls = gi.thermal_oscillator(n, omega=omega, kappa=kappa, nth=0.0)
    ev = D.liouvillian_eigenvalues(H, Ls)
    ref = np.array([-kappa * (p + q) / 2 + 1j * omega * (q - p) for p in range(n) for q in range(n)])
    # one-to-one matching (every closed-form value found, none left over)
    left = list(ev)
    for r in ref:
        i = int(np.argmin(np.abs(np.array(left) - r)))
        assert abs(left.pop(i) - r) < 1e-9
    assert not left


def test_qubit_decay_closed_forms(golden):
    """Footnote of Sec. 3.1: R K rho = (gamma/lam) rho_11 |0><0|, K R rho = gamma/(gamma+lam) rho_11 |0><0|,
    and the two induced trace norms.  Catches: resolvent sign (lam - S vs lam + S), G's factor 1/2."""
    _, rows = golden("qubit_decay.txt")
    rho = gi.random_density(2, seed=5)
    for gamma, lam, r_rk, r_kr in rows:
        H, Ls = gi.qubit_decay(gamma)
        G = D.G_matrix(H, Ls)
        R = D.resolvent_S(G, lam)
        Kop = D.K_super(Ls)
        RK = D.unvec(R @ Kop @ D.vec(rho), 2)
        KR = D.unvec(Kop @ R @ D.vec(rho), 2)
        e00 = np.zeros((2, 2), dtype=np.complex128)
        e00[0, 0] = 1.0
        assert np.abs(RK - r_rk * rho[1, 1] * e00).max() < 1e-12
        assert np.abs(KR - r_kr * rho[1, 1] * e00).max() < 1e-12
        assert abs(D.cp_trace_norm(R @ Kop, 2) - r_rk) < 1e-10 * r_rk
        assert abs(D.cp_trace_norm(Kop @ R, 2) - r_kr) < 1e-12


def test_qubit_decay_is_case_one():
    """Theorem 1, first case: G = -(gamma/2)|1><1| has eigenvalue 0 (on iR); rho_inf = |0><0|."""
    H, Ls = gi.qubit_decay(0.8)
    G = D.G_matrix(H, Ls)
    assert np.min(np.abs(np.linalg.eigvals(G).real)) == 0.0
    rho = D.steady_state_lu(H, Ls)
    assert abs(rho[0, 0] - 1) < 1e-14 and abs(rho[1, 1]) < 1e-14


# ----------------------------------------------------------------------------- printed values
def test_three_level_peripheral_spectrum(golden):
    """Remark 'Peripheral spectra of Phi': rho_inf = I/3, Phi has 1, exp(+-2 pi i/3) on the unit circle."""
    kv, _ = golden("three_level_peripheral.txt")
    H, Ls = gi.three_level_cycle()
    rho = D.steady_state_lu(H, Ls)
    assert np.abs(np.diag(rho).real - kv["steady_state_diag"]).max() < 1e-14
    ev = np.linalg.eigvals(D.Phi_super(H, Ls))
    per = ev[np.abs(np.abs(ev) - 1) < 1e-9]
    ref = np.array(kv["peripheral_re"]) + 1j * np.array(kv["peripheral_im"])
    assert len(per) == 3
    for r in ref:
        assert np.min(np.abs(per - r)) < 1e-12


def test_three_level_gauge_shift(golden):
    """Conclusion: with c = (1,0,0) the pair becomes 1/2 +- i/(2 sqrt 2), all others |.| <= sqrt(3/8).
    Exercises Phi with a non-scalar G, so a wrong S^{-1} or a wrong G fails."""
    kv, _ = golden("three_level_gauge.txt")
    H, Ls = gi.three_level_cycle()
    c = kv["c"]
    Ht, Lt = D.gauge_split(H, Ls, c)
    # the gauge leaves L unchanged (Eq. lindblad_gauge_split)
    assert np.abs(D.liouvillian(Ht, Lt) - D.liouvillian(H, Ls)).max() < 1e-14
    ev = np.linalg.eigvals(D.Phi_super(Ht, Lt))
    i1 = np.argmin(np.abs(ev - 1))
    assert abs(ev[i1] - 1) < 1e-12
    others = np.delete(ev, i1)
    assert np.abs(others).max() <= kv["max_other_modulus"][0] + 1e-12
    for re, im in zip(kv["pair_re"], kv["pair_im"]):
        assert np.min(np.abs(others - (re + 1j * im))) < 1e-12


# ----------------------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def rand6():
    return gi.random_lindbladian(6, d=3, seed=11)


def test_phi_trace_preserving_and_M_not(rand6):
    """App. C: Phi = -K S^{-1} is TP (Phi^*(I) = I).  M = -S^{-1} K is similar but not TP,
    so this also catches a swapped composition order."""
    H, Ls = rand6
    n = 6
    P = D.Phi_super(H, Ls)
    M = D.M_super(H, Ls)
    X = gi.random_operator(n, seed=2)
    assert abs(np.trace(D.unvec(P @ D.vec(X), n)) - np.trace(X)) < 1e-12
    assert np.abs(D.superop_adjoint_apply(P, np.eye(n), n) - np.eye(n)).max() < 1e-12
    assert abs(np.trace(D.unvec(M @ D.vec(X), n)) - np.trace(X)) > 1e-3
    assert _same_multiset(np.linalg.eigvals(P), np.linalg.eigvals(M), 1e-9)


def test_complete_positivity(rand6):
    """-S^{-1} and Phi are CP (Eq. lyapunov_solution, Theorem 1): their Choi matrices are PSD."""
    H, Ls = rand6
    n = 6
    G = D.G_matrix(H, Ls)
    for op in (-np.linalg.inv(D.S_super(G)), D.Phi_super(H, Ls)):
        C = D.choi(op, n)
        C = 0.5 * (C + C.conj().T)
        assert np.linalg.eigvalsh(C).min() > -1e-12


def test_lyapunov_integral_form(rand6):
    """S^{-1}(Y) = -int_0^inf e^{tG} Y e^{tG^dag} dt (Eq. lyapunov_solution), by quadrature."""
    H, Ls = rand6
    n = 6
    G = D.G_matrix(H, Ls)
    Y = gi.random_hermitian(n, seed=4)
    rate = -np.linalg.eigvals(G).real.max()
    Tend = 60.0 / rate

    def f(t):
        E = sla.expm(t * G)
        return (E @ Y @ E.conj().T).reshape(-1)

    integ, _ = quad_vec(f, 0.0, Tend, epsabs=1e-13, epsrel=1e-12, limit=400)
    X = -integ.reshape(n, n)
    Xs = D.unvec(np.linalg.solve(D.S_super(G), D.vec(Y)), n)
    assert np.abs(X - Xs).max() < 1e-8 * np.abs(Xs).max()


def test_kernel_correspondence(rand6):
    """Theorem 1 / Remark: rho_inf = -c S^{-1} xi_inf with xi_inf the fixed point of Phi, and M rho_inf = rho_inf."""
    H, Ls = rand6
    n = 6
    G = D.G_matrix(H, Ls)
    P = D.Phi_super(H, Ls)
    ev, V = np.linalg.eig(P)
    xi = V[:, np.argmin(np.abs(ev - 1))]
    rho = D.hermitize_normalize(D.unvec(-np.linalg.solve(D.S_super(G), xi), n) / np.exp(1j * np.angle(xi[0])))
    ref = D.steady_state_lu(H, Ls)
    assert np.abs(rho - ref).max() < 1e-11
    M = D.M_super(H, Ls)
    assert np.abs(M @ D.vec(ref) - D.vec(ref)).max() < 1e-11


def test_deflation_spectrum(rand6):
    """Sec. 4.2: spec(L~_eta) = spec(L) with 0 replaced by eta*n."""
    H, Ls = rand6
    n, eta = 6, 0.37
    ev = np.linalg.eigvals(D.liouvillian(H, Ls))
    evd = np.linalg.eigvals(D.deflated_liouvillian(H, Ls, eta))
    ref = np.delete(ev, np.argmin(np.abs(ev)))
    ref = np.append(ref, eta * n)
    for r in ref:
        assert np.min(np.abs(evd - r)) < 1e-9


@pytest.mark.parametrize("lam", [0.0, 0.8])
def test_sherman_morrison_preconditioner(rand6, lam):
    """Alg. 2 equals the brute-force inverse of (lam - S) - c|I><I| (Eq. ShermanMorr)."""
    H, Ls = rand6
    n, c = 6, 1.0
    G = D.G_matrix(H, Ls)
    X = gi.random_operator(n, seed=9)
    P = D.precond_alg2(G, lam, c, X)
    ref = D.unvec(D.deflated_noJump_inverse(G, lam, c) @ D.vec(X), n)
    assert np.abs(P - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("lam", [0.05, 0.5, 3.0])
def test_contraction_theorem(rand6, lam):
    """Theorem 2: ||K R_lam^S|| = 1 - lam*delta_lam < 1, delta_lam = min_rho Tr R_lam^S(rho)
    = lambda_min(R^*(I)); and the right-preconditioning identity (lam - L) R = Id - K R."""
    H, Ls = rand6
    n = 6
    G = D.G_matrix(H, Ls)
    R = D.resolvent_S(G, lam)
    Kop = D.K_super(Ls)
    nrm = D.cp_trace_norm(Kop @ R, n)
    RstarI = D.superop_adjoint_apply(R, np.eye(n), n)
    delta = np.linalg.eigvalsh(0.5 * (RstarI + RstarI.conj().T)).min()
    assert nrm < 1.0
    assert abs(nrm - (1.0 - lam * delta)) < 1e-10
    lhs = (lam * np.eye(n * n) - D.liouvillian(H, Ls)) @ R
    assert np.abs(lhs - (np.eye(n * n) - Kop @ R)).max() < 1e-10


def test_phi_norm_is_one_at_zero_shift(rand6):
    """Remark 'Loss of the contraction at zero shift': ||K R_0^S|| = ||Phi|| = 1."""
    H, Ls = rand6
    assert abs(D.cp_trace_norm(D.Phi_super(H, Ls), 6) - 1.0) < 1e-11


# ----------------------------------------------------------------------------- matrix-free tier
@pytest.mark.parametrize("route", ["schur", "eig"])
@pytest.mark.parametrize("lam", [0.0, 0.9])
def test_tierb_resolvent_matches_dense(rand6, route, lam):
    """App. A.1: both Lyapunov routes equal the dense (lam - S)^{-1}."""
    H, Ls = rand6
    s = K.System(H, Ls, route=route)
    X = gi.random_operator(6, seed=1)
    ref = D.unvec(D.resolvent_S(s.G, lam) @ D.vec(X), 6)
    assert np.abs(s.resolvent_S(X, lam) - ref).max() < 1e-11 * np.abs(ref).max()


def test_tierb_phi_and_M_match_dense(rand6):
    H, Ls = rand6
    s = K.System(H, Ls)
    X = gi.random_operator(6, seed=7)
    assert np.abs(s.Phi(X) - D.unvec(D.Phi_super(H, Ls) @ D.vec(X), 6)).max() < 1e-11
    assert np.abs(s.M(X) - D.unvec(D.M_super(H, Ls) @ D.vec(X), 6)).max() < 1e-11


def test_tierb_lyapunov_residual_large():
    """The definition G X + X G^dag = Y checked directly at a size the dense tier cannot reach."""
    H, Ls = gi.random_lindbladian(160, d=4, seed=1)
    s = K.System(H, Ls)
    Y = gi.random_hermitian(160, seed=2)
    X = s.S_inv(Y)
    assert np.abs(s.S(X) - Y).max() < 1e-10 * np.abs(Y).max()
    assert np.abs(X - X.conj().T).max() < 1e-10 * np.abs(X).max()   # Hermitian in -> Hermitian out


@pytest.mark.parametrize("make", [lambda: gi.kerr_cat(14), lambda: gi.random_lindbladian(9, d=3, seed=4)])
def test_tierb_alg4_and_alg3_match_lu(make):
    H, Ls = make()
    s = K.System(H, Ls)
    ref = D.steady_state_lu(H, Ls)
    r4, info4 = K.steady_state_phi_arnoldi(s, tol=1e-12, m=16)
    r3, info3 = K.steady_state_gmres(s, tol=1e-12, m=16)
    assert info4["residual"] < 1e-12 and info3["residual"] < 1e-12
    assert np.linalg.norm(r4 - ref) / np.linalg.norm(ref) < 1e-9
    assert np.linalg.norm(r3 - ref) / np.linalg.norm(ref) < 1e-9


def test_tierb_alg4_three_level_peripheral():
    """Arnoldi with the nearest-to-1 Ritz rule converges despite the peripheral eigenvalues."""
    H, Ls = gi.three_level_cycle()
    rho, info = K.steady_state_phi_arnoldi(K.System(H, Ls), tol=1e-13, m=8)
    assert np.abs(rho - np.eye(3) / 3).max() < 1e-13


def test_tierb_thermal_closed_form_larger_n():
    n, nth = 48, 0.4
    H, Ls = gi.thermal_oscillator(n, omega=1.0, kappa=0.5, nth=nth)
    W = gi.haar_unitary(n, seed=1)
    Hr, Lr = gi.conjugate_system(H, Ls, W)
    rho, info = K.steady_state_phi_arnoldi(K.System(Hr, Lr), tol=1e-13, m=20)
    ref = W @ _thermal_closed_form(n, nth) @ W.conj().T
    assert np.abs(rho - ref).max() < 1e-11


@pytest.mark.parametrize("k_recycle", [0, 6])
def test_tierb_shift_invert_matches_dense(k_recycle):
    """Alg. 5 returns the k smallest-|lambda| nonzero eigenvalues of the dense L (inner solves plain or
    with the recycled pair threaded through every OP application)."""
    H, Ls = gi.random_lindbladian(7, d=3, seed=8)
    s = K.System(H, Ls)
    lam, vecs, info = K.low_spectrum_shift_invert(s, k=4, tol=1e-10, m=16, k_recycle=k_recycle)
    ref = D.low_spectrum(H, Ls, 4)
    for r in ref:
        assert np.min(np.abs(lam - r)) < 1e-8 * abs(r)
    for l, v in zip(lam, vecs):
        assert abs(np.trace(v)) < 1e-8 * np.abs(v).max() * 7   # nonzero modes are traceless


def test_damped_oscillator_low_spectrum_shift_invert():
    """Low-lying damped-oscillator rates from Alg. 5 with mu > 0 (case 1: S singular at nth = 0)."""
    n, omega, kappa = 12, 1.0, 0.5
    H, Ls = gi.thermal_oscillator(n, omega=omega, kappa=kappa, nth=0.0)
    s = K.System(H, Ls)
    lam, _, info = K.low_spectrum_shift_invert(s, k=3, mu=0.05, tol=1e-9, m=16)
    ref = np.array([-kappa / 2 - 1j * omega, -kappa / 2 + 1j * omega, -kappa + 0j])
    for r in ref:
        assert np.min(np.abs(lam - r)) < 1e-8


# ----------------------------------------------------------------------------- gradient
def _tfim_param_fns(N):
    HJ, Hh, decay, dephase, Sz = gi.tfim_terms(N)

    def Hf(t):
        return t[0] * HJ + t[1] * Hh

    def Lf(t):
        return [np.sqrt(t[2]) * L for L in decay] + [np.sqrt(t[3]) * L for L in dephase]

    Z = np.zeros_like(HJ)

    def dL(t):
        return [D.liouvillian(HJ, []), D.liouvillian(Hh, []),
                D.liouvillian(Z, decay), D.liouvillian(Z, dephase)]
    return Hf, Lf, dL, Sz


def test_dense_adjoint_gradient_vs_finite_differences():
    """Remark 'Differentiating the steady state': the adjoint gradient equals central differences."""
    N = 3
    Hf, Lf, dL, Sz = _tfim_param_fns(N)
    theta = np.array([1.0, 0.7, 0.5, 0.1])
    g, rho = D.steady_state_gradient(Hf, Lf, dL, theta, Sz)
    for i in range(4):
        h = 1e-5 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fp = np.trace(Sz @ D.steady_state_lu(Hf(tp), Lf(tp))).real
        fm = np.trace(Sz @ D.steady_state_lu(Hf(tm), Lf(tm))).real
        assert abs(g[i] - (fp - fm) / (2 * h)) < 1e-6 * max(1.0, abs(g[i]))
    # Euler scaling identity: L(s theta) = s L(theta) => sum_i theta_i dJ/dtheta_i = 0
    assert abs(np.dot(theta, g)) < 1e-10


# ----------------------------------------------------------------------------- generators
def test_tfim_conventions_and_reflection_symmetry():
    N = 4
    H, Ls = gi.tfim(N, J=1.0, h=0.7, gamma=0.5, gamma_phi=0.1)
    n = 2 ** N
    assert np.abs(H - H.conj().T).max() == 0.0
    up = np.zeros(n)
    up[0] = 1.0                           # all sites up = |00..0>
    assert np.abs(Ls[0] @ up).max() > 0   # sigma_minus on site 1 lowers |0...>
    rho = D.steady_state_lu(H, Ls)
    _, _, _, dephase, _ = gi.tfim_terms(N)
    sz = [np.trace(P @ rho).real for P in dephase]
    assert np.allclose(sz, sz[::-1], atol=1e-12)
    assert np.linalg.eigvalsh(rho).min() > -1e-12


def test_single_entry_jump_term_and_G_rows_match_dense():
    """The entry-wise oracle (used at n = 4096) against the dense superoperator and G at small n,
    for dense random jumps and for the sparse TFIM decay jumps."""
    rng = np.random.default_rng(11)
    for H, Ls in (gi.random_lindbladian(9, d=3, seed=5), gi.tfim(3, J=1.0, h=0.7, gamma=0.5, gamma_phi=0.1)):
        n = H.shape[0]
        X = gi.random_operator(n, seed=2)
        KX = D.unvec(D.K_super(Ls) @ D.vec(X), n)
        pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(25, 2))]
        got = D.jump_term_entries(Ls, X, pairs)
        ref = np.array([KX[a, b] for a, b in pairs])
        assert np.abs(got - ref).max() < 1e-13 * max(1.0, np.abs(KX).max())
        idx = [0, n - 1, n // 2]
        assert np.abs(D.G_rows(H, Ls, idx) - D.G_matrix(H, Ls)[idx]).max() < 1e-13


# ----------------------------------------------------------------------------- adjoint, vectors
def test_L_adjoint_is_the_hilbert_schmidt_adjoint():
    """System.L_adjoint against the conjugate transpose of the dense Liouvillian and the defining
    identity <Y, L(X)> = <L^*(Y), X> (a dropped G term or a swapped dagger fails both)."""
    H, Ls = gi.random_lindbladian(6, d=3, seed=2)
    s = K.System(H, Ls)
    X, Y = gi.random_operator(6, seed=3), gi.random_operator(6, seed=4)
    ref = D.unvec(D.liouvillian(H, Ls).conj().T @ D.vec(Y), 6)
    assert np.abs(s.L_adjoint(Y) - ref).max() < 1e-13
    assert abs(K.hs_inner(Y, s.L(X)) - K.hs_inner(s.L_adjoint(Y), X)) < 1e-12
    # L^* is unital: L^*(I) = 0 (trace preservation of the dynamics)
    assert np.abs(s.L_adjoint(np.eye(6, dtype=np.complex128))).max() < 1e-13


def test_low_spectrum_with_vectors_damped_oscillator():
    """The damped oscillator at n_th = 0 has the exact truncated spectrum -kappa(p+q)/2 + i omega(q-p)
    (triangular in the excitation number): values and eigenvectors (L v = lambda v) are checked."""
    n, omega, kappa = 7, 1.0, 1.0
    H, Ls = gi.thermal_oscillator(n, omega=omega, kappa=kappa, nth=0.0)
    lam, vecs = D.low_spectrum_with_vectors(H, Ls, 3)
    full = np.array([-kappa * (p + q) / 2 + 1j * omega * (q - p) for p in range(n) for q in range(n)])
    full = full[np.argsort(np.abs(full))]
    ref = full[1:4]          # -1 and the pair -1/2 +- i; the next modulus (2) is well separated
    assert np.abs(np.abs(full[4]) - np.abs(full[3])) > 0.5
    assert _same_multiset(lam, ref, 1e-10)
    Lmat = D.liouvillian(H, Ls)
    for l, v in zip(lam, vecs):
        r = D.unvec(Lmat @ D.vec(v), n) - l * v
        assert np.abs(r).max() < 1e-10 * np.abs(v).max()
        assert abs(np.trace(v)) < 1e-10 * np.abs(v).max() * n


# ----------------------------------------------------------------------------- gauge split
def test_gauge_split_keeps_L_and_moves_B_into_the_jump_part():
    """Eq. lindblad_gauge_split on a random system: L unchanged, G~ = G - B - 1/2 sum |c_j|^2 with
    B = sum c_j^* L_j, and K~ Kraus (K~ - K = B rho + rho B^dag + sum |c_j|^2 rho)."""
    H, Ls = gi.random_lindbladian(5, d=3, seed=9)
    c = np.array([0.3 - 0.2j, -0.7 + 0.1j, 0.25j])
    Ht, Lt = D.gauge_split(H, Ls, c)
    assert np.abs(Ht - Ht.conj().T).max() < 1e-14
    assert np.abs(D.liouvillian(Ht, Lt) - D.liouvillian(H, Ls)).max() < 1e-13
    Bm = sum(np.conj(cj) * L for cj, L in zip(c, Ls))
    Gt = D.G_matrix(Ht, Lt)
    assert np.abs(Gt - (D.G_matrix(H, Ls) - Bm - 0.5 * np.sum(np.abs(c) ** 2) * np.eye(5))).max() < 1e-13
    X = gi.random_operator(5, seed=1)
    dK = D.unvec((D.K_super(Lt) - D.K_super(Ls)) @ D.vec(X), 5)
    assert np.abs(dK - (Bm @ X + X @ Bm.conj().T + np.sum(np.abs(c) ** 2) * X)).max() < 1e-13


# ----------------------------------------------------------------------------- resolvent of L
@pytest.mark.parametrize("lam", [2.0, 0.3])
def test_resolvent_L_neumann_series_trace_and_laplace(rand6, lam):
    """Corollary 'Resolvent of the Lindbladian': R_lam^L = R_lam^S sum_k (K R_lam^S)^k (a truncated
    series, independent of the LU); Tr R_lam^L(B) = Tr B / lam; and the Laplace transform
    R_lam^L(B) = int_0^inf e^{-lam t} e^{L t} B dt by quadrature."""
    H, Ls = rand6
    n = 6
    B = gi.random_hermitian(n, seed=5)
    X = D.resolvent_L(H, Ls, lam, B)
    RS = D.resolvent_S(D.G_matrix(H, Ls), lam)
    N = D.K_super(Ls) @ RS
    acc, term = np.zeros(n * n, dtype=np.complex128), D.vec(B).astype(np.complex128)
    for _ in range(4000):
        acc = acc + term
        term = N @ term
        if np.abs(term).max() < 1e-17:
            break
    assert np.abs(D.unvec(RS @ acc, n) - X).max() < 1e-11 * np.abs(X).max()
    assert abs(np.trace(X) - np.trace(B) / lam) < 1e-12 * abs(np.trace(B) / lam)
    Lm = D.liouvillian(H, Ls)
    f = lambda t: np.exp(-lam * t) * (sla.expm(Lm * t) @ D.vec(B))
    lap, _ = quad_vec(f, 0.0, np.inf, epsabs=1e-12, epsrel=1e-11)
    assert np.abs(D.unvec(lap, n) - X).max() < 1e-8 * np.abs(X).max()


# ----------------------------------------------------------------------------- implicit Euler
def test_implicit_euler_eigenvector_exact_and_first_order():
    """Eq. resolvent: an eigenvector v (L v = lambda v) evolves exactly as (1 - dt lambda)^-k v; the
    trace is kept at every step; and the error against e^{L t} rho0 halves with dt (first order)."""
    H, Ls = gi.random_lindbladian(5, d=2, seed=3)
    lam, vecs = D.low_spectrum_with_vectors(H, Ls, 1)
    v = vecs[0]
    dt, k = 0.3, 4
    out = D.implicit_euler(H, Ls, v, dt, k)
    assert np.abs(out[-1] - v * (1 - dt * lam[0]) ** (-k)).max() < 1e-12 * np.abs(v).max()
    rho0 = gi.random_density(5, seed=2)
    T = 1.0
    exact = D.unvec(sla.expm(D.liouvillian(H, Ls) * T) @ D.vec(rho0), 5)
    errs = []
    for steps in (20, 40, 80):
        traj = D.implicit_euler(H, Ls, rho0, T / steps, steps)
        assert all(abs(np.trace(r) - 1.0) < 1e-12 for r in traj)
        errs.append(np.abs(traj[-1] - exact).max())
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


# ----------------------------------------------------------------------------- recycled GMRES
def test_gcrodr_solves_and_keeps_its_recycled_relation():
    """GCRO-DR on a small shifted system: the solution equals the dense solve, the returned pair
    satisfies B U = C with C orthonormal, and a second right-hand side solved with that pair needs
    fewer matrix-vector products than a solve without it."""
    H, Ls = gi.random_lindbladian(8, d=3, seed=6)
    s = K.System(H, Ls)
    lam = 0.05
    mv = lambda X: lam * X - s.L(X)
    pc = lambda X: s.resolvent_S(X, lam)
    b1, b2 = gi.random_operator(8, seed=1), gi.random_operator(8, seed=2)
    x1, (U, C), info1 = K.gcrodr(mv, pc, b1, np.zeros_like(b1), m=12, k=4, atol=1e-13, max_cycles=60)
    ref = D.resolvent_L(H, Ls, lam, b1)
    assert np.abs(x1 - ref).max() < 1e-10 * np.abs(ref).max()
    Gm = np.array([[K.hs_inner(a, c) for c in C] for a in C])
    assert np.abs(Gm - np.eye(len(C))).max() < 1e-12
    for u, c in zip(U, C):
        assert np.abs(mv(pc(u)) - c).max() < 1e-10
    _, _, cold = K.gcrodr(mv, pc, b2, np.zeros_like(b2), m=12, k=4, atol=1e-11, max_cycles=60)
    x2, _, warm = K.gcrodr(mv, pc, b2, np.zeros_like(b2), m=12, k=4, recycle=(U, C), atol=1e-11, max_cycles=60)
    assert np.abs(x2 - D.resolvent_L(H, Ls, lam, b2)).max() < 1e-9 * np.abs(x2).max()
    assert warm["steps"] < cold["steps"]


@pytest.mark.parametrize("make", [lambda: gi.kerr_cat(14), lambda: gi.random_lindbladian(9, d=3, seed=4)])
def test_tierb_alg3_recycled_matches_lu(make):
    H, Ls = make()
    rho, info = K.steady_state_gmres(K.System(H, Ls), tol=1e-12, m=16, k_recycle=4)
    ref = D.steady_state_lu(H, Ls)
    assert info["residual"] < 1e-12
    assert np.linalg.norm(rho - ref) / np.linalg.norm(ref) < 1e-9


def test_tierb_resolvent_gmres_matches_dense_at_three_shifts():
    """The resolvent benchmark's solve (Sec. 3.4): B = I/n, lam = lam_max 10^{0,-1,-2}."""
    H, Ls = gi.paper_random_lindbladian(7, seed=0)
    s = K.System(H, Ls)
    lmax = np.abs(D.liouvillian_eigenvalues(H, Ls)).max()
    B = np.eye(7, dtype=np.complex128) / 7
    rec = None
    for lam in (lmax, lmax / 10, lmax / 100):
        X, rec, info = K.resolvent_gmres(s, lam, B, tol=1e-12, m=16, k_recycle=4)
        ref = D.resolvent_L(H, Ls, lam, B)
        assert info["residual"] < 1e-12
        assert np.abs(X - ref).max() < 1e-10 * np.abs(ref).max()
        rec = None   # each shift is another operator


@pytest.mark.parametrize("n,m,k", [(8, 12, 4), (16, 40, 8)])
def test_tierb_implicit_euler_gmres_matches_dense(n, m, k):
    """Each step's solve converges inside one cycle (lam = 1/dt is large), so the recycled pair is carried
    across solves from nearly converged cycles: the case that makes [U, V] numerically rank-deficient."""
    H, Ls = gi.stiff_random_lindbladian(n, K=2.0, seed=1)
    rho0 = np.zeros((n, n), dtype=np.complex128)
    rho0[0, 0] = 1.0
    dt = 0.05
    ref = D.implicit_euler(H, Ls, rho0, dt, 6)
    got = K.implicit_euler_gmres(K.System(H, Ls), rho0, dt, 6, tol=1e-12, m=m, k_recycle=k)
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() < 1e-10


def test_memory_buffer_cat_generator():
    """App. B cat qubit: a = a~ (x) I and b = I (x) b~ commute, the truncations follow
    n_a = round(sqrt(3 n)), n_b = floor(n_a / 3), S is invertible (case 2 of Theorem 1) and the
    steady state is unique (LU and SVD null vectors agree)."""
    assert gi.memory_buffer_dims(64) == (14, 4)
    na, nb = 6, 2
    H, Ls = gi.memory_buffer_cat(na, nb)
    n = na * nb
    assert H.shape == (n, n) and len(Ls) == 4
    b, a = Ls[0], Ls[2]
    assert np.abs(a @ b - b @ a).max() < 1e-14
    assert np.abs(a @ b.conj().T - b.conj().T @ a).max() < 1e-14
    G = D.G_matrix(H, Ls)
    assert np.abs(np.linalg.eigvals(G).real).min() > 1e-6
    r_lu = D.steady_state_lu(H, Ls)
    r_svd, sv = D.steady_state_svd(H, Ls)
    assert sv[-2] > 1e3 * sv[-1]
    assert np.abs(r_lu - r_svd).max() < 1e-9


def test_gcrodr_pair_stays_consistent_over_a_sequence_of_solves():
    """Twenty unrelated right-hand sides through one recycled pair (the shift-invert use of GCRO-DR,
    Parks et al. 2006): after every solve the pair still satisfies its defining relations, B U = C
    with B = A P and C orthonormal, and the true residual of every solve is at the requested
    tolerance.  A wrong factor in the update (Q instead of Q R, Z without R^{-1}, a basis that is not
    orthonormal) breaks the first relation at once; a pair that decays over the sequence breaks it late."""
    H, Ls = gi.random_lindbladian(8, d=3, seed=2)
    s = K.System(H, Ls)
    mv = lambda X: s.shifted_deflated(X, 0.0, 1.0)
    pc = lambda X: s.precond(X, 0.0, 1.0)
    rng = np.random.default_rng(0)
    rec = None
    worst, worst_rel, worst_orth, formed = 0.0, 0.0, 0.0, 0
    for _ in range(20):
        b = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
        x, rec, info = K.gcrodr(mv, pc, b, np.zeros_like(b), m=16, k=4, recycle=rec,
                                atol=1e-10 * K.hs_norm(b), max_cycles=30)
        worst = max(worst, K.hs_norm(b - mv(x)) / K.hs_norm(b))
        if rec is not None and rec[0] is not None:
            U, C = rec
            formed += 1
            for u, c in zip(U, C):
                worst_rel = max(worst_rel, K.hs_norm(mv(pc(u)) - c) / K.hs_norm(c))
            gram = np.array([[np.vdot(a, c) for c in C] for a in C])
            worst_orth = max(worst_orth, float(np.abs(gram - np.eye(len(C))).max()))
    assert formed >= 10
    assert worst < 1e-9
    assert worst_rel < 1e-10
    assert worst_orth < 1e-9    # one-pass combination of the Arnoldi basis: 1.5e-11 measured
