"""GPU parity of the FP64 path against the CPU oracle, element by element, through the C ABI.

Tolerances (FP64 arithmetic, relative to the oracle's magnitude):
  * single operator applications (Phi, M, R_lam^S, L): 1e-11 relative max-norm -- a few hundred
    ulps for the O(n) accumulations and the Bartels-Stewart back-substitution;
  * steady states: relative Frobenius error <= 1e-10, after iterating to ||L rho||_max <= 1e-13
    (small-gap systems amplify the residual into the error by ~1/gap);
  * eigenvalues: |lambda - lambda_ref| <= 1e-8 |lambda_ref|.
"""
import numpy as np
import pytest
import torch

import lindblad_inputs as gi
from oracle import dense as D
from oracle import krylov as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2608_30860_b300 as B
    B.load_library()
    return B


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _setup(B, H, Ls, **kw):
    opts = B.default_opts(**kw)
    return B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)), opts), opts


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SYSTEMS = {
    "random6": lambda: gi.random_lindbladian(6, d=3, seed=11),
    "kerr12": lambda: gi.kerr_cat(12),
    "thermal9": lambda: gi.thermal_oscillator(9, omega=1.1, kappa=0.6, nth=0.4),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_phi_and_M_match_dense(B, name):
    H, Ls = SYSTEMS[name]()
    n = H.shape[0]
    h, _ = _setup(B, H, Ls)
    X = gi.random_operator(n, seed=3)
    Xd = _cuda(X)
    for form, sup in (("phi", D.Phi_super(H, Ls)), ("M", D.M_super(H, Ls))):
        ref = D.unvec(sup @ D.vec(X), n)
        got = B.phi_apply(h, Xd, form=form).cpu().numpy()
        assert _rel(got, ref) < 1e-11, (form, _rel(got, ref))
    B.lindblad_destroy(h)


@pytest.mark.parametrize("lam", [0.0, 0.7])
def test_resolvent_and_lindbladian_match_dense(B, lam):
    H, Ls = gi.random_lindbladian(7, d=2, seed=5)
    n = 7
    h, _ = _setup(B, H, Ls)
    Y = gi.random_operator(n, seed=8)
    G = D.G_matrix(H, Ls)
    ref = D.unvec(D.resolvent_S(G, lam) @ D.vec(Y), n)
    got = B.resolvent_apply(h, _cuda(Y), lam).cpu().numpy()
    assert _rel(got, ref) < 1e-11
    refL = D.unvec(D.liouvillian(H, Ls) @ D.vec(Y), n)
    gotL = B.lindbladian_apply(h, _cuda(Y)).cpu().numpy()
    assert _rel(gotL, refL) < 1e-12
    B.lindblad_destroy(h)


@pytest.mark.parametrize("n", [33, 70, 131])
def test_phi_ragged_sizes_match_matrix_free_oracle(B, n):
    """Several 32-wide Sylvester blocks and 64-wide GEMM tiles plus a ragged tail."""
    H, Ls = gi.random_lindbladian(n, d=3, seed=n)
    h, _ = _setup(B, H, Ls)
    sysm = K.System(H, Ls)
    X = gi.random_hermitian(n, seed=1)
    got = B.phi_apply(h, _cuda(X)).cpu().numpy()
    ref = sysm.Phi(X)
    assert _rel(got, ref) < 1e-11
    # trace preservation (App. C) holds for the GPU result itself
    assert abs(np.trace(got) - np.trace(X)) < 1e-11 * np.abs(X).sum()
    Y = gi.random_operator(n, seed=2)
    gotR = B.resolvent_apply(h, _cuda(Y), 0.3).cpu().numpy()
    assert _rel(gotR, sysm.resolvent_S(Y, 0.3)) < 1e-11
    B.lindblad_destroy(h)


def test_setup_reports_schur_quality(B):
    H, Ls = gi.kerr_cat(32)
    h, _ = _setup(B, H, Ls)
    assert h.setup_info["schur_backward_err"] < 1e-13
    G = D.G_matrix(H, Ls)
    assert abs(h.setup_info["min_abs_re_T"] - np.abs(np.linalg.eigvals(G).real).min()) < 1e-10
    B.lindblad_destroy(h)


@pytest.mark.parametrize("name,make", [
    ("kerr_cat_n32", lambda: gi.kerr_cat(32)),
    ("random_n48", lambda: gi.random_lindbladian(48, d=4, seed=0)),
    ("tfim_N5", lambda: gi.tfim(5, J=1.0, h=0.7, gamma=0.5, gamma_phi=0.1)),
])
def test_steady_state_matches_dense_lu(B, name, make):
    H, Ls = make()
    ref = D.steady_state_lu(H, Ls)
    h, opts = _setup(B, H, Ls, tol=1e-13, krylov_m=20, max_restarts=80)
    rho, info, st = B.steady_state(h, opts)
    rho = rho.cpu().numpy()
    assert st == 0, info
    assert info["residual_max"] < 1e-13
    assert np.linalg.norm(rho - ref) / np.linalg.norm(ref) < 1e-10
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.abs(rho - rho.conj().T).max() == 0.0
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    B.lindblad_destroy(h)


def test_steady_state_thermal_closed_form_rotated(B):
    n, nth = 40, 0.4
    H, Ls = gi.thermal_oscillator(n, omega=1.0, kappa=0.5, nth=nth)
    W = gi.haar_unitary(n, seed=1)
    Hr, Lr = gi.conjugate_system(H, Ls, W)
    x = nth / (1 + nth)
    ref = W @ np.diag((1 - x) * x ** np.arange(n) / (1 - x ** n)) @ W.conj().T
    h, opts = _setup(B, Hr, Lr, tol=1e-13)
    rho, info, st = B.steady_state(h, opts)
    assert st == 0
    assert np.abs(rho.cpu().numpy() - ref).max() < 1e-11
    B.lindblad_destroy(h)


def test_three_level_peripheral_converges(B):
    H, Ls = gi.three_level_cycle()
    h, opts = _setup(B, H, Ls, tol=1e-13, krylov_m=6)
    rho, info, st = B.steady_state(h, opts)
    assert st == 0
    assert np.abs(rho.cpu().numpy() - np.eye(3) / 3).max() < 1e-13
    B.lindblad_destroy(h)


def test_case_one_pure_state(B):
    """Theorem 1 case 1: damped oscillator at zero temperature, |0> in ker a."""
    H, Ls = gi.thermal_oscillator(10, omega=1.0, kappa=0.5, nth=0.0)
    h, opts = _setup(B, H, Ls)
    rho, info, st = B.steady_state(h, opts)
    assert st == 2
    ref = np.zeros((10, 10))
    ref[0, 0] = 1
    assert np.abs(rho.cpu().numpy() - ref).max() < 1e-13
    with pytest.raises(B.LindbladError):
        B.phi_apply(h, _cuda(np.eye(10, dtype=complex)))
    B.lindblad_destroy(h)


def test_low_spectrum_matches_dense_eig(B):
    H, Ls = gi.kerr_cat(16)
    ref = D.low_spectrum(H, Ls, 4)
    h, opts = _setup(B, H, Ls, tol=1e-10, krylov_m=20)
    ev, vecs, info, st = B.low_spectrum(h, 4, want_vectors=True, opts=opts)
    assert st == 0, info
    ev = ev.numpy()
    for r in ref:
        assert np.min(np.abs(ev - r)) <= 1e-8 * abs(r)
    V = vecs.cpu().numpy()
    Lmat = D.liouvillian(H, Ls)
    for lam, v in zip(ev, V):
        r = D.unvec(Lmat @ D.vec(v), 16) - lam * v
        assert np.abs(r).max() / np.abs(v).max() < 1e-10
        assert abs(np.trace(v)) < 1e-9 * np.abs(v).max() * 16
    B.lindblad_destroy(h)


def test_low_spectrum_damped_oscillator_positive_shift(B):
    """S is singular (case 1) at nth = 0, so mu > 0; the truncated spectrum is exact:
    {-kappa(p+q)/2 + i omega (q-p)}."""
    n, omega, kappa = 12, 1.0, 0.5
    H, Ls = gi.thermal_oscillator(n, omega=omega, kappa=kappa, nth=0.0)
    h, opts = _setup(B, H, Ls, tol=1e-10, krylov_m=16)
    with pytest.raises(B.LindbladError):
        B.low_spectrum(h, 3, mu=0.0, opts=opts)
    ev, _, info, st = B.low_spectrum(h, 3, mu=0.05, opts=opts)
    assert st == 0, info
    ref = np.array([-kappa / 2 - 1j * omega, -kappa / 2 + 1j * omega, -kappa + 0j])
    for r in ref:
        assert np.min(np.abs(ev.numpy() - r)) < 1e-8
    B.lindblad_destroy(h)


def test_eta_excluded_value_rejected(B):
    H, Ls = gi.random_lindbladian(6, d=2, seed=3)
    G = D.G_matrix(H, Ls)
    W = D.unvec(D.resolvent_S(G, 0.0) @ D.vec(np.eye(6)), 6)
    eta_bad = 1.0 / np.trace(W).real
    h, opts = _setup(B, H, Ls)
    with pytest.raises(B.LindbladError) as e:
        B.low_spectrum(h, 2, mu=0.0, eta=eta_bad, opts=opts)
    assert e.value.status == -3
    B.lindblad_destroy(h)


@pytest.mark.parametrize("lam", [0.0, 0.6])
def test_eigenbasis_route_matches_schur_route_and_oracle(B, lam):
    """Alg. 1 (eigenbasis divide, in Schur coordinates via R = Q^dag U) against Bartels-Stewart and
    the oracle's eigen route; well-conditioned random system (cond ~ 8 << gate 1e3)."""
    H, Ls = gi.random_lindbladian(96, d=3, seed=21)
    n = 96
    he, oe = _setup(B, H, Ls, route=B.LB_ROUTE_EIG)
    assert he.setup_info["route"] == B.LB_ROUTE_EIG and 1.0 <= he.setup_info["cond_eig"] < 1e3
    hs, _ = _setup(B, H, Ls)
    Y = gi.random_operator(n, seed=2)
    ge = B.resolvent_apply(he, _cuda(Y), lam).cpu().numpy()
    gs = B.resolvent_apply(hs, _cuda(Y), lam).cpu().numpy()
    ref = K.System(H, Ls, route="eig").resolvent_S(Y, lam)
    assert _rel(ge, ref) < 1e-11 and _rel(ge, gs) < 1e-11
    rho, info, st = B.steady_state(he, B.default_opts(tol=1e-13, route=B.LB_ROUTE_EIG))
    assert st == 0 and info["route"] == B.LB_ROUTE_EIG and info["residual_max"] < 1e-13
    rho_s, _, st_s = B.steady_state(hs, B.default_opts(tol=1e-13))
    rho, rho_s = rho.cpu().numpy(), rho_s.cpu().numpy()
    assert np.linalg.norm(rho - rho_s) / np.linalg.norm(rho_s) < 1e-10
    B.lindblad_destroy(he)
    B.lindblad_destroy(hs)


def test_eigenbasis_route_gate_refuses(B):
    """With the gate below the system's cond(U) the set-up reports LB_ILL_CONDITIONED (3) and keeps
    the Schur route, whose results stay exact."""
    H, Ls = gi.random_lindbladian(40, d=2, seed=5)
    opts = B.default_opts(route=B.LB_ROUTE_EIG, eig_cond_max=1.0)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)), opts)
    assert h.setup_info["status"] == 3 and h.setup_info["route"] == B.LB_ROUTE_SCHUR
    assert h.setup_info["cond_eig"] > 1.0
    X = gi.random_operator(40, seed=1)
    ref = D.unvec(D.Phi_super(H, Ls) @ D.vec(X), 40)
    assert _rel(B.phi_apply(h, _cuda(X)).cpu().numpy(), ref) < 1e-11
    B.lindblad_destroy(h)


def test_schur_backward_error_gate(B):
    """The set-up's Schur form (QR of the eigenvector matrix) on a non-normal Kerr cat (n = 160,
    eps2 = 8: eigenvector condition ~35) stays backward stable, ||lower(Q^dag G Q)||_F / ||G||_F
    below the default gate; a gate below that value makes the set-up fail with LB_SOLVER_ERROR
    instead of returning the Schur factor of another matrix."""
    H, Ls = gi.kerr_cat(160, eps2=8.0)
    h, _ = _setup(B, H, Ls)
    err = h.setup_info["schur_backward_err"]
    assert 0.0 < err < 1e-12
    B.lindblad_destroy(h)
    with pytest.raises(B.LindbladError) as e:
        _setup(B, H, Ls, schur_tol=0.1 * err)
    assert e.value.status == -6


@pytest.mark.parametrize("n", [70, 131])
def test_hermitian_flag_matches_general_path(B, n):
    """LB_APPLY_HERMITIAN (upper-tile jump term + mirror) gives the general path's result on a Hermitian
    input, to FP64 rounding, and an exactly Hermitian output; in both coordinate systems."""
    H, Ls = gi.random_lindbladian(n, d=3, seed=n + 1)
    h, _ = _setup(B, H, Ls)
    X = _cuda(gi.random_hermitian(n, seed=4))
    for schur in (False, True):
        yg = B.phi_apply(h, X, schur=schur).cpu().numpy()
        yh = B.phi_apply(h, X, schur=schur, hermitian=True).cpu().numpy()
        assert _rel(yh, yg) < 1e-12
        if schur:
            assert np.abs(yh - yh.conj().T).max() == 0.0
        kg = B.jump_apply(h, X, schur=schur).cpu().numpy()
        kh = B.jump_apply(h, X, schur=schur, hermitian=True).cpu().numpy()
        assert _rel(kh, kg) < 1e-13 and np.abs(kh - kh.conj().T).max() == 0.0
    B.lindblad_destroy(h)
