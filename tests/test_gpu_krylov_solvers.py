"""GPU parity of the GMRES-based solvers against the CPU oracle, through the C ABI:
Alg. 3 (steady state as a recycled preconditioned linear solve), the resolvent of the Lindbladian
(Sec. 3.4), implicit Euler (Sec. 4.3), the gauge-shifted split (Remark "Non-uniqueness of the
decomposition") and the memory-buffer cat qubit (App. B).

Bars (FP64): steady states 1e-10 relative Frobenius (or the problem's conditioning limit
10 ||r||_F / sigma_2(L), as in test_gpu_fp64.py); resolvent solves 1e-10 relative max-norm after a
1e-12 absolute max-norm stop (the solution has entries O(1 / (n lam)), so an absolute 1e-12 residual
bounds the relative error by cond / n); implicit Euler steps 1e-10 absolute per state (each step
stops at 1e-12 relative residual and the map is a contraction); eigenvalues 1e-8 relative.
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


def _state_bar(H, Ls, info, ref):
    Lm = D.liouvillian(H, Ls)
    sigma2 = np.linalg.svd(Lm, compute_uv=False)[-2]
    return max(1e-10, 10 * info["residual_fro"] / sigma2 / np.linalg.norm(ref))


@pytest.mark.parametrize("name,make", [
    ("kerr_cat_n32", lambda: gi.kerr_cat(32)),
    ("random_n48", lambda: gi.random_lindbladian(48, d=4, seed=0)),
    ("tfim_N5", lambda: gi.tfim(5, J=1.0, h=0.7, gamma=0.5, gamma_phi=0.1)),
])
def test_alg3_steady_state_matches_dense_lu(B, name, make):
    H, Ls = make()
    ref = D.steady_state_lu(H, Ls)
    h, opts = _setup(B, H, Ls, tol=1e-13, gmres_m=32, recycle_k=8, max_restarts=100)
    rho, info, st = B.steady_state_gmres(h, opts)
    print(name, info)
    rho = rho.cpu().numpy()
    assert st == 0, info
    assert info["residual_max"] < 1e-13
    assert np.linalg.norm(rho - ref) / np.linalg.norm(ref) < _state_bar(H, Ls, info, ref)
    assert abs(np.trace(rho) - 1) < 1e-13 and np.abs(rho - rho.conj().T).max() == 0.0
    B.lindblad_destroy(h)


def test_alg3_recycling_against_plain_restarts(B):
    """The same solve without recycling (recycle_k = 0) reaches the same state; recycling does not
    need more preconditioned applications on this slowly converging Kerr cat."""
    H, Ls = gi.kerr_cat(24, eps2=6.0)
    h, _ = _setup(B, H, Ls)
    o_rec = B.default_opts(tol=1e-12, gmres_m=24, recycle_k=8, max_restarts=200)
    o_plain = B.default_opts(tol=1e-12, gmres_m=24, recycle_k=0, max_restarts=200)
    r1, i1, s1 = B.steady_state_gmres(h, o_rec)
    r0, i0, s0 = B.steady_state_gmres(h, o_plain)
    print("recycled", i1, "plain", i0)
    assert s1 == 0 and s0 == 0
    assert i1["phi_applies"] <= i0["phi_applies"]
    ref = D.steady_state_lu(H, Ls)
    for r, i in ((r1, i1), (r0, i0)):
        r = r.cpu().numpy()
        assert np.linalg.norm(r - ref) / np.linalg.norm(ref) < _state_bar(H, Ls, i, ref)
    B.lindblad_destroy(h)


@pytest.mark.parametrize("n", [70, 160])
def test_alg3_mixed_refined_to_fp64(B, n):
    """Tensor-core GMRES cycles with FP64 residual corrections: ||L rho||_max <= 1e-11 and 1e-9
    relative agreement with the oracle's Alg. 4."""
    H, Ls = gi.random_lindbladian(n, d=4, seed=0)
    ref = K.steady_state_phi_arnoldi(K.System(H, Ls), tol=1e-13)[0]
    h, _ = _setup(B, H, Ls)
    rho, info, st = B.steady_state_gmres(h, B.default_opts(precision=B.LB_PREC_MIXED, tol=1e-11))
    print(n, info)
    assert st == 0, info
    assert info["residual_max"] <= 1e-11
    rho = rho.cpu().numpy()
    assert np.linalg.norm(rho - ref) / np.linalg.norm(ref) < 1e-9
    B.lindblad_destroy(h)


def test_resolvent_solve_three_shifts_match_dense(B):
    """Sec. 3.4's workload on the paper's dense family: (lam - L) X = I/n at lam = lam_max 10^{0,-1,-2}."""
    n = 12
    H, Ls = gi.paper_random_lindbladian(n, seed=0)
    lmax = np.abs(D.liouvillian_eigenvalues(H, Ls)).max()
    h, _ = _setup(B, H, Ls)
    Bm = np.eye(n, dtype=np.complex128) / n
    for lam in (lmax, lmax / 10, lmax / 100):
        X, info, st = B.resolvent_solve(h, lam, _cuda(Bm), B.default_opts(tol=1e-12, gmres_m=32))
        ref = D.resolvent_L(H, Ls, lam, Bm)
        err = np.abs(X.cpu().numpy() - ref).max() / np.abs(ref).max()
        print(f"lam={lam:.3e} err={err:.2e}", info)
        assert st == 0 and info["residual_max"] < 1e-12
        assert err < 1e-10
    B.lindblad_destroy(h)


@pytest.mark.parametrize("n", [33, 131])
def test_resolvent_solve_ragged_matches_matrix_free_oracle(B, n):
    """Several Sylvester blocks and GEMM tiles plus a ragged tail; non-Hermitian right-hand side."""
    H, Ls = gi.random_lindbladian(n, d=3, seed=n)
    lam = 0.2
    Bm = gi.random_operator(n, seed=5)
    h, _ = _setup(B, H, Ls)
    X, info, st = B.resolvent_solve(h, lam, _cuda(Bm), B.default_opts(tol=1e-12))
    ref, _, _ = K.resolvent_gmres(K.System(H, Ls), lam, Bm, tol=1e-13, m=30, k_recycle=8)
    assert st == 0
    assert np.abs(X.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
    B.lindblad_destroy(h)


def test_resolvent_solve_mixed_precision(B):
    n = 200
    H, Ls = gi.random_lindbladian(n, d=4, seed=1)
    h, _ = _setup(B, H, Ls)
    Bm = _cuda(np.eye(n, dtype=np.complex128) / n)
    X64, i64, s64 = B.resolvent_solve(h, 0.05, Bm, B.default_opts(tol=1e-13))
    Xmx, imx, smx = B.resolvent_solve(h, 0.05, Bm, B.default_opts(tol=1e-13, precision=B.LB_PREC_MIXED))
    print("fp64", i64, "mixed", imx)
    assert s64 == 0 and smx == 0
    err = float((Xmx - X64).abs().max() / X64.abs().max())
    assert err < 1e-9
    B.lindblad_destroy(h)


@pytest.mark.parametrize("Kerr", [0.0, 8.0])
def test_implicit_euler_matches_dense(B, Kerr):
    """Sec. 4.3's stiff family (n = 32 dense random + K N^2): the trajectory of 12 steps agrees with
    the dense (Id - dt L)^{-1} iteration."""
    n = 32
    H, Ls = gi.stiff_random_lindbladian(n, K=Kerr, seed=0)
    rho0 = np.zeros((n, n), dtype=np.complex128)
    rho0[0, 0] = 1.0
    dt, steps = 0.02, 12
    ref = D.implicit_euler(H, Ls, rho0, dt, steps)
    h, _ = _setup(B, H, Ls)
    rho, traj, info, st = B.implicit_euler(h, _cuda(rho0), dt, steps, B.default_opts(tol=1e-12), trajectory=True)
    print(Kerr, info)
    assert st == 0
    traj = traj.cpu().numpy()
    for a, r in zip(traj, ref):
        assert np.abs(a - r).max() < 1e-10
    assert np.abs(rho.cpu().numpy() - ref[-1]).max() < 1e-10
    assert abs(np.trace(traj[-1]) - 1.0) < 1e-12
    B.lindblad_destroy(h)


def test_gauge_split_three_level_printed_spectrum(B, golden):
    """Conclusion: with c = (1, 0, 0) the map Phi~ of the gauge-shifted split keeps 1 simple, maps the
    pair exp(+-2 pi i / 3) to 1/2 +- i / (2 sqrt 2) and every other eigenvalue inside sqrt(3/8).
    Phi~ is applied by the library to the 9 matrix units and its spectrum taken on the host."""
    kv, _ = golden("three_level_gauge.txt")
    H, Ls = gi.three_level_cycle()
    c = np.array(kv["c"], dtype=np.complex128)
    cbuf = np.ascontiguousarray(np.stack([c.real, c.imag], axis=1).reshape(-1))
    opts = B.default_opts()
    opts.gauge_c = cbuf.ctypes.data_as(__import__("ctypes").POINTER(__import__("ctypes").c_double))
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)), opts)
    Phi = np.zeros((9, 9), dtype=np.complex128)
    for j in range(9):
        E = np.zeros((3, 3), dtype=np.complex128)
        E[j % 3, j // 3] = 1.0                # column-major vec
        Phi[:, j] = D.vec(B.phi_apply(h, _cuda(E)).cpu().numpy())
    ev = np.linalg.eigvals(Phi)
    i1 = np.argmin(np.abs(ev - 1))
    assert abs(ev[i1] - 1) < 1e-12
    others = np.delete(ev, i1)
    assert np.abs(others).max() <= kv["max_other_modulus"][0] + 1e-12
    for re, im in zip(kv["pair_re"], kv["pair_im"]):
        assert np.min(np.abs(others - (re + 1j * im))) < 1e-12
    # and the steady state is unchanged by the gauge: I / 3
    rho, info, st = B.steady_state(h, B.default_opts(tol=1e-13, krylov_m=6))
    assert st == 0 and np.abs(rho.cpu().numpy() - np.eye(3) / 3).max() < 1e-13
    B.lindblad_destroy(h)


def test_memory_buffer_cat_steady_state_spectrum_and_gauge(B):
    """App. B's memory-buffer cat (n_a = 9, n_b = 3): Alg. 4 and Alg. 3 against the dense LU, the
    three slowest modes (bit flip, two phase flips) against the dense eigenvalues, and a gauge
    c_j = -Tr(L_j rho_inf) (jumps centred on their steady-state mean) leaving the state unchanged."""
    H, Ls = gi.memory_buffer_cat(9, 3)
    n = H.shape[0]
    ref = D.steady_state_lu(H, Ls)
    h, _ = _setup(B, H, Ls)
    r4, i4, s4 = B.steady_state(h, B.default_opts(tol=1e-13, max_restarts=200))
    r3, i3, s3 = B.steady_state_gmres(h, B.default_opts(tol=1e-13, max_restarts=200))
    print("alg4", i4, "alg3", i3)
    assert s4 == 0 and s3 == 0
    for r, i in ((r4, i4), (r3, i3)):
        assert np.linalg.norm(r.cpu().numpy() - ref) / np.linalg.norm(ref) < _state_bar(H, Ls, i, ref)
    ev, _, info, st = B.low_spectrum(h, 3, opts=B.default_opts(tol=1e-10, krylov_m=20))
    dref = D.low_spectrum(H, Ls, 3)
    assert st == 0, info
    for r in dref:
        assert np.min(np.abs(ev.numpy() - r)) <= 1e-8 * abs(r)
    B.lindblad_destroy(h)
    c = np.array([-np.trace(L @ ref) for L in Ls])
    cbuf = np.ascontiguousarray(np.stack([c.real, c.imag], axis=1).reshape(-1))
    import ctypes
    opts = B.default_opts(tol=1e-13, max_restarts=200)
    opts.gauge_c = cbuf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    hg = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)), opts)
    rg, ig, sg = B.steady_state(hg, opts)
    print("gauged alg4", ig)
    assert sg == 0
    assert np.linalg.norm(rg.cpu().numpy() - ref) / np.linalg.norm(ref) < _state_bar(H, Ls, ig, ref)
    B.lindblad_destroy(hg)
