"""GPU parity of the tensor-core (tcgen05) path.

The split-FP16 operand format keeps ~22 significant bits per entry (hi + lo, each 11 bits)
relative to a per-matrix power-of-two scale, and the products accumulate in FP32.  For one
complex GEMM with K-length k the error bound is ~ (3 * 2^-22 + k * 2^-24) * sum|a||b|; the jump
term chains two such GEMMs, so the test bar is 2e-5 relative to max|K(X)| -- well above the
~1e-6 measured -- and the FP64 refinement of the steady state closes the gap to 1e-10.
"""
import numpy as np
import pytest
import torch

import lindblad_inputs as gi
from oracle import krylov as K

pytestmark = pytest.mark.gpu
TOL_MIXED = 2e-5          # split-FP16 jump term
TOL_PHI_MIXED = 2e-3      # Phi: jump term + BF16-split Sylvester


@pytest.fixture(scope="module")
def B():
    import paper_2608_30860_b300 as B
    B.load_library()
    return B


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n,d", [(70, 3), (128, 2), (300, 4), (512, 4)])
def test_jump_term_tensor_cores_match_oracle(B, n, d):
    H, Ls = gi.random_lindbladian(n, d=d, seed=n + d)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    X = gi.random_operator(n, seed=4)
    ref = K.System(H, Ls).K(X)
    got = B.jump_apply(h, _cuda(X), precision=B.LB_PREC_MIXED).cpu().numpy()
    err = _rel(got, ref)
    print(f"n={n} d={d} mixed jump-term rel err {err:.2e}")
    assert err < TOL_MIXED
    # the FP64 path through the same entry point is exact to rounding
    got64 = B.jump_apply(h, _cuda(X), precision=B.LB_PREC_FP64).cpu().numpy()
    assert _rel(got64, ref) < 1e-12
    B.lindblad_destroy(h)


def test_jump_term_schur_coordinates_hermitian(B):
    n, d = 256, 3
    H, Ls = gi.random_lindbladian(n, d=d, seed=7)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    X = _cuda(gi.random_hermitian(n, seed=2))
    y64 = B.jump_apply(h, X, schur=True, precision=B.LB_PREC_FP64).cpu().numpy()
    ymx = B.jump_apply(h, X, schur=True, precision=B.LB_PREC_MIXED).cpu().numpy()
    assert _rel(ymx, y64) < TOL_MIXED
    B.lindblad_destroy(h)


@pytest.mark.parametrize("n", [96, 200])
def test_phi_mixed_matches_oracle(B, n):
    H, Ls = gi.random_lindbladian(n, d=3, seed=n)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    X = gi.random_hermitian(n, seed=1)
    ref = K.System(H, Ls).Phi(X)
    got = B.phi_apply(h, _cuda(X), precision=B.LB_PREC_MIXED).cpu().numpy()
    print(f"n={n} mixed Phi rel err {_rel(got, ref):.2e}")
    assert _rel(got, ref) < TOL_PHI_MIXED
    B.lindblad_destroy(h)


@pytest.mark.parametrize("n,lam", [(70, 0.0), (200, 0.0), (300, 0.5), (512, 0.0)])
def test_triangular_sylvester_tensor_cores(B, n, lam):
    """Mixed Bartels-Stewart solve: BF16 hi/lo (16 significant bits) tcgen05 block updates and FP32
    leaves.  Bar: 2e-3 relative to max|X| (16-bit operands, error grown through the back
    substitution by |T| / sep(T, -T^dag)); measured values are printed."""
    H, Ls = gi.random_lindbladian(n, d=3, seed=n)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    Y = gi.random_operator(n, seed=3)
    ref = K.System(H, Ls).resolvent_S(Y, lam)
    got = B.resolvent_apply(h, _cuda(Y), lam, precision=B.LB_PREC_MIXED).cpu().numpy()
    err = _rel(got, ref)
    print(f"n={n} lam={lam} mixed Sylvester rel err {err:.2e}")
    assert err < 2e-3
    B.lindblad_destroy(h)


@pytest.mark.parametrize("name,make", [
    ("kerr_cat_n32", lambda: gi.kerr_cat(32)),
    ("random_n160", lambda: gi.random_lindbladian(160, d=4, seed=0)),
])
def test_mixed_steady_state_refined_to_fp64(B, name, make):
    """Low-precision Phi-Arnoldi followed by FP64 residual refinement reaches ||L rho||_max <= 1e-11
    and agrees with the FP64 oracle to 1e-9 relative (the mixed-precision bar) or to the
    conditioning limit of the problem, whichever is larger."""
    from oracle import dense as D
    H, Ls = make()
    n = H.shape[0]
    if n <= 64:
        ref = D.steady_state_lu(H, Ls)
        sigma2 = np.linalg.svd(D.liouvillian(H, Ls), compute_uv=False)[-2]
    else:
        ref = K.steady_state_phi_arnoldi(K.System(H, Ls), tol=1e-13)[0]
        sigma2 = None
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    opts = B.default_opts(precision=B.LB_PREC_MIXED, tol=1e-11, max_refine=10)
    rho, info, st = B.steady_state(h, opts)
    print(name, info)
    rho = rho.cpu().numpy()
    assert st == 0, info
    assert info["residual_max"] <= 1e-11
    # a residual r determines the state only to ||r|| / sigma_2(L) (the Kerr cat's slow mode makes
    # sigma_2 ~ 2.5e-8), so the bar is 1e-9 or ten times that conditioning bound
    bar = 1e-9
    if sigma2 is not None:
        bar = max(bar, 10 * info["residual_fro"] / sigma2 / np.linalg.norm(ref))
    assert np.linalg.norm(rho - ref) / np.linalg.norm(ref) < bar
    B.lindblad_destroy(h)


def test_refinement_cap_returns_the_running_best(B):
    """max_refine = 1 with an unreachable tolerance: LB_NOT_CONVERGED (1), and the state returned is
    the best one seen, with the residual the library reports equal to the one recomputed from it."""
    H, Ls = gi.random_lindbladian(96, d=3, seed=2)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    opts = B.default_opts(precision=B.LB_PREC_MIXED, tol=1e-30, max_refine=1)
    rho, info, st = B.steady_state(h, opts)
    assert st == 1 and info["refine_steps"] == 1
    R = B.lindbladian_apply(h, rho)
    assert abs(float(R.abs().max()) - info["residual_max"]) <= 1e-3 * info["residual_max"]
    # one refinement step from the low-precision Arnoldi state already lands well below its residual
    assert info["residual_max"] < 1e-9
    B.lindblad_destroy(h)


@pytest.mark.parametrize("n", [200, 384])
def test_hermitian_flag_tensor_core_jump_term(B, n):
    """Upper-tile tcgen05 product (2) + mirror against the full product on a Hermitian input, and the
    oracle's K(X)."""
    H, Ls = gi.random_lindbladian(n, d=3, seed=n)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    X = gi.random_hermitian(n, seed=6)
    ref = K.System(H, Ls).K(X)
    kg = B.jump_apply(h, _cuda(X), precision=B.LB_PREC_MIXED).cpu().numpy()
    kh = B.jump_apply(h, _cuda(X), precision=B.LB_PREC_MIXED, hermitian=True).cpu().numpy()
    assert _rel(kh, ref) < TOL_MIXED and _rel(kh, kg) < TOL_MIXED
    Xs = _cuda(X)
    ys = B.phi_apply(h, Xs, schur=True, precision=B.LB_PREC_MIXED, hermitian=True).cpu().numpy()
    assert np.abs(ys - ys.conj().T).max() == 0.0
    B.lindblad_destroy(h)
