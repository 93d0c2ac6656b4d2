"""Failure handling on the GPU, in forms that fault, trap or hang nothing.

* a bounded mbarrier wait of the tensor-core kernel made to run out (a stage whose loads are never
  issued, limit 50 ms): the call returns LB_CUDA_ERROR through the device error word, the kernel
  ends, and the same handle and context keep working;
* NaN / Inf inputs refused before any factorisation (LB_INVALID_ARG);
* iteration caps: LB_NOT_CONVERGED with the best iterate and the residual that belongs to it;
* a Krylov size larger than the workspace (LB_INVALID_ARG).
"""
import time

import numpy as np
import pytest
import torch

import lindblad_inputs as gi
from oracle import krylov as K

pytestmark = pytest.mark.gpu
LB_NOT_CONVERGED, LB_INVALID_ARG, LB_CUDA_ERROR = 1, -1, -2
TOL_MIXED = 2e-5          # split-FP16 jump term (as in the tensor-core parity tests)


@pytest.fixture(scope="module")
def B():
    import paper_2608_30860_b300 as B
    B.load_library()
    return B


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("stall_iteration", [0, 1, 5])
def test_bounded_wait_runs_out_and_the_context_survives(B, stall_iteration):
    n, d = 256, 2     # product (1): 4 x 2 CTAs, 12 K iterations each -- all resident at once
    H, Ls = gi.random_lindbladian(n, d=d, seed=3)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    X = gi.random_operator(n, seed=1)
    ref = K.System(H, Ls).K(X)
    B.lb_test_bounded_wait(h, stall_iteration, 50.0)
    t0 = time.time()
    with pytest.raises(B.LindbladError) as e:
        B.jump_apply(h, _cuda(X), precision=B.LB_PREC_MIXED)
    elapsed = time.time() - t0
    assert e.value.status == LB_CUDA_ERROR
    # each role gives up after 50 ms (the MMA issuer, then the producer's wait for the stalled stage)
    assert elapsed < 5.0
    # the stall was for one launch; the limit stays 50 ms and the next call is exact again
    got = B.jump_apply(h, _cuda(X), precision=B.LB_PREC_MIXED).cpu().numpy()
    assert _rel(got, ref) < TOL_MIXED
    B.lb_test_bounded_wait(h, -1, 0.0)
    phi = B.phi_apply(h, _cuda(gi.random_hermitian(n, seed=2)), precision=B.LB_PREC_MIXED)
    assert torch.isfinite(phi).all()
    B.lindblad_destroy(h)
    torch.cuda.synchronize()


def test_bounded_wait_argument_checks(B):
    H, Ls = gi.random_lindbladian(16, d=1, seed=0)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    for it, ms in ((-2, 10.0), (0, -1.0), (0, 2500.0), (0, float("nan"))):
        with pytest.raises(B.LindbladError) as e:
            B.lb_test_bounded_wait(h, it, ms)
        assert e.value.status == LB_INVALID_ARG
    B.lindblad_destroy(h)


@pytest.mark.parametrize("where,value", [("H", np.nan), ("L", np.inf), ("L", -np.inf)])
def test_non_finite_operators_are_refused(B, where, value):
    H, Ls = gi.random_lindbladian(24, d=2, seed=4)
    L = np.stack(Ls)
    if where == "H":
        H = H.copy()
        H[3, 5] = value
    else:
        L[1, 7, 2] = value
    with pytest.raises(B.LindbladError) as e:
        B.lindblad_setup(_cuda(H), _cuda(L))
    assert e.value.status == LB_INVALID_ARG


def test_non_finite_right_hand_sides_are_refused(B):
    H, Ls = gi.random_lindbladian(24, d=2, seed=4)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    Bm = gi.random_hermitian(24, seed=1)
    Bm[2, 2] = np.nan
    with pytest.raises(B.LindbladError) as e:
        B.resolvent_solve(h, 1.0, _cuda(Bm))
    assert e.value.status == LB_INVALID_ARG
    rho0 = gi.random_density(24, seed=2)
    rho0[0, 1] = np.inf
    with pytest.raises(B.LindbladError) as e:
        B.implicit_euler(h, _cuda(rho0), 0.1, 3)
    assert e.value.status == LB_INVALID_ARG
    # the handle is unharmed
    X, info, st = B.resolvent_solve(h, 1.0, _cuda(gi.random_hermitian(24, seed=1)))
    assert st == 0
    B.lindblad_destroy(h)


def test_restart_caps_return_the_best_iterate(B):
    """tol = 1e-30 cannot be met: each solver stops at its cap with LB_NOT_CONVERGED, and the residual it
    reports is the one of the state it returns (recomputed here in FP64)."""
    H, Ls = gi.random_lindbladian(48, d=3, seed=9)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    s = K.System(H, Ls)
    opts = B.default_opts(tol=1e-30, max_restarts=1)
    rho, info, st = B.steady_state(h, opts)
    assert st == LB_NOT_CONVERGED and info["restarts"] <= 1
    r = np.abs(s.L(rho.cpu().numpy())).max()
    assert abs(r - info["residual_max"]) <= 1e-6 * r + 1e-13   # FP64 rounding of the residual itself
    rho, info, st = B.steady_state_gmres(h, B.default_opts(tol=1e-30, max_restarts=2))
    assert st == LB_NOT_CONVERGED
    r = np.abs(s.L(rho.cpu().numpy())).max()
    assert abs(r - info["residual_max"]) <= 1e-6 * r + 1e-13   # FP64 rounding of the residual itself
    assert abs(np.trace(rho.cpu().numpy()) - 1) < 1e-12
    ev, _, info, st = B.low_spectrum(h, 2, opts=B.default_opts(tol=1e-30, krylov_m=12, max_restarts=1))
    assert st == LB_NOT_CONVERGED and np.isfinite(ev.numpy()).all()
    B.lindblad_destroy(h)


def test_krylov_size_beyond_the_workspace_is_refused(B):
    H, Ls = gi.random_lindbladian(16, d=1, seed=0)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    with pytest.raises(B.LindbladError) as e:
        B.steady_state_gmres(h, B.default_opts(gmres_m=1000))
    assert e.value.status == LB_INVALID_ARG
    with pytest.raises(B.LindbladError) as e:
        B.low_spectrum(h, 2, opts=B.default_opts(krylov_m=1000))
    assert e.value.status == LB_INVALID_ARG
    B.lindblad_destroy(h)
