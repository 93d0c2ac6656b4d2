"""Parity at the configured workloads' own sizes (the Kerr cat at n = 32 and the random Lindbladian at
n = 512), and the mixed-precision shift-invert path, through the C ABI.

* Kerr cat, n = 32, d = 2: the 4 smallest-|lambda| nonzero eigenvalues by shift-invert Arnoldi
  (Alg. 5) against the dense 1024 x 1024 Lindbladian's eigenvalues, 1e-8 relative, plus the
  eigen-residual ||L v - lambda v||_max / ||v||_max < 1e-8 recomputed from the dense matrix.
* Random Lindbladian, n = 512, d = 4, seed 0: the steady state in FP64 (Alg. 4) against the
  matrix-free oracle's Alg. 4 at 1e-10 relative Frobenius, the mixed (tensor-core + FP64 refinement)
  state at 1e-9, Alg. 3 (recycled GMRES) at 1e-10, and the 8 smallest-|lambda| nonzero eigenvalues
  against the oracle's Alg. 5 (tests/golden/random_n512_d4_spectrum.txt, written by
  tests/golden/make_random_n512_spectrum.py from oracle/ only) at 1e-8 relative.
* Mixed-precision shift-invert at n = 40 (Kerr cat): tensor-core inner solves, FP64 refinement cycles,
  eigenvalues against the dense 1600 x 1600 eigenvalues at 1e-8 relative.
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


def _match(ev, ref, rel):
    for r in ref:
        assert np.min(np.abs(ev - r)) <= rel * abs(r), (r, ev)


def _eig_residual(Lm, lam, v, n):
    r = D.unvec(Lm @ D.vec(v), n) - lam * v
    return np.abs(r).max() / np.abs(v).max()


def test_config_kerr_cat_n32_four_lowest_eigenvalues(B):
    H, Ls = gi.kerr_cat(32, K=1.0, eps2=4.0, kappa2=1.0, kappa1=0.01)
    ref = D.low_spectrum(H, Ls, 4)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    opts = B.default_opts(tol=1e-10, krylov_m=24)
    ev, vecs, info, st = B.low_spectrum(h, 4, want_vectors=True, opts=opts)
    print("kerr32 k=4", ev.numpy(), info)
    assert st == 0, info
    _match(ev.numpy(), ref, 1e-8)
    Lm = D.liouvillian(H, Ls)
    for lam, v in zip(ev.numpy(), vecs.cpu().numpy()):
        assert _eig_residual(Lm, lam, v, 32) < 1e-8
    B.lindblad_destroy(h)


@pytest.fixture(scope="module")
def random512(B):
    H, Ls = gi.random_lindbladian(512, d=4, seed=0)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    ref, info = K.steady_state_phi_arnoldi(K.System(H, Ls), tol=1e-13, m=20, N=60)
    assert info["residual"] < 1e-13
    yield H, Ls, h, ref
    B.lindblad_destroy(h)


def test_config_random_n512_fp64_steady_state(B, random512):
    H, Ls, h, ref = random512
    rho, info, st = B.steady_state(h, B.default_opts(tol=1e-13))
    print("n512 fp64", info)
    assert st == 0 and info["residual_max"] < 1e-13
    assert np.linalg.norm(rho.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_config_random_n512_mixed_steady_state(B, random512):
    H, Ls, h, ref = random512
    rho, info, st = B.steady_state(h, B.default_opts(tol=1e-11, precision=B.LB_PREC_MIXED))
    print("n512 mixed", info)
    assert st == 0 and info["residual_max"] < 1e-11
    assert np.linalg.norm(rho.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-9


def test_config_random_n512_alg3_steady_state(B, random512):
    H, Ls, h, ref = random512
    rho, info, st = B.steady_state_gmres(h, B.default_opts(tol=1e-13, gmres_m=32, recycle_k=8))
    print("n512 alg3", info)
    assert st == 0 and info["residual_max"] < 1e-13
    assert np.linalg.norm(rho.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_config_random_n512_eight_lowest_eigenvalues(B, random512, golden):
    H, Ls, h, _ = random512
    kv, _ = golden("random_n512_d4_spectrum.txt")
    ref = np.array(kv["re"]) + 1j * np.array(kv["im"])
    ev, _, info, st = B.low_spectrum(h, 8, opts=B.default_opts(tol=1e-9, krylov_m=24))
    print("n512 k=8", ev.numpy(), info)
    assert st == 0, info
    _match(ev.numpy(), ref, 1e-8)


def test_mixed_shift_invert_refined_matches_dense(B):
    H, Ls = gi.kerr_cat(40, eps2=4.0)
    ref = D.low_spectrum(H, Ls, 4)
    h = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)))
    opts = B.default_opts(tol=1e-10, krylov_m=24, precision=B.LB_PREC_MIXED)
    ev, vecs, info, st = B.low_spectrum(h, 4, want_vectors=True, opts=opts)
    print("mixed SI kerr40", ev.numpy(), info)
    assert st == 0, info
    _match(ev.numpy(), ref, 1e-8)
    Lm = D.liouvillian(H, Ls)
    for lam, v in zip(ev.numpy(), vecs.cpu().numpy()):
        assert _eig_residual(Lm, lam, v, 40) < 1e-9
    B.lindblad_destroy(h)
