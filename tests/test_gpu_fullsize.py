"""Parity at the benchmark's full size: 12-site TFIM, n = 4096, d = 12, mixed precision, the same
set-up and kernels bench.py times.

The dense oracle cannot run at n = 4096, so the checks are (i) sampled entries computed one by one
by the oracle from the definition (oracle.dense.jump_term_entries / G_rows: the TFIM decay jumps are
stored dense but have one nonzero per row and column), and (ii) properties that hold at any size,
recomputed independently of the library: Phi is trace preserving and maps Hermitian to Hermitian
(App. C), M(X) = -S^{-1} K(X) satisfies G W + W G^dag + K(X) = 0 (Eqs. (2)-(3)), and the refined
steady state has ||L(rho)||_max < 1e-10 (torch FP64 matmuls).  Bars: the jump term's second GEMM
accumulates K = d n = 49152 products in FP32, so its bound (3 * 2^-22 + K * 2^-24) per GEMM, twice,
is 5.9e-3 here (the n <= 512 tests of test_gpu_mixed.py use 2e-5 at K <= 2048; measured 3.6e-4 at
n = 4096); 2e-3 for the mixed Sylvester solve, as in test_gpu_mixed.py; 1e-10 for the refined state.
"""
import numpy as np
import pytest
import torch

import lindblad_inputs as gi
from oracle import dense as D

pytestmark = pytest.mark.gpu
N, D_JUMPS = 4096, 12
TOL_JUMP = 2 * (3 * 2.0 ** -22 + D_JUMPS * N * 2.0 ** -24)
TOL_SYLV = 2e-3


@pytest.fixture(scope="module")
def tfim12():
    import paper_2608_30860_b300 as B
    H, Ls = gi.tfim(12, J=1.0, h=1.0, gamma=0.3)
    Hd = torch.from_numpy(H).cuda()
    Ld = torch.from_numpy(np.stack(Ls)).cuda()
    h = B.lindblad_setup(Hd, Ld, B.default_opts(precision=B.LB_PREC_MIXED))
    yield B, H, Ls, Hd, Ld, h
    B.lindblad_destroy(h)


def _pairs(n, count, seed):
    rng = np.random.default_rng(seed)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(count, 2))]
    return pairs + [(a, a) for a in rng.integers(0, n, size=16).tolist()]


def test_jump_term_sampled_entries_n4096(tfim12):
    B, H, Ls, Hd, Ld, h = tfim12
    n = H.shape[0]
    X = gi.random_operator(n, seed=21)
    Y = B.jump_apply(h, torch.from_numpy(X).cuda(), precision=B.LB_PREC_MIXED).cpu().numpy()
    pairs = _pairs(n, 400, 1)
    ref = D.jump_term_entries(Ls, X, pairs)
    got = np.array([Y[a, b] for a, b in pairs])
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    print(f"n=4096 mixed jump term, sampled rel err {err:.2e}")
    assert err < TOL_JUMP


def test_phi_schur_mixed_trace_and_hermiticity_n4096(tfim12):
    """The benchmark's step: Phi~ in Schur coordinates, mixed precision, Hermitian input."""
    B, H, Ls, Hd, Ld, h = tfim12
    n = H.shape[0]
    X = torch.from_numpy(gi.random_hermitian(n, seed=1)).cuda()
    X = X / torch.linalg.matrix_norm(X)
    Y = B.phi_apply(h, X, schur=True, precision=B.LB_PREC_MIXED)
    ymax = float(Y.abs().max())
    tr_err = abs(complex(torch.trace(Y) - torch.trace(X))) / abs(complex(torch.trace(X)))
    herm_err = float((Y - Y.conj().T).abs().max()) / ymax
    print(f"n=4096 mixed Phi~: trace rel err {tr_err:.2e}, hermiticity {herm_err:.2e}")
    assert tr_err < TOL_SYLV
    assert herm_err < TOL_SYLV


def test_M_form_lyapunov_identity_sampled_n4096(tfim12):
    """W = M(X) = -S^{-1} K(X) in the original basis: (G W + W G^dag + K(X))_ab = 0 on sampled
    entries, with G's rows and K(X)'s entries from the oracle."""
    B, H, Ls, Hd, Ld, h = tfim12
    n = H.shape[0]
    X = gi.random_hermitian(n, seed=3)
    W = B.phi_apply(h, torch.from_numpy(X).cuda(), form="M", precision=B.LB_PREC_MIXED).cpu().numpy()
    rng = np.random.default_rng(4)
    rows = sorted(set(rng.integers(0, n, size=24).tolist()))
    cols = sorted(set(rng.integers(0, n, size=24).tolist()))
    Grow = D.G_rows(H, Ls, rows)
    Gcol = D.G_rows(H, Ls, cols)
    pairs = [(a, b) for a in rows for b in cols]
    KX = D.jump_term_entries(Ls, X, pairs)
    res = np.empty(len(pairs), dtype=np.complex128)
    for t, (a, b) in enumerate(pairs):
        ia, ib = rows.index(a), cols.index(b)
        res[t] = Grow[ia] @ W[:, b] + W[a, :] @ np.conj(Gcol[ib]) + KX[t]
    err = np.abs(res).max() / np.abs(KX).max()
    print(f"n=4096 mixed M: sampled Lyapunov identity rel err {err:.2e}")
    assert err < TOL_SYLV


def test_mixed_steady_state_residual_n4096(tfim12):
    """The mixed solve (tensor-core Phi-Arnoldi + FP64 refinement) reaches ||L(rho)||_max < 1e-10,
    recomputed with torch FP64 matmuls from H and L; the state is Hermitian, trace 1, PSD."""
    B, H, Ls, Hd, Ld, h = tfim12
    rho, info, st = B.steady_state(h, B.default_opts(precision=B.LB_PREC_MIXED, tol=1e-10))
    assert st == 0, info
    G = -1j * Hd
    for j in range(Ld.shape[0]):
        G = G - 0.5 * (Ld[j].conj().T @ Ld[j])
    R = G @ rho + rho @ G.conj().T
    for j in range(Ld.shape[0]):
        R = R + Ld[j] @ rho @ Ld[j].conj().T
    res = float(R.abs().max())
    print(f"n=4096 mixed steady state: library residual {info['residual_max']:.2e}, recomputed {res:.2e}")
    assert res < 1e-10
    assert abs(complex(torch.trace(rho)) - 1.0) < 1e-12
    assert float((rho - rho.conj().T).abs().max()) < 1e-13
    assert float(torch.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min()) > -1e-10
