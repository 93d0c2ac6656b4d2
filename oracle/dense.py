"""Dense (n^2 x n^2) oracle: the plain definitions, written out.  TEST INFRASTRUCTURE ONLY.

Vectorisation is column-major: vec(X) stacks columns, so that
vec(A X B) = kron(B^T, A) vec(X) and <I|vec(X)> = vec(I)^T vec(X) = Tr X.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------------------- vec helpers
def vec(X: np.ndarray) -> np.ndarray:
    return np.asarray(X).reshape(-1, order="F")


def unvec(x: np.ndarray, n: int) -> np.ndarray:
    return np.asarray(x).reshape(n, n, order="F")


def sandwich(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Matrix of the superoperator X -> A X B."""
    return np.kron(B.T, A)


def dag(A):
    return A.conj().T


# ----------------------------------------------------------------------------- generator pieces
def G_matrix(H, Ls):
    """G = -iH - 1/2 sum_j L_j^dag L_j  (Eq. (3), Sec. 1.2)."""
    G = -1j * np.asarray(H, dtype=np.complex128)
    for L in Ls:
        G = G - 0.5 * (dag(L) @ L)
    return G


def liouvillian(H, Ls):
    """Dense L of Eq. (1): -i[H, rho] + sum_j (L_j rho L_j^dag - 1/2 {L_j^dag L_j, rho})."""
    n = H.shape[0]
    I = np.eye(n, dtype=np.complex128)
    Lv = -1j * (sandwich(H, I) - sandwich(I, H))
    for L in Ls:
        LdL = dag(L) @ L
        Lv = Lv + sandwich(L, dag(L)) - 0.5 * (sandwich(LdL, I) + sandwich(I, LdL))
    return Lv


def S_super(G):
    """No-jump generator S(X) = G X + X G^dag (Eq. (2))."""
    n = G.shape[0]
    I = np.eye(n, dtype=np.complex128)
    return sandwich(G, I) + sandwich(I, dag(G))


def K_super(Ls):
    """Jump generator K(X) = sum_j L_j X L_j^dag (Eq. (2))."""
    n = Ls[0].shape[0]
    out = np.zeros((n * n, n * n), dtype=np.complex128)
    for L in Ls:
        out = out + sandwich(L, dag(L))
    return out


def Phi_super(H, Ls):
    """Phi = -K S^{-1} (Sec. 2.2, Theorem 1)."""
    G = G_matrix(H, Ls)
    return -K_super(Ls) @ np.linalg.inv(S_super(G))


def M_super(H, Ls):
    """M = -S^{-1} K, similar to Phi (proof of Theorem 1)."""
    G = G_matrix(H, Ls)
    return -np.linalg.solve(S_super(G), K_super(Ls))


def resolvent_S(G, lam):
    """No-jump resolvent R_lam^S = (lam - S)^{-1} (Eq. of Sec. 3.1)."""
    n = G.shape[0]
    return np.linalg.inv(lam * np.eye(n * n) - S_super(G))


def deflation_term(n):
    """Matrix of rho -> Tr(rho) I, i.e. |I><I| in column-major vec: the deflation term of
    Eq. steady_state_linear_problem."""
    v = vec(np.eye(n, dtype=np.complex128))
    return np.outer(v, v)


def deflated_liouvillian(H, Ls, eta=1.0):
    """L~_eta = L + eta Tr(.) I (Eq. steady_state_linear_problem)."""
    n = H.shape[0]
    return liouvillian(H, Ls) + eta * deflation_term(n)


def precond_alg2(G, lam, c, X):
    """Alg. 2 applied to X with dense resolvents: Z + c Tr Z/(1 - c Tr W) W."""
    n = G.shape[0]
    R = resolvent_S(G, lam)
    Z = unvec(R @ vec(X), n)
    W = unvec(R @ vec(np.eye(n, dtype=np.complex128)), n)
    return Z + c * np.trace(Z) / (1.0 - c * np.trace(W)) * W


def deflated_noJump_inverse(G, lam, c):
    """((lam - S) - c |I><I|)^{-1}, the operator Alg. 2 inverts exactly (Eq. ShermanMorr)."""
    n = G.shape[0]
    return np.linalg.inv(lam * np.eye(n * n) - S_super(G) - c * deflation_term(n))


# ----------------------------------------------------------------------------- single entries
def _row_support(M, i):
    nz = np.nonzero(M[i])[0]
    return nz, M[i, nz]


def jump_term_entries(Ls, X, pairs):
    """Selected entries of K(X) = sum_j L_j X L_j^dag (Eq. (2)) straight from the definition,
    K(X)_ab = sum_j sum_{k,l} L_j[a,k] X[k,l] conj(L_j[b,l]), summing over the nonzeros of rows a
    and b of each L_j (cheap for sparse jumps stored dense, exact for any)."""
    out = np.zeros(len(pairs), dtype=np.complex128)
    for j, L in enumerate(Ls):
        rows = {}
        for t, (a, b) in enumerate(pairs):
            for r in (a, b):
                if r not in rows:
                    rows[r] = _row_support(L, r)
            ka, va = rows[a]
            kb, vb = rows[b]
            if len(ka) and len(kb):
                out[t] += va @ X[np.ix_(ka, kb)] @ np.conj(vb)
    return out


def G_rows(H, Ls, idx):
    """Rows idx of G = -iH - 1/2 sum_j L_j^dag L_j (Eq. (2)); (L^dag L)[a, :] = sum_m conj(L[m, a]) L[m, :]
    over the nonzeros of column a of L."""
    out = -1j * np.asarray(H[idx], dtype=np.complex128)
    for L in Ls:
        for t, a in enumerate(idx):
            ms = np.nonzero(L[:, a])[0]
            if len(ms):
                out[t] -= 0.5 * (np.conj(L[ms, a]) @ L[ms])
    return out


# ----------------------------------------------------------------------------- steady state
def hermitize_normalize(rho):
    """(rho + rho^dag) / 2 divided by its trace: the reconstruction step of Alg. 4."""
    r = 0.5 * (rho + dag(rho))
    return r / np.trace(r).real


def steady_state_lu(H, Ls, eta=1.0):
    """rho_inf from the deflated linear system L~_eta rho = eta I by LU (Eq. steady_state_linear_problem)."""
    n = H.shape[0]
    A = deflated_liouvillian(H, Ls, eta)
    b = eta * vec(np.eye(n, dtype=np.complex128))
    x = sla.solve(A, b)
    return hermitize_normalize(unvec(x, n))


def steady_state_svd(H, Ls):
    """rho_inf as the right singular vector of L for its smallest singular value (the null vector of the
    Lindbladian of Eq. lindblad_def; cross-check of the deflated solve)."""
    n = H.shape[0]
    _, s, Vh = np.linalg.svd(liouvillian(H, Ls))
    x = Vh[-1].conj()
    return hermitize_normalize(unvec(x, n)), s


# ----------------------------------------------------------------------------- spectra
def liouvillian_eigenvalues(H, Ls):
    """All eigenvalues of the dense Lindbladian of Eq. lindblad_def."""
    return sla.eigvals(liouvillian(H, Ls))


def low_spectrum(H, Ls, k, zero_tol=None):
    """The k smallest-|lambda| nonzero eigenvalues of L (Sec. 4.2), sorted by
    |lambda|, then Re descending, then Im ascending.

    The single eigenvalue of smallest modulus is the steady-state zero mode and is
    dropped (the Lindbladians used here have a one-dimensional kernel)."""
    ev = liouvillian_eigenvalues(H, Ls)
    order = np.argsort(np.abs(ev))
    ev = ev[order][1:]
    key = np.lexsort((ev.imag, -ev.real, np.round(np.abs(ev), 12)))
    return ev[key][:k]


def low_spectrum_with_vectors(H, Ls, k):
    """k smallest-|lambda| nonzero eigenpairs (values, list of n x n eigenvectors): the low-lying spectrum
    of Sec. 4.2 by dense eigendecomposition."""
    n = H.shape[0]
    ev, V = sla.eig(liouvillian(H, Ls))
    order = np.argsort(np.abs(ev))[1:k + 1]
    return ev[order], [unvec(V[:, i], n) for i in order]


# ----------------------------------------------------------------------------- gauge, resolvent, Euler
def gauge_split(H, Ls, c):
    """The gauge of Remark 'Non-uniqueness of the decomposition' (Eqs. lindblad_gauge and
    lindblad_gauge_2): L~_j = L_j + c_j I and H~ = H + (1/2i) sum_j (c_j^* L~_j - c_j L~_j^dag).
    The Lindbladian built from (H~, L~) is the same; its no-jump / jump split is not."""
    n = H.shape[0]
    I = np.eye(n, dtype=np.complex128)
    Lt = [np.asarray(L, dtype=np.complex128) + cj * I for L, cj in zip(Ls, c)]
    Ht = np.asarray(H, dtype=np.complex128) + sum(np.conj(cj) * L - cj * dag(L) for L, cj in zip(Lt, c)) / 2j
    return Ht, Lt


def resolvent_L(H, Ls, lam, B):
    """R_lam^L(B) = (lam - L)^{-1}(B) by LU of the dense n^2 x n^2 matrix (Sec. 3.3, Corollary
    'Resolvent of the Lindbladian'; the solve of the resolvent benchmarks, Sec. 3.4)."""
    n = H.shape[0]
    A = lam * np.eye(n * n, dtype=np.complex128) - liouvillian(H, Ls)
    return unvec(sla.solve(A, vec(B)), n)


def implicit_euler(H, Ls, rho0, dt, steps):
    """Implicit Euler (Eq. resolvent, Sec. 4.3): rho_{t+dt} = (Id - dt L)^{-1} rho_t, the dense
    n^2 x n^2 matrix factorised once; returns the states after each of the `steps` steps."""
    n = H.shape[0]
    A = np.eye(n * n, dtype=np.complex128) - dt * liouvillian(H, Ls)
    lu = sla.lu_factor(A)
    out, x = [], vec(np.asarray(rho0, dtype=np.complex128))
    for _ in range(steps):
        x = sla.lu_solve(lu, x)
        out.append(unvec(x, n).copy())
    return out


# ----------------------------------------------------------------------------- adjoint gradient
def steady_state_gradient(H_of_theta, Ls_of_theta, dL_super_of_theta, theta, O, eta=1.0):
    """Implicit differentiation of J = Tr(O rho_inf) (Remark 'Differentiating the steady state').

    Solves L~_eta^* w = O (dense adjoint = conjugate transpose) and returns
    dJ/dtheta_i = -Re <w, (d_i L~_eta) rho_inf> with <A, B> = Tr(A^dag B) = vec(A)^H vec(B).
    ``dL_super_of_theta(theta)`` returns the list of dense d_i L matrices.
    """
    H = H_of_theta(theta)
    Ls = Ls_of_theta(theta)
    n = H.shape[0]
    A = deflated_liouvillian(H, Ls, eta)
    b = eta * vec(np.eye(n, dtype=np.complex128))
    x = sla.solve(A, b)                # un-normalised solution; trace is 1 by construction
    w = sla.solve(dag(A), vec(O))
    grads = []
    for dL in dL_super_of_theta(theta):
        grads.append(-np.real(np.vdot(w, dL @ x)))
    return np.array(grads), hermitize_normalize(unvec(x, n))


# ----------------------------------------------------------------------------- misc
def choi(superop, n):
    """Choi matrix sum_ij |i><j| (x) E(|i><j|) of a superoperator given as a dense matrix (its positive
    semidefiniteness is the complete positivity of Theorem 1)."""
    C = np.zeros((n * n, n * n), dtype=np.complex128)
    for i in range(n):
        for j in range(n):
            Eij = np.zeros((n, n), dtype=np.complex128)
            Eij[i, j] = 1.0
            out = unvec(superop @ vec(Eij), n)
            C += np.kron(Eij, out)
    return C


def superop_adjoint_apply(superop, X, n):
    """E^*(X) for the Hilbert-Schmidt inner product (the superoperator adjoint of Sec. 1.2's notation):
    the conjugate-transpose matrix."""
    return unvec(dag(superop) @ vec(X), n)


def cp_trace_norm(superop, n):
    """Induced trace norm of a CP map = ||E^*(I)||_inf (Russo-Dye, proof of Theorem 2)."""
    E = superop_adjoint_apply(superop, np.eye(n, dtype=np.complex128), n)
    E = 0.5 * (E + dag(E))
    return np.max(np.abs(np.linalg.eigvalsh(E)))
