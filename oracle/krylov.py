"""Matrix-free oracle: the paper's algorithms, unblocked, in float64.  TEST INFRASTRUCTURE ONLY.

Used where the dense n^2 x n^2 oracle cannot run (n > ~100) and as the timed
CPU baseline.  Operators are n x n complex128 arrays; the inner product is the
Hilbert-Schmidt one <A, B> = Tr(A^dag B).

Contents (paper location):
  * System.resolvent_S      -- Bartels-Stewart no-jump resolvent (App. A.1.1):
                               Schur G = Q T Q^dag, shift T -> T - lam/2,
                               triangular Sylvester by LAPACK ztrsyl.
  * System.resolvent_S_eig  -- eigendecomposition route (App. A.1.2, Alg. 1).
  * System.Phi / System.M   -- Phi = -K S^{-1} (Theorem 1), M = -S^{-1} K.
  * System.precond          -- Alg. 2 (Sherman-Morrison deflated preconditioner).
  * arnoldi                 -- Arnoldi with full (two-pass) re-orthogonalisation.
  * steady_state_phi_arnoldi-- Alg. 4.
  * gcrodr                  -- right-preconditioned GMRES with Krylov subspace recycling
                               (GCRO-DR of Parks, de Sturler, Mackey, Johnson and Maiti 2006,
                               the recycling named in App. A.2).
  * steady_state_gmres      -- Alg. 3 (restarted right-preconditioned GMRES, optionally recycled).
  * resolvent_gmres         -- (lam - L) X = B with the preconditioner R_lam^S (Sec. 3.1, 3.4).
  * implicit_euler_gmres    -- implicit Euler steps by the same solve at lam = 1/dt (Sec. 4.3).
  * low_spectrum_shift_invert -- Alg. 5 (shift-invert Arnoldi with thick restart).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from scipy.linalg import lapack


def dag(A):
    return A.conj().T


def hs_inner(A, B):
    """<A, B> = Tr(A^dag B)."""
    return np.vdot(A.reshape(-1), B.reshape(-1))


def hs_norm(A):
    return float(np.sqrt(np.real(hs_inner(A, A))))


def hermitize_normalize(rho):
    """Phase-fix by the trace, hermitize, renormalise to trace 1 (Alg. 3/4 reconstruction).

    Dividing by Tr(rho) first removes the arbitrary complex phase of a Ritz
    vector; then rho_hat = (rho + rho^dag)/2 and rho_hat /= Tr rho_hat."""
    r = rho / np.trace(rho)
    r = 0.5 * (r + dag(r))
    return r / np.trace(r).real


class System:
    """One Lindbladian (H, {L_j}) with its no-jump / jump split (Eqs. (2)-(3))."""

    def __init__(self, H, Ls, route="schur"):
        self.H = np.asarray(H, dtype=np.complex128)
        self.Ls = [np.asarray(L, dtype=np.complex128) for L in Ls]
        self.n = self.H.shape[0]
        self.G = -1j * self.H
        for L in self.Ls:
            self.G = self.G - 0.5 * (dag(L) @ L)
        self.route = route
        self._schur = None
        self._eig = None
        self._W = {}

    # -- Schur / eigen factors, computed once (App. A.1) ----------------------
    @property
    def schur(self):
        if self._schur is None:
            T, Q = sla.schur(self.G, output="complex")
            self._schur = (T, Q)
        return self._schur

    @property
    def eig(self):
        if self._eig is None:
            sig, U = sla.eig(self.G)
            V = dag(np.linalg.inv(U))
            self._eig = (sig, U, V)
        return self._eig

    # -- superoperators ---------------------------------------------------------
    def K(self, X):
        """Jump part K(X) = sum_j L_j X L_j^dag (Eq. lindblad_decomposition)."""
        out = np.zeros_like(X)
        for L in self.Ls:
            out += L @ X @ dag(L)
        return out

    def S(self, X):
        """No-jump part S(X) = G X + X G^dag (Eq. lindblad_decomposition, G of Eq. G)."""
        return self.G @ X + X @ dag(self.G)

    def L(self, X):
        """Lindbladian L = S + K (Eq. (2))."""
        return self.S(X) + self.K(X)

    def L_adjoint(self, X):
        """L^*(X) = G^dag X + X G + sum_j L_j^dag X L_j (Hilbert-Schmidt adjoint; the adjoint system of the
        Remark on differentiating the steady state, Sec. 4.1)."""
        out = dag(self.G) @ X + X @ self.G
        for L in self.Ls:
            out += dag(L) @ X @ L
        return out

    def resolvent_S(self, Y, lam=0.0):
        """R_lam^S(Y) = (lam - S)^{-1}(Y) by Bartels-Stewart (App. A.1.1).

        (lam - S)X = -(G_lam X + X G_lam^dag) with G_lam = G - lam/2 I, so with
        G = Q T Q^dag the triangular equation is
        T_lam Xt + Xt T_lam^dag = -Q^dag Y Q, and X = Q Xt Q^dag."""
        if self.route == "eig":
            return self.resolvent_S_eig(Y, lam)
        T, Q = self.schur
        Tl = T - 0.5 * lam * np.eye(self.n)
        Yt = dag(Q) @ (-Y) @ Q
        Xt, scale, info = lapack.ztrsyl(Tl, Tl, Yt, trana="N", tranb="C", isgn=1)
        if info < 0:
            raise RuntimeError(f"ztrsyl failed, info={info}")
        Xt = Xt / scale
        return Q @ Xt @ dag(Q)

    def resolvent_S_eig(self, Y, lam=0.0):
        """R_lam^S(Y) = U[(V^dag Y V)_ij / (lam - sigma_i - conj(sigma_j))]U^dag (Alg. 1)."""
        sig, U, V = self.eig
        Yh = dag(V) @ Y @ V
        D = lam - sig[:, None] - sig.conj()[None, :]
        return U @ (Yh / D) @ dag(U)

    def S_inv(self, Y):
        """S^{-1} = -R_0^S (Sec. 3.1)."""
        return -self.resolvent_S(Y, 0.0)

    def Phi(self, xi):
        """Phi(xi) = -K(S^{-1} xi) (Theorem 1)."""
        return -self.K(self.S_inv(xi))

    def M(self, rho):
        """M(rho) = -S^{-1}(K rho) (proof of Theorem 1)."""
        return -self.S_inv(self.K(rho))

    def W(self, lam):
        """W = R_lam^S(I), precomputed once per shift (Alg. 2)."""
        if lam not in self._W:
            self._W[lam] = self.resolvent_S(np.eye(self.n, dtype=np.complex128), lam)
        return self._W[lam]

    def precond(self, X, lam, c):
        """Alg. 2: Z = R(X); return Z + c Tr Z / (1 - c Tr W) W."""
        Z = self.resolvent_S(X, lam)
        W = self.W(lam)
        denom = 1.0 - c * np.trace(W)
        return Z + (c * np.trace(Z) / denom) * W

    def shifted_deflated(self, X, mu, eta):
        """(mu - L~_eta)(X) = mu X - L(X) - eta Tr(X) I: the deflated operator of
        Eq. steady_state_linear_problem, shifted as in Alg. 5."""
        return mu * X - self.L(X) - eta * np.trace(X) * np.eye(self.n)


# ----------------------------------------------------------------------------- Arnoldi
def arnoldi(op, v0, m, breakdown_tol=1e-14):
    """m Arnoldi steps with full two-pass Gram-Schmidt re-orthogonalisation.

    Returns (V, Hm, k): V list of k+1 orthonormal operators, Hm the (k+1) x k
    upper-Hessenberg matrix with op(V[:k]) = V Hm; k < m only on breakdown."""
    beta = hs_norm(v0)
    V = [v0 / beta]
    Hm = np.zeros((m + 1, m), dtype=np.complex128)
    for k in range(m):
        w = op(V[k])
        for _ in range(2):
            for i in range(k + 1):
                h = hs_inner(V[i], w)
                Hm[i, k] += h
                w = w - h * V[i]
        hn = hs_norm(w)
        Hm[k + 1, k] = hn
        if hn <= breakdown_tol * max(1.0, np.abs(Hm[: k + 1, k]).max()):
            return V, Hm[: k + 2, : k + 1], k + 1
        V.append(w / hn)
    return V, Hm, m


def _pick_nearest_one(theta):
    """Index of the Ritz value nearest 1; ties -> larger Re -> smaller index."""
    d = np.abs(theta - 1.0)
    best = 0
    for i in range(1, len(theta)):
        if d[i] < d[best] - 1e-15 or (abs(d[i] - d[best]) <= 1e-15 and theta[i].real > theta[best].real):
            best = i
    return best


def steady_state_phi_arnoldi(sysm: System, tol=1e-10, m=20, N=50, xi0=None):
    """Alg. 4: explicitly restarted Arnoldi on Phi.

    Each cycle keeps the Ritz vector xi with Ritz value nearest 1, reconstructs
    rho = -S^{-1} xi, hermitises and trace-normalises it, stops when
    ||L(rho_hat)||_max < tol, else restarts from xi; returns the running best.
    Start vector (not fixed by the paper): I/n."""
    n = sysm.n
    xi = np.eye(n, dtype=np.complex128) / n if xi0 is None else xi0.copy()
    best, best_res = None, np.inf
    hist = []
    applies = 0
    for _ in range(N):
        V, Hm, k = arnoldi(sysm.Phi, xi, m)
        applies += k
        theta, Y = np.linalg.eig(Hm[:k, :k])
        i = _pick_nearest_one(theta)
        y = Y[:, i]
        xi = sum(y[t] * V[t] for t in range(k))
        rho = -sysm.S_inv(xi)
        rho_hat = hermitize_normalize(rho)
        res = float(np.abs(sysm.L(rho_hat)).max())
        hist.append(res)
        if res < best_res:
            best, best_res = rho_hat, res
        if res < tol:
            break
        xi = xi / np.trace(xi)
    return best, dict(residual=best_res, history=hist, applies=applies, ritz=theta[i])


# ----------------------------------------------------------------------------- GMRES
def gmres_right(matvec, precond, b, x0, m=30, restarts=50, atol=1e-12, cycle_hook=None):
    """Restarted GMRES(m) with right preconditioning: A P y = r0, x = x0 + P y.

    The least-squares problem is solved on the small Hessenberg by lstsq.
    ``cycle_hook(x)`` may return True to stop early (Alg. 3's state test)."""
    x = x0.copy()
    for _ in range(restarts):
        r = b - matvec(x)
        beta = hs_norm(r)
        if beta <= atol:
            break
        V, Hm, k = arnoldi(lambda v: matvec(precond(v)), r, m)
        e1 = np.zeros(k + 1, dtype=np.complex128)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(Hm[: k + 1, :k], e1, rcond=None)
        upd = sum(y[t] * V[t] for t in range(k))
        x = x + precond(upd)
        if cycle_hook is not None and cycle_hook(x):
            break
    return x


def _gs_qr(vectors):
    """QR of a list of operators by Gram-Schmidt applied twice: (Q list, R upper triangular)."""
    k = len(vectors)
    Q, R = [], np.zeros((k, k), dtype=np.complex128)
    for j, v in enumerate(vectors):
        w = v.copy()
        for _ in range(2):
            for i, q in enumerate(Q):
                h = hs_inner(q, w)
                R[i, j] += h
                w = w - h * q
        R[j, j] = hs_norm(w)
        Q.append(w / R[j, j])
    return Q, R


def _combine(basis, coeffs):
    out = np.zeros_like(basis[0])
    for c, v in zip(coeffs, basis):
        out = out + c * v
    return out


def gcrodr(matvec, precond, b, x0, m=32, k=8, recycle=None, atol=0.0, max_cycles=50, cycle_hook=None):
    """GCRO-DR(m, k) with right preconditioning (Parks et al. 2006; App. A.2's recycled GMRES).

    Solves A x = b through the operator B = A P (x = x0 + P y).  A recycled pair (U, C) with
    B U = C, C orthonormal, enters every cycle: the Arnoldi process runs on (I - C C^H) B for
    m - k steps, giving B [U D, V_p] = [C, V_{p+1}] G with G = [[D, C^H B V_p], [0, Hbar]]
    (D scales U to unit columns); y minimises ||[C, V_{p+1}]^H r - G y||.  After each cycle the
    k harmonic Ritz vectors of B on range([U D, V_p]) with the smallest harmonic Ritz values,
    i.e. G^H G z = theta G^H [C, V_{p+1}]^H [U D, V_p] z, become the new (U, C) through the small QR
    G Z = Q R (C = [C, V_{p+1}] Q, U = [U D, V_p] Z R^{-1}); the problem is posed on an orthonormal basis
    of range([U D, V_p]); the pair is kept unchanged when R is ill-conditioned (pivots below 1e-6 of
    the largest) or when the cycle met the tolerance.
    ``recycle`` = (U, C) of an earlier solve with the same operator (kept as is); the returned
    pair is to be passed to the next solve.  ``cycle_hook(x)`` returning True stops early."""
    x = np.array(x0, dtype=np.complex128)
    r = b - matvec(x)
    U = C = None
    if recycle is not None and recycle[0]:
        U = [u.copy() for u in recycle[0]]
        C = [c.copy() for c in recycle[1]]
        coef = [hs_inner(c, r) for c in C]
        x = x + precond(_combine(U, coef))
        r = r - _combine(C, coef)
    cycles = steps = 0
    while cycles < max_cycles:
        beta = hs_norm(r)
        if beta <= atol:
            break
        kk = len(U) if U else 0
        p = m - kk
        V = [r / beta]
        Hb = np.zeros((p + 1, p), dtype=np.complex128)
        Bm = np.zeros((kk, p), dtype=np.complex128)
        done = p
        for j in range(p):
            w = matvec(precond(V[j]))
            steps += 1
            for _ in range(2):
                for i in range(kk):
                    h = hs_inner(C[i], w)
                    Bm[i, j] += h
                    w = w - h * C[i]
                for i in range(j + 1):
                    h = hs_inner(V[i], w)
                    Hb[i, j] += h
                    w = w - h * V[i]
            hn = hs_norm(w)
            Hb[j + 1, j] = hn
            if hn <= 1e-14 * max(1.0, np.abs(Hb[: j + 1, j]).max()):
                done = j + 1
                V.append(np.zeros_like(w))
                break
            V.append(w / hn)
        p = done
        Hb, Bm, V = Hb[: p + 1, :p], Bm[:, :p], V[: p + 1]
        dn = np.array([1.0 / hs_norm(u) for u in U]) if kk else np.zeros(0)
        Ut = [u * dv for u, dv in zip(U, dn)] if kk else []
        G = np.zeros((kk + p + 1, kk + p), dtype=np.complex128)
        G[:kk, :kk] = np.diag(dn)
        G[:kk, kk:] = Bm
        G[kk:, kk:] = Hb
        rhs = np.zeros(kk + p + 1, dtype=np.complex128)
        rhs[kk] = beta
        y, *_ = np.linalg.lstsq(G, rhs, rcond=None)
        What = Ut + V[:p]
        Vhat = (C if kk else []) + V
        x = x + precond(_combine(What, y))
        r = _combine(Vhat, rhs - G @ y)
        cycles += 1
        # new recycled pair: the harmonic Ritz vectors of smallest |theta|, taken on an orthonormal
        # basis [U D, V_p] S of range([U D, V_p]) (S from the eigenpairs of its Gram matrix above 1e-10 of
        # the largest: once a cycle has nearly converged [U D, V_p] is numerically rank-deficient and its
        # null directions would pass for spurious harmonic Ritz vectors), as the Schur vectors of the
        # selected values; then the small QR G Z = Q R gives C = [C, V_{p+1}] Q, U = [U D, V_p] Z R^{-1}
        F = np.zeros((kk + p + 1, kk + p), dtype=np.complex128)
        Gam = np.eye(kk + p, dtype=np.complex128)
        for j in range(kk):
            for i in range(kk):
                F[i, j] = hs_inner(C[i], Ut[j])
                Gam[i, j] = hs_inner(Ut[i], Ut[j])
            for i in range(p + 1):
                F[kk + i, j] = hs_inner(V[i], Ut[j])
            for i in range(p):
                Gam[kk + i, j] = F[kk + i, j]
                Gam[j, kk + i] = np.conj(F[kk + i, j])
        F[kk:, kk:] = np.eye(p + 1, p)
        lam, E = np.linalg.eigh(Gam)
        keepg = lam > 1e-10 * lam.max()
        S = E[:, keepg] / np.sqrt(lam[keepg])
        GS = G @ S
        Qg, Rg = np.linalg.qr(GS)
        Mh = np.linalg.solve(Rg, Qg.conj().T @ (F @ S))      # eigenvalues 1 / theta
        kq = min(k, Mh.shape[0])
        mu = np.linalg.eigvals(Mh)
        thr = np.sort(np.abs(mu))[-kq] * (1.0 - 1e-12)
        _, Ys, sdim = sla.schur(Mh, output="complex", sort=lambda z: abs(z) >= thr)
        Z = S @ Ys[:, :min(sdim, kq)]
        Qs, Rs = np.linalg.qr(G @ Z)
        dg = np.abs(np.diag(Rs))
        # a cycle that met the tolerance keeps the pair: the end of a converged Krylov space is rounding
        # noise, and each update multiplies the pair's relation error by ||R^{-1}||
        if dg.size and dg.min() > 1e-6 * dg.max() and hs_norm(r) > atol:
            ZR = Z @ np.linalg.inv(Rs)
            C = [_combine(Vhat, Qs[:, t]) for t in range(Qs.shape[1])]
            U = [_combine(What, ZR[:, t]) for t in range(ZR.shape[1])]
        if cycle_hook is not None and cycle_hook(x):
            break
    return x, (U, C), dict(cycles=cycles, steps=steps, residual=hs_norm(r))


def steady_state_gmres(sysm: System, tol=1e-10, m=20, restarts=50, eta=1.0, k_recycle=0):
    """Alg. 3: L~_eta rho = eta I by GMRES right-preconditioned with Precond(., 0, eta),
    warm start |0><0|, test ||L(rho_hat)||_max < tol on the hermitised state each cycle.
    k_recycle > 0 recycles that many harmonic Ritz vectors across restarts (App. A.2)."""
    n = sysm.n
    I = np.eye(n, dtype=np.complex128)
    x0 = np.zeros((n, n), dtype=np.complex128)
    x0[0, 0] = 1.0
    # L~_eta rho = eta I  <=>  (0 - L~_eta) rho = -eta I
    mv = lambda X: sysm.shifted_deflated(X, 0.0, eta)
    pc = lambda X: sysm.precond(X, 0.0, eta)
    state = {"cycles": 0}

    def hook(x):
        rh = hermitize_normalize(x)
        res = float(np.abs(sysm.L(rh)).max())
        state["rho"], state["res"] = rh, res
        state["cycles"] += 1
        return res < tol

    if k_recycle > 0:
        _, _, info = gcrodr(mv, pc, -eta * I, x0, m=m, k=k_recycle, atol=0.0, max_cycles=restarts, cycle_hook=hook)
        state["steps"] = info["steps"]
    else:
        gmres_right(mv, pc, -eta * I, x0, m=m, restarts=restarts, atol=0.0, cycle_hook=hook)
    return state["rho"], dict(residual=state["res"], cycles=state["cycles"], steps=state.get("steps"))


def resolvent_gmres(sysm: System, lam, B, tol=1e-10, m=32, k_recycle=8, recycle=None, x0=None, max_cycles=50):
    """(lam - L) X = B for lam > 0 by GMRES right-preconditioned with the no-jump resolvent R_lam^S
    (Sec. 3.1: (lam - L) R_lam^S = Id - K R_lam^S), recycled (App. A.2).  The test of Sec. 3.4 /
    App. B: for Hermitian B the iterate is hermitised and rescaled to its exact trace
    Tr X = Tr B / lam, and the solve stops when ||(lam - L)(X_hat) - B||_max < tol.
    Returns (X_hat, (U, C), info)."""
    herm = np.abs(B - dag(B)).max() == 0.0
    mv = lambda X: lam * X - sysm.L(X)
    pc = lambda X: sysm.resolvent_S(X, lam)
    target = np.trace(B) / lam
    state = {}

    def finish(x):
        xh = 0.5 * (x + dag(x)) if herm else x
        tr = np.trace(xh)
        if abs(tr) > 0:
            xh = xh * (target / tr)
        return xh

    def hook(x):
        xh = finish(x)
        res = float(np.abs(mv(xh) - B).max())
        state["x"], state["res"] = xh, res
        return res < tol

    x0 = np.zeros_like(B) if x0 is None else x0
    if hook(x0):
        return state["x"], recycle, dict(residual=state["res"], cycles=0, steps=0)
    x, rec, info = gcrodr(mv, pc, B, x0, m=m, k=k_recycle, recycle=recycle, atol=0.0, max_cycles=max_cycles,
                          cycle_hook=hook)
    return state["x"], rec, dict(residual=state["res"], cycles=info["cycles"], steps=info["steps"])


def implicit_euler_gmres(sysm: System, rho0, dt, steps, tol=1e-10, m=32, k_recycle=8):
    """Implicit Euler (Eq. resolvent, Sec. 4.3): each step solves (1/dt - L) rho_{t+dt} = rho_t / dt
    with the preconditioner R_{1/dt}^S, warm-started from rho_t, the recycled subspace carried from
    step to step (one operator for all steps).  Each solve stops when the max-norm residual is below
    tol * ||rho_t / dt||_max.  Returns the list of states."""
    lam = 1.0 / dt
    out, rho, rec = [], np.array(rho0, dtype=np.complex128), None
    for _ in range(steps):
        B = rho * lam
        rho, rec, _ = resolvent_gmres(sysm, lam, B, tol=tol * np.abs(B).max(), m=m, k_recycle=k_recycle,
                                      recycle=rec, x0=rho)
        out.append(rho.copy())
    return out


# ----------------------------------------------------------------------------- shift-invert
def low_spectrum_shift_invert(sysm: System, k=4, mu=0.0, eta=1.0, tol=1e-8, m=20, p=None,
                              restarts=30, inner_tol=1e-12, seed=0, k_recycle=0, inner_m=30):
    """Alg. 5: Krylov-Schur shift-invert Arnoldi on OP = (mu - L~_eta)^{-1}.

    OP(b) is a right-preconditioned GMRES solve (Precond(., mu, eta)); with k_recycle > 0 the
    recycled pair of GCRO-DR is threaded through every OP application (App. A.2).  Ritz
    values nu map back by lambda = mu - 1/nu; a thick restart keeps the p
    largest-|nu| Schur vectors.  Stops when max_k ||L v_k - lambda_k v_k||_max
    < tol on the raw (unnormalised, non-hermitised) Ritz vectors."""
    n = sysm.n
    p = p or max(k + 2, min(m - 2, 2 * k))
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    v0 -= np.trace(v0) / n * np.eye(n)           # nonzero eigenvectors are traceless
    mv = lambda X: sysm.shifted_deflated(X, mu, eta)
    pc = lambda X: sysm.precond(X, mu, eta)

    rec = [None]

    def OP(b):
        if k_recycle > 0:
            x, rec[0], _ = gcrodr(mv, pc, b, np.zeros_like(b), m=inner_m, k=k_recycle, recycle=rec[0],
                                  atol=inner_tol * max(hs_norm(b), 1e-300), max_cycles=20)
            return x
        return gmres_right(mv, pc, b, np.zeros_like(b), m=inner_m, restarts=20,
                           atol=inner_tol * max(hs_norm(b), 1e-300))

    V = [v0 / hs_norm(v0)]
    Hk = np.zeros((1, 0), dtype=np.complex128)   # (j+1) x j Arnoldi / Krylov-Schur relation
    lam = vecs = None
    res = np.inf
    for _ in range(restarts):
        j0 = len(V) - 1
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        Hm[: j0 + 1, :j0] = Hk
        for j in range(j0, m):
            w = OP(V[j])
            for _ in range(2):
                for i in range(j + 1):
                    h = hs_inner(V[i], w)
                    Hm[i, j] += h
                    w = w - h * V[i]
            hn = hs_norm(w)
            Hm[j + 1, j] = hn
            V.append(w / hn)
        # Ritz pairs of OP; the k of largest |nu| give lambda = mu - 1/nu
        nu, Y = np.linalg.eig(Hm[:m, :m])
        idx = np.argsort(-np.abs(nu))[:k]
        lam = mu - 1.0 / nu[idx]
        vecs = [sum(Y[s, t] * V[s] for s in range(m)) for t in idx]
        res = max(float(np.abs(sysm.L(v) - l * v).max() / np.abs(v).max())
                  for l, v in zip(lam, vecs))
        if res < tol:
            break
        # thick restart: sorted Schur form puts the p largest-|nu| values first
        thr = np.sort(np.abs(nu))[-p] * (1.0 - 1e-12)
        Tm, Z, sdim = sla.schur(Hm[:m, :m], output="complex", sort=lambda x: abs(x) >= thr)
        Vn = [sum(Z[s, t] * V[s] for s in range(m)) for t in range(sdim)]
        Hk = np.zeros((sdim + 1, sdim), dtype=np.complex128)
        Hk[:sdim, :sdim] = Tm[:sdim, :sdim]
        Hk[sdim, :] = Hm[m, :m] @ Z[:, :sdim]
        V = Vn + [V[m]]
    order = np.lexsort((lam.imag, -lam.real, np.round(np.abs(lam), 12)))
    return lam[order], [vecs[i] for i in order], dict(residual=res)
