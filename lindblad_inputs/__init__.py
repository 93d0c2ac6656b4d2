"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This module builds problem data only -- Hamiltonians, jump operators and random
operands -- and holds none of the method's arithmetic (no Lindbladian, no
Lyapunov solve, no Krylov step).  Every array is complex128, C-contiguous,
row-major, shape (n, n).

Systems (paper section / Eq. in brackets):
  * Kerr-cat oscillator  H = -K a^dag2 a^2 + eps2 (a^dag2 + a^2),
    L1 = sqrt(kappa2) a^2, L2 = sqrt(kappa1) a.  The truncated ladder operator is
    the superdiagonal sqrt(1..n-1) matrix of App. B ("Cat qubit").
  * Random Lindbladian with 1/sqrt(n) scaling: H = (A + A^dag)/(2 sqrt(n)), A with
    circular complex Gaussian entries of unit variance; L_j entries circular
    complex Gaussian of variance 1/n.
  * The paper's own dense random family (App. B "Random (dense)"):
    H = (A0 + A0^dag)/2, L_j = sqrt(gamma) A_j, Re and Im i.i.d. N(0, 1).
  * Open transverse-field Ising chain, Pauli matrices with eigenvalues +-1,
    |0> = up (sigma_z = +1), sigma_minus = |1><0|, site 1 the most significant
    Kronecker factor, open boundary (N-1 bonds).
  * Thermally damped oscillator H = omega a^dag a, L1 = sqrt(kappa (1+nth)) a,
    L2 = sqrt(kappa nth) a^dag.
  * The qubit-decay example (footnote of Sec. 3.1) and the three-level cyclic
    example (Remark "Peripheral spectra of Phi").
  * The memory-buffer cat qubit (App. B "Cat qubit", Table of its parameters):
    H = g2 (a^2 b^dag + a^dag2 b) - eps_d (b + b^dag), four thermal jumps on the
    memory a = a~ (x) I and the buffer b = I (x) b~, eps_d = g2 n_a / 5,
    n_a = round(sqrt(3 n)), n_b = floor(n_a / 3).  Rates in units of 2 pi MHz.
  * The stiff implicit-Euler family (Sec. 4.3 and App. B "Time evolution"): the
    paper's dense random system plus K N^2 on H, N = diag(0, ..., n-1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "ladder", "kerr_cat", "random_lindbladian", "paper_random_lindbladian",
    "tfim", "tfim_terms", "thermal_oscillator", "qubit_decay", "three_level_cycle",
    "haar_unitary", "conjugate_system", "random_operator", "random_hermitian",
    "random_density", "kerr_cat_sweep", "memory_buffer_cat", "memory_buffer_dims",
    "stiff_random_lindbladian", "CONFIGS",
]


def ladder(n: int) -> np.ndarray:
    """Truncated annihilation operator: superdiagonal sqrt(1), ..., sqrt(n-1)."""
    a = np.zeros((n, n), dtype=np.complex128)
    idx = np.arange(1, n)
    a[idx - 1, idx] = np.sqrt(idx)
    return a


def kerr_cat(n: int, K: float = 1.0, eps2: float = 4.0, kappa2: float = 1.0,
             kappa1: float = 0.01):
    """Kerr-cat oscillator truncated at n Fock levels; returns (H, [L1, L2])."""
    a = ladder(n)
    ad = a.conj().T
    a2 = a @ a
    ad2 = ad @ ad
    H = -K * (ad2 @ a2) + eps2 * (ad2 + a2)
    H = 0.5 * (H + H.conj().T)
    Ls = [np.sqrt(kappa2) * a2, np.sqrt(kappa1) * a]
    return np.ascontiguousarray(H), [np.ascontiguousarray(L) for L in Ls]


def _circular_gaussian(rng: np.random.Generator, n: int, var: float) -> np.ndarray:
    # Re and Im ~ N(0, var/2) so that E|z|^2 = var; real block drawn first.
    s = np.sqrt(var / 2.0)
    re = rng.standard_normal((n, n)) * s
    im = rng.standard_normal((n, n)) * s
    return re + 1j * im


def random_lindbladian(n: int, d: int = 4, seed: int = 0):
    """Random dense Lindbladian, H = (A + A^dag)/(2 sqrt n), Var(L_ij) = 1/n."""
    rng = np.random.default_rng(seed)
    A = _circular_gaussian(rng, n, 1.0)
    H = (A + A.conj().T) / (2.0 * np.sqrt(n))
    Ls = [_circular_gaussian(rng, n, 1.0 / n) for _ in range(d)]
    return np.ascontiguousarray(H), Ls


def paper_random_lindbladian(n: int, seed: int = 0, gamma: float = 0.1, d: int = 3):
    """App. B dense family: Re, Im i.i.d. standard normal; H=(A0+A0^dag)/2, L_j=sqrt(gamma) A_j."""
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(d + 1):
        re = rng.standard_normal((n, n))
        im = rng.standard_normal((n, n))
        mats.append(re + 1j * im)
    H = (mats[0] + mats[0].conj().T) / 2.0
    Ls = [np.sqrt(gamma) * A for A in mats[1:]]
    return np.ascontiguousarray(H), Ls


_SZ = np.array([[1.0, 0.0], [0.0, -1.0]], dtype=np.complex128)
_SX = np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)
_SM = np.array([[0.0, 0.0], [1.0, 0.0]], dtype=np.complex128)  # |1><0|, up -> down


def _site_op(op: np.ndarray, i: int, N: int) -> np.ndarray:
    out = np.ones((1, 1), dtype=np.complex128)
    for k in range(N):
        out = np.kron(out, op if k == i else np.eye(2, dtype=np.complex128))
    return out


def _site_pair(op1, i, op2, j, N):
    out = np.ones((1, 1), dtype=np.complex128)
    for k in range(N):
        if k == i:
            f = op1
        elif k == j:
            f = op2
        else:
            f = np.eye(2, dtype=np.complex128)
        out = np.kron(out, f)
    return out


def tfim_terms(N: int):
    """Structural pieces of the open TFIM chain.

    Returns (H_J, H_h, decay_ops, dephase_ops, Sz_mean) with
    H = J H_J + h H_h, jumps sqrt(gamma) decay_ops[i] and sqrt(gamma_phi) dephase_ops[i],
    and Sz_mean = (1/N) sum_i sigma_z^i (the observable 'mean sz').
    """
    n = 2 ** N
    HJ = np.zeros((n, n), dtype=np.complex128)
    Hh = np.zeros((n, n), dtype=np.complex128)
    for i in range(N - 1):
        HJ += _site_pair(_SZ, i, _SZ, i + 1, N)
    for i in range(N):
        Hh += _site_op(_SX, i, N)
    decay = [_site_op(_SM, i, N) for i in range(N)]
    dephase = [_site_op(_SZ, i, N) for i in range(N)]
    Sz = sum(dephase) / N
    return HJ, Hh, decay, dephase, Sz


def tfim(N: int, J: float = 1.0, h: float = 0.7, gamma: float = 0.5,
         gamma_phi: float = 0.0):
    """Open TFIM chain with dense jumps sqrt(gamma) s-_i (and sqrt(gamma_phi) sz_i if > 0)."""
    HJ, Hh, decay, dephase, _ = tfim_terms(N)
    H = J * HJ + h * Hh
    Ls = [np.sqrt(gamma) * L for L in decay]
    if gamma_phi > 0.0:
        Ls += [np.sqrt(gamma_phi) * L for L in dephase]
    return np.ascontiguousarray(H), [np.ascontiguousarray(L) for L in Ls]


def thermal_oscillator(n: int, omega: float = 1.0, kappa: float = 0.5, nth: float = 0.3):
    """Damped oscillator H = omega a^dag a, L1 = sqrt(kappa(1+nth)) a, L2 = sqrt(kappa nth) a^dag."""
    a = ladder(n)
    ad = a.conj().T
    H = omega * (ad @ a)
    Ls = [np.sqrt(kappa * (1.0 + nth)) * a]
    if nth > 0.0:
        Ls.append(np.sqrt(kappa * nth) * ad)
    return np.ascontiguousarray(H), [np.ascontiguousarray(L) for L in Ls]


def qubit_decay(gamma: float = 1.0):
    """n=2, H=0, L = sqrt(gamma)|0><1| (footnote of Sec. 3.1)."""
    H = np.zeros((2, 2), dtype=np.complex128)
    L = np.zeros((2, 2), dtype=np.complex128)
    L[0, 1] = np.sqrt(gamma)
    return H, [L]


def three_level_cycle():
    """n=3, H=0, L1=|0><1|, L2=|1><2|, L3=|2><0| (Remark 'Peripheral spectra of Phi')."""
    H = np.zeros((3, 3), dtype=np.complex128)
    Ls = []
    for (i, j) in ((0, 1), (1, 2), (2, 0)):
        L = np.zeros((3, 3), dtype=np.complex128)
        L[i, j] = 1.0
        Ls.append(L)
    return H, Ls


def haar_unitary(n: int, seed: int = 0) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix with the R-diagonal phases removed."""
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return np.ascontiguousarray(Q * ph[None, :])


def conjugate_system(H, Ls, W):
    """Rotate the problem data by a unitary W: H -> W H W^dag, L_j -> W L_j W^dag."""
    Wd = W.conj().T
    return (np.ascontiguousarray(W @ H @ Wd),
            [np.ascontiguousarray(W @ L @ Wd) for L in Ls])


def random_operator(n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(_circular_gaussian(rng, n, 1.0))


def random_hermitian(n: int, seed: int = 0) -> np.ndarray:
    X = random_operator(n, seed)
    return np.ascontiguousarray(0.5 * (X + X.conj().T))


def random_density(n: int, seed: int = 0) -> np.ndarray:
    X = random_operator(n, seed)
    rho = X @ X.conj().T
    return np.ascontiguousarray(rho / np.trace(rho).real)


def kerr_cat_sweep(count: int = 1024, seed: int = 0, nmin: int = 16, nmax: int = 160):
    """Parameter list for a sweep of Kerr-cat instances of uneven size.

    One seeded stream, drawn in instance order: n ~ U{nmin..nmax} (inclusive),
    eps2 ~ U[1, 8], K ~ U[0.5, 2], kappa1 ~ U[1e-3, 1e-1]; kappa2 = 1.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        eps2 = float(rng.uniform(1.0, 8.0))
        K = float(rng.uniform(0.5, 2.0))
        kappa1 = float(rng.uniform(1e-3, 1e-1))
        out.append(dict(n=n, eps2=eps2, K=K, kappa1=kappa1, kappa2=1.0))
    return out


# App. B table (memory-buffer cat), in units of 2 pi MHz: g2/2pi = 0.763 MHz, kappa_b/2pi = 2.6 MHz,
# kappa_a/2pi = 9.3 kHz, thermal occupations 10 % (memory) and 1.1 % (buffer).
MEMORY_BUFFER = dict(g2=0.763, kappa_b=2.6, kappa_a=0.0093, nth_a=0.10, nth_b=0.011)


def memory_buffer_dims(n: int):
    """Truncations for a target dimension n (App. B): n_a = round(sqrt(3 n)), n_b = floor(n_a / 3)."""
    na = int(round(np.sqrt(3.0 * n)))
    nb = max(1, na // 3)
    return na, nb


def memory_buffer_cat(na: int, nb: int, g2: float = MEMORY_BUFFER["g2"], kappa_b: float = MEMORY_BUFFER["kappa_b"],
                      kappa_a: float = MEMORY_BUFFER["kappa_a"], nth_a: float = MEMORY_BUFFER["nth_a"],
                      nth_b: float = MEMORY_BUFFER["nth_b"], eps_d: float | None = None):
    """Memory-buffer cat qubit of dimension n = na * nb; returns (H, [L1, L2, L3, L4]) with
    L1 = sqrt(kb (1 + nb_th)) b, L2 = sqrt(kb nb_th) b^dag, L3 = sqrt(ka (1 + na_th)) a,
    L4 = sqrt(ka na_th) a^dag; eps_d defaults to g2 na / 5 (cat size |alpha|^2 = na / 5)."""
    if eps_d is None:
        eps_d = g2 * na / 5.0
    a = np.kron(ladder(na), np.eye(nb, dtype=np.complex128))
    b = np.kron(np.eye(na, dtype=np.complex128), ladder(nb))
    ad, bd = a.conj().T, b.conj().T
    H = g2 * (a @ a @ bd + ad @ ad @ b) - eps_d * (b + bd)
    H = 0.5 * (H + H.conj().T)
    Ls = [np.sqrt(kappa_b * (1.0 + nth_b)) * b, np.sqrt(kappa_b * nth_b) * bd,
          np.sqrt(kappa_a * (1.0 + nth_a)) * a, np.sqrt(kappa_a * nth_a) * ad]
    return np.ascontiguousarray(H), [np.ascontiguousarray(L) for L in Ls]


def stiff_random_lindbladian(n: int = 32, K: float = 0.0, seed: int = 0, gamma: float = 0.1):
    """The implicit-Euler benchmark system: App. B's dense random family with K N^2 added to H."""
    H, Ls = paper_random_lindbladian(n, seed=seed, gamma=gamma)
    N = np.arange(n, dtype=np.float64)
    H = H + np.diag(K * N ** 2).astype(np.complex128)
    return np.ascontiguousarray(H), Ls


# The five synthetic workloads: name -> (builder, kwargs, description).
CONFIGS = {
    "kerr_cat_n32": (kerr_cat, dict(n=32, K=1.0, eps2=4.0, kappa2=1.0, kappa1=0.01),
                     "Kerr-cat oscillator, n=32, d=2"),
    "random_n512_d4": (random_lindbladian, dict(n=512, d=4, seed=0),
                       "random Lindbladian, n=512, d=4, seed 0"),
    "tfim10_n1024_d20": (tfim, dict(N=10, J=1.0, h=0.7, gamma=0.5, gamma_phi=0.1),
                         "10-site open TFIM, n=1024, d=20"),
    "tfim12_n4096_d12": (tfim, dict(N=12, J=1.0, h=1.0, gamma=0.3, gamma_phi=0.0),
                         "12-site open TFIM, n=4096, d=12 decay jumps"),
}
