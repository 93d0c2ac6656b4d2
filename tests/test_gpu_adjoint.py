"""Implicit differentiation of the steady state (Remark "Differentiating the steady state"):
the adjoint solve and the sensitivity matrices, through the C ABI, against the dense oracle's
adjoint gradient, central finite differences and the Euler scaling identity
(L(s theta) = s L(theta) for theta = (J, h, gamma, gamma_phi), so sum_i theta_i dJ/dtheta_i = 0)."""
import numpy as np
import pytest
import torch

import lindblad_inputs as gi
from oracle import dense as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2608_30860_b300 as B
    B.load_library()
    return B


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _tfim_pieces(N):
    HJ, Hh, decay, dephase, Sz = gi.tfim_terms(N)
    return HJ, Hh, decay, dephase, Sz


def _theta_grad(B, N, theta, tol=1e-13):
    """dJ/dtheta from the library's sensitivities, J = <mean sz>."""
    J, h, gam, gph = theta
    HJ, Hh, decay, dephase, Sz = _tfim_pieces(N)
    H = J * HJ + h * Hh
    Ls = [np.sqrt(gam) * L for L in decay] + [np.sqrt(gph) * L for L in dephase]
    opts = B.default_opts(tol=tol, max_restarts=100)
    hd = B.lindblad_setup(_cuda(H), _cuda(np.stack(Ls)), opts)
    rho, info, st = B.steady_state(hd, opts)
    assert st == 0, info
    w, gH, gL, ainfo, ast = B.steady_state_adjoint(hd, rho, _cuda(Sz), opts)
    B.lindblad_destroy(hd)
    gH, gL = gH.cpu().numpy(), gL.cpu().numpy()
    ip = lambda G, dX: np.real(np.vdot(G.reshape(-1), dX.reshape(-1)))
    d = len(decay)
    dJ = [ip(gH, HJ), ip(gH, Hh),
          sum(ip(gL[j], decay[j] / (2 * np.sqrt(gam))) for j in range(d)),
          sum(ip(gL[d + j], dephase[j] / (2 * np.sqrt(gph))) for j in range(d))]
    return np.array(dJ), ainfo, ast, rho.cpu().numpy()


def test_adjoint_gradient_matches_dense_oracle(B):
    N = 4
    theta = np.array([1.0, 0.7, 0.5, 0.1])
    g, ainfo, ast, rho = _theta_grad(B, N, theta)
    assert ast == 0 and ainfo["residual_max"] < 1e-10, ainfo
    HJ, Hh, decay, dephase, Sz = _tfim_pieces(N)
    Hf = lambda t: t[0] * HJ + t[1] * Hh
    Lf = lambda t: [np.sqrt(t[2]) * L for L in decay] + [np.sqrt(t[3]) * L for L in dephase]
    Z = np.zeros_like(HJ)
    dL = lambda t: [D.liouvillian(HJ, []), D.liouvillian(Hh, []), D.liouvillian(Z, decay),
                    D.liouvillian(Z, dephase)]
    ref, _ = D.steady_state_gradient(Hf, Lf, dL, theta, Sz)
    assert np.abs(g - ref).max() < 1e-8 * np.abs(ref).max(), (g, ref)


def test_euler_identity_ten_site_chain(B):
    """The 1024-dimensional, 20-jump chain: the scaling identity holds to solver accuracy."""
    theta = np.array([1.0, 0.7, 0.5, 0.1])
    g, ainfo, ast, rho = _theta_grad(B, 10, theta, tol=1e-11)
    assert ast == 0, ainfo
    assert abs(np.dot(theta, g)) < 1e-7 * np.abs(g).max(), (g, np.dot(theta, g))


def test_autograd_function_matches_finite_differences(B):
    from paper_2608_30860_b300.autograd import steady_state_expectation
    N = 3
    HJ, Hh, decay, dephase, Sz = _tfim_pieces(N)
    tHJ, tHh, tSz = _cuda(HJ), _cuda(Hh), _cuda(Sz)
    tdec, tdep = _cuda(np.stack(decay)), _cuda(np.stack(dephase))

    def J_of(t):
        H = t[0] * tHJ + t[1] * tHh
        L = torch.cat([torch.sqrt(t[2]) * tdec, torch.sqrt(t[3]) * tdep])
        return steady_state_expectation(H.to(torch.complex128), L.to(torch.complex128), tSz)

    theta = torch.tensor([1.0, 0.7, 0.5, 0.1], dtype=torch.float64, device="cuda", requires_grad=True)
    val = J_of(theta)
    (g,) = torch.autograd.grad(val, theta)
    g = g.cpu().numpy()
    for i in range(4):
        hstep = 1e-5 * max(1.0, float(theta[i]))
        tp = theta.detach().clone()
        tm = theta.detach().clone()
        tp[i] += hstep
        tm[i] -= hstep
        fd = (float(J_of(tp)) - float(J_of(tm))) / (2 * hstep)
        assert abs(g[i] - fd) < 1e-6 * max(1.0, abs(g[i])), (i, g[i], fd)
