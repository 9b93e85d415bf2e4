"""Analytic gradients of a scalar loss of W in pair form (no counterpart in the paper).

With A = I - v Q chi0 Q and W = A^-1 v, dW = W Q dchi0 Q W, so a loss with
gradient Gamma_W = dL/dW has dL/dchi0 = Q W^T Gamma_W W^T Q.  chi0 is
symmetric, so only the symmetric part Gsym of that matrix matters; writing
Gsym = sum_k lam_k u_k u_k^T, each term contributes
  lam_k u^T chi0 u = 4 lam_k sum_{v,c} w_v w_c kappa_vc |B_vc|^2,
  B_vc = sum_p u_p conj psi_v(p) psi_c(p).
Differentiating at fixed mu and quadrature (t_i, W_i):
  dL/deps_v = -sum_c 4 lam w w' |B|^2 dkappa/dalpha, alpha = mu - eps_v
  dL/deps_c = -sum_v 4 lam w w' |B|^2 dkappa/dbeta,  beta  = mu - eps_c
  dL/dpsi_c(p) = 8 lam u_p sum_v w w' kappa B_vc psi_v(p)
  dL/dpsi_v(p) = 8 lam u_p sum_c w w' kappa conj(B_vc) psi_c(p)
(complex gradients in the dL/dRe + i dL/dIm convention).
"""
import numpy as np

from .quadrature import dkappa_exact, dkappa_quadrature, kappa_exact, kappa_quadrature


def gamma_chi0(W, wts, gamma_w):
    q = np.asarray(wts, float)
    return (q[:, None] * W.T) @ gamma_w @ (W.T * q[None, :])


def grad_pairs(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, t, Wq, gamma, exact=False):
    """Gradients of L with dL/dchi0 = gamma (any [npts,npts] matrix)."""
    alpha = mu - np.asarray(e_o, float)
    beta = mu - np.asarray(e_u, float)
    if exact:
        kap = kappa_exact(alpha[:, None], beta[None, :])
        dka, dkb = dkappa_exact(alpha[:, None], beta[None, :])
    else:
        kap = kappa_quadrature(alpha[:, None], beta[None, :], t, Wq)
        dka, dkb = dkappa_quadrature(alpha[:, None], beta[None, :], t, Wq)
    ww = w_o[:, None] * w_u[None, :]
    gs = 0.5 * (gamma + gamma.T)
    lam, vecs = np.linalg.eigh(gs)
    ge_o = np.zeros(len(e_o)); ge_u = np.zeros(len(e_u))
    gp_o = np.zeros(psi_o.shape, np.complex128); gp_u = np.zeros(psi_u.shape, np.complex128)
    for k in range(len(lam)):
        if lam[k] == 0.0:
            continue
        u = vecs[:, k]
        b = (np.conj(psi_o) * u[:, None]).T @ psi_u            # B_vc [Ko, Ku]
        b2 = np.abs(b) ** 2
        ge_o += -4.0 * lam[k] * (ww * b2 * dka).sum(1)
        ge_u += -4.0 * lam[k] * (ww * b2 * dkb).sum(0)
        m = ww * kap * b
        gp_u += 8.0 * lam[k] * u[:, None] * (psi_o @ m)
        gp_o += 8.0 * lam[k] * u[:, None] * (psi_u @ np.conj(m).T)
    return ge_o, ge_u, gp_o, gp_u
