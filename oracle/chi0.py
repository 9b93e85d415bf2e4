"""Static RPA polarizability chi0(r, r') on a site grid, two independent routes.

Definitions (Sec. II.A and VI.A, VI.D):
  Eq. (eq-rpa)   chi0(1,2) = -i g0(1,2) g0(2,1+)
  Eq. (eq-green) g(r,r',E) = sum_kb w_k psi*_kb(r) psi_kb(r') / (E - eps_kb)
  Eq. (chi1)     chi0(r,r',0) = sum_spin int dt/2pi g(r,r',mu+it) g(r',r,mu+it)

chi0_pairs (the sum-over-states form): the t-integral of
1/((alpha+it)(beta+it)), alpha = mu-eps_b, beta = mu-eps_b', is
(sign alpha - sign beta)/(2(beta-alpha)): it vanishes unless one band is
occupied and the other is not, and for occupied v, unoccupied c it is
kappa = 1/(eps_v - eps_c).  Summing both orders of each pair and both spins,
  chi0(p,p') = 4 sum_{v,c} w_v w_c kappa(v,c) Re[A_vc(p) conj A_vc(p')],
  A_vc(p) = conj psi_v(p) psi_c(p).
With kappa = kappa_quadrature it equals the quadrature of Eq. (chi1) exactly
(up to rounding); with kappa_exact it is the brute-force physical value.

chi0_green (the paper's route, Sec. VI.D with App. D.1): for each frequency
build the Green's functions restricted to the site from Eq. (eq-green) and
accumulate (2/pi) sum_i W_i Re[g(r,r') g(r',r)].  By default only the
occupied x unoccupied cross terms of the product are kept (their exact
integrals are the only non-zero ones); full_g=True squares the whole g as
printed in App. D.1.
"""
import numpy as np

from .quadrature import kappa_exact, kappa_quadrature


def chi0_pairs(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, t=None, W=None,
               exact=False, rows=None, block=16):
    """chi0[rows, :] by the pair sum.  psi_o [npts,Ko], psi_u [npts,Ku] complex."""
    npts = psi_o.shape[0]
    rows = np.arange(npts) if rows is None else np.asarray(rows)
    alpha = mu - np.asarray(e_o, float)
    beta = mu - np.asarray(e_u, float)
    out = np.zeros((len(rows), npts))
    for v0 in range(0, psi_o.shape[1], block):
        v1 = min(v0 + block, psi_o.shape[1])
        if exact:
            kap = kappa_exact(alpha[v0:v1, None], beta[None, :])
        else:
            kap = kappa_quadrature(alpha[v0:v1, None], beta[None, :], t, W)
        c = (w_o[v0:v1, None] * w_u[None, :] * kap).reshape(-1)      # [nv*Ku]
        a = (np.conj(psi_o[:, v0:v1])[:, :, None] * psi_u[:, None, :]).reshape(npts, -1)
        ar, ai = a.real, a.imag
        out += 4.0 * ((ar[rows] * c) @ ar.T + (ai[rows] * c) @ ai.T)
    return out


def green_pair(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, t):
    """g_o(p,p') and g_u(p',p) at energy mu + i t (Eq. (eq-green) split by occupation)."""
    d_o = w_o / (mu + 1j * t - e_o)
    d_u = w_u / (mu + 1j * t - e_u)
    g_o = (np.conj(psi_o) * d_o) @ psi_o.T            # sum_v conj psi_v(p) d_v psi_v(p')
    g_u_t = (psi_u * d_u) @ np.conj(psi_u).T          # sum_c conj psi_c(p') d_c psi_c(p)
    return g_o, g_u_t


def chi0_green(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, t, W, full_g=False, rows=None):
    """chi0 [npts, npts], or only its rows `rows` (cross terms only): the same sum with the
    Green's functions evaluated where those rows need them, g(rows, :) and g(:, rows)."""
    if rows is not None:
        return _chi0_green_rows(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, t, W, np.asarray(rows))
    npts = psi_o.shape[0]
    acc = np.zeros((npts, npts))
    for ti, wi in zip(t, W):
        g_o, g_u_t = green_pair(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, ti)
        if full_g:
            # g(p,p') g(p',p) with g = g_o + g_u; g_u(p,p') is g_u_t transposed.
            g = g_o + g_u_t.T
            acc += wi * (g * g.T).real
        else:
            y = g_o * g_u_t                           # g_o(p,p') g_u(p',p)
            acc += wi * (y + y.T).real
    return (2.0 / np.pi) * acc


def _chi0_green_rows(psi_o, psi_u, e_o, e_u, w_o, w_u, mu, t, W, rows):
    """Rows p in `rows` of (2/pi) sum_i W_i Re[y(p,p') + y(p',p)], y = g_o(p,p') g_u(p',p)."""
    acc = np.zeros((len(rows), psi_o.shape[0]))
    for ti, wi in zip(t, W):
        d_o = w_o / (mu + 1j * ti - e_o)
        d_u = w_u / (mu + 1j * ti - e_u)
        g_o_r = (np.conj(psi_o[rows]) * d_o) @ psi_o.T       # g_o(p, p'),  p in rows
        g_o_c = (np.conj(psi_o) * d_o) @ psi_o[rows].T       # g_o(p', p)
        g_u_r = (psi_u[rows] * d_u) @ np.conj(psi_u).T       # g_u(p', p)
        g_u_c = (psi_u * d_u) @ np.conj(psi_u[rows]).T       # g_u(p, p')
        acc += wi * (g_o_r * g_u_r + (g_o_c * g_u_c).T).real
    return (2.0 / np.pi) * acc
