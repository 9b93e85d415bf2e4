"""Imaginary-frequency quadrature of Eq. (chi1), App. D.1 "Energy integration".

Eq. (chi1) integrates g(r,r',mu+it) g(r',r,mu+it) over t on the whole real
line with measure dt/2pi.  Because the integrand at -t is the complex
conjugate of the one at +t, the line integral equals (1/pi) int_0^inf Re[...] dt.
The single-grid map of App. D.1 takes Gauss-Legendre points x_i, w_i on
[-1, 1], shifts and halves them to a_i = (x_i+1)/2, w_i/2 on [0, 1], and uses
t_i = zeta a_i / (1 - a_i) with weight W_i = zeta (w_i/2) / (1 - a_i)^2, so that
int_0^inf f(t) dt ~ sum_i W_i f(t_i).

mu sits mid-gap (Sec. VI.D).  zeta is the geometric mean of the smallest and
largest |mu - eps|, with 0.5 eV added in quadrature to the smallest (App. D.1).
"""
import numpy as np

HARTREE_EV = 27.211386245988
ZETA_FLOOR_EV = 0.5


def chemical_potential_midgap(energies, nocc):
    """mu halfway between the highest occupied and lowest unoccupied level over all k."""
    top = max(np.max(energies[k, :int(nocc[k])]) for k in range(len(nocc)))
    bottom = min(np.min(energies[k, int(nocc[k]):]) for k in range(len(nocc)))
    return 0.5 * (top + bottom)


def zeta_rule(energies, mu):
    d = np.abs(mu - np.asarray(energies, float).ravel())
    dmin = np.sqrt(np.min(d) ** 2 + (ZETA_FLOOR_EV / HARTREE_EV) ** 2)
    return float(np.sqrt(dmin * np.max(d)))


def frequency_grid(nf, zeta):
    """Nodes t_i and weights W_i of int_0^inf dt (single-grid map)."""
    x, w = np.polynomial.legendre.leggauss(nf)
    a = 0.5 * (x + 1.0)
    wa = 0.5 * w
    return zeta * a / (1.0 - a), zeta * wa / (1.0 - a) ** 2


def kappa_quadrature(alpha, beta, t, W):
    """(1/pi) sum_i W_i Re[1/((alpha+it)(beta+it))] for alpha = mu-eps_v, beta = mu-eps_c.

    Re[1/((alpha+it)(beta+it))] = (alpha beta - t^2)/((alpha^2+t^2)(beta^2+t^2)).
    Broadcasts over alpha and beta.
    """
    alpha = np.asarray(alpha, float)[..., None]
    beta = np.asarray(beta, float)[..., None]
    t2 = np.asarray(t, float) ** 2
    f = (alpha * beta - t2) / ((alpha ** 2 + t2) * (beta ** 2 + t2))
    return (f * np.asarray(W, float)).sum(-1) / np.pi


def kappa_exact(alpha, beta):
    """(1/2pi) int_R dt 1/((alpha+it)(beta+it)) = 1/(beta - alpha) when alpha > 0 > beta."""
    return 1.0 / (np.asarray(beta, float) - np.asarray(alpha, float))


def dkappa_quadrature(alpha, beta, t, W):
    """Partial derivatives of kappa_quadrature with respect to alpha and beta."""
    alpha = np.asarray(alpha, float)[..., None]
    beta = np.asarray(beta, float)[..., None]
    t2 = np.asarray(t, float) ** 2
    a2, b2 = alpha ** 2 + t2, beta ** 2 + t2
    da = (-alpha ** 2 * beta + beta * t2 + 2.0 * alpha * t2) / (a2 ** 2 * b2)
    db = (-beta ** 2 * alpha + alpha * t2 + 2.0 * beta * t2) / (a2 * b2 ** 2)
    W = np.asarray(W, float)
    return (da * W).sum(-1) / np.pi, (db * W).sum(-1) / np.pi


def dkappa_exact(alpha, beta):
    d = np.asarray(beta, float) - np.asarray(alpha, float)
    return 1.0 / d ** 2, -1.0 / d ** 2
