"""Coulomb operator on a site grid in multipole form (Sec. VI.E).

v(r, r') = sum_lm 4pi/(2l+1) r_<^l / r_>^(l+1) Y_lm(r^) Y*_lm(r'^); by the
addition theorem of spherical harmonics this is
  v(r, r') = sum_{l=0}^{L} r_<^l / r_>^(l+1) P_l(r^ . r'^),
truncated at the multipole order L that the angular grid resolves.  It is
finite on the diagonal and positive semidefinite (each term is a positive
radial kernel times a positive-definite zonal kernel).
"""
import numpy as np
from scipy.special import eval_legendre


def coulomb_multipole(pts, lmax):
    pts = np.asarray(pts, float)
    r = np.linalg.norm(pts, axis=1)
    if np.any(r <= 0.0):
        raise ValueError("site grid point at the origin has no direction")
    u = pts / r[:, None]
    cosg = np.clip(u @ u.T, -1.0, 1.0)
    rl = np.minimum.outer(r, r)
    rg = np.maximum.outer(r, r)
    v = np.zeros_like(cosg)
    for l in range(int(lmax) + 1):
        v += (rl ** l / rg ** (l + 1)) * eval_legendre(l, cosg)
    return v
