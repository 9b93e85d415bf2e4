"""Screened interaction from the Dyson equation (Sec. II.A, VI.E).

Eq. (eq-reducible) chi = chi0 + chi0 v chi and Eq. (eq-W) W = v + v chi v
combine into W = v + v chi0 W.  On the grid every integral over a point
carries its weight, Q = diag(weights), so
  (I - v Q chi0 Q) W = v,
solved by LU with partial pivoting (LAPACK dgesv through numpy.linalg.solve).
"""
import numpy as np


def dyson_matrix(v, chi0, wts):
    q = np.asarray(wts, float)
    return np.eye(v.shape[0]) - (v * q[None, :]) @ (chi0 * q[None, :])


def screened_interaction(v, chi0, wts):
    return np.linalg.solve(dyson_matrix(v, chi0, wts), v)
