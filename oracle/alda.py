"""ALDA vertex correction of the polarizability (Sec. VII "Beyond RPA
screening", Eq. (chi-alda) and (kxc_alda)).

TEST INFRASTRUCTURE ONLY (see the package header).

  chi~ = (1 - chi0 (v + f_xc))^-1 chi0,   f_xc(r, r') = delta(r - r') dv_xc/dn |_{n(r)}
  W~ = v + v chi~ v                        (the screened interaction of chi~)

On the grid every integral carries its weight (Q = diag(w)); the contact
kernel becomes D = diag(f_xc(r_p) w_p) in the products:
  chi~ = (I - chi0 Q v Q - chi0 D)^-1 chi0.
The density n(r) = 2 sum_k w_k sum_occ |psi_kv(r)|^2 (spin-unpolarised), and
the exchange-only ALDA kernel of the uniform electron gas (Dirac exchange,
e_x(n) = -(3/4) (3/pi)^(1/3) n^(4/3) per volume) is
  f_x(n) = d^2 e_x / dn^2 = -(1/3) (3/pi)^(1/3) n^(-2/3).
"""
import numpy as np


def density(psi_o, w_o):
    """n(r_p) = 2 sum_c w_c |psi_o[p, c]|^2 over occupied columns (k-weight w_c)."""
    return 2.0 * (np.abs(psi_o) ** 2 @ np.asarray(w_o, float))


def exchange_energy_density(n):
    return -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * np.asarray(n, float) ** (4.0 / 3.0)


def fx_exchange(n):
    return -(1.0 / 3.0) * (3.0 / np.pi) ** (1.0 / 3.0) * np.asarray(n, float) ** (-2.0 / 3.0)


def chi_alda(chi0, v, fxc, wts):
    """chi~ of Eq. (chi-alda) by a dense solve on the grid."""
    q = np.asarray(wts, float)
    n = chi0.shape[0]
    k = (v * q[None, :]) * q[:, None] + np.diag(np.asarray(fxc, float) * q)   # Q v Q + D
    return np.linalg.solve(np.eye(n) - chi0 @ k, chi0)


def screened_interaction_alda(chi0, v, fxc, wts):
    """W~ = v + v Q chi~ Q v."""
    q = np.asarray(wts, float)
    chi = chi_alda(chi0, v, fxc, wts)
    return v + (v * q[None, :]) @ chi @ (v * q[:, None])
