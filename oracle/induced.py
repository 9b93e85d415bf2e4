"""Screening of a spherical short-range potential in the (radial, l, m) basis:
the induced density and potential of Sec. VI.E (the core-hole response),
with the short-range part v1 of Eq. (eq-partition).

TEST INFRASTRUCTURE ONLY (see the package header).

Steps, in the paper's order, on a product grid p = j * nang + a (radii r_j,
directions Omega_a, radial weights w_r(j) including r^2, angular weights
w_a summing to 4 pi):

  v1(r) = q (1/r - 1/R_S) for r < R_S, 0 beyond          Eq. (eq-partition), v_ext = q / r
  chi0_{lm;l'm'}(r_j, r_j') = sum_{a,a'} Y_lm(a) w_a chi0[(j,a),(j',a')] w_a' Y_l'm'(a')
                                                          expansion of chi0 in Y_lm
  S = I - chi0_lm W_r c W_r                               S of Sec. VI.E, l, l' <= l_resp
  chi = S^-1 chi0_lm
  rho_lm(r_j) = sum_j' w_r(j') chi_{lm;00}(r_j, r_j') sqrt(4 pi) v1(r_j')
  v_ind_lm(r_j) = sum_j' w_r(j') rho_lm(r_j') 4 pi / (2l+1) r_<^l / r_>^(l+1)

with c_l(r, r') = 4 pi / (2l+1) r_<^l / r_>^(l+1) and every radial integral
replaced by its quadrature (the operators compose with W_r between them).
Y_lm are real spherical harmonics: Y_l^0, sqrt(2) Re Y_l^m (m > 0),
sqrt(2) Im Y_l^|m| (m < 0), Y_l^m the complex harmonics with the
Condon-Shortley phase; index l^2 + l + m.
"""
import numpy as np
from scipy import special


def real_harmonics(lmax, dirs):
    """[ndir, (lmax+1)^2] real spherical harmonics at unit vectors dirs [ndir, 3]."""
    d = np.asarray(dirs, float)
    theta = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.zeros((d.shape[0], (lmax + 1) ** 2))
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            if hasattr(special, "sph_harm_y"):
                y = special.sph_harm_y(l, m, theta, phi)
            else:
                y = special.sph_harm(m, l, phi, theta)
            if m == 0:
                out[:, l * l + l] = y.real
            else:
                out[:, l * l + l + m] = np.sqrt(2.0) * y.real
                out[:, l * l + l - m] = np.sqrt(2.0) * y.imag
    return out


def short_range_potential(r, q, rs):
    r = np.asarray(r, float)
    return np.where(r < rs, q * (1.0 / r - 1.0 / rs), 0.0)


def radial_coulomb(radii, l):
    lo = np.minimum.outer(radii, radii)
    hi = np.maximum.outer(radii, radii)
    return 4.0 * np.pi / (2 * l + 1) * (lo / hi) ** l / hi


def induced_potential(chi0, pts, wts, nrad, nang, q, rs, lresp):
    """Return (radii, rho_lm [nrad, (lresp+1)^2], vind_lm [nrad, (lresp+1)^2])."""
    pts = np.asarray(pts, float)
    wts = np.asarray(wts, float)
    radii = np.linalg.norm(pts[::nang], axis=1)
    dirs = pts[:nang] / radii[0]
    w = wts.reshape(nrad, nang)
    w_r = w.sum(axis=1) / (4.0 * np.pi)           # radial weights (Lebedev weights sum to 4 pi)
    w_a = w[0] / w_r[0]
    L2 = (lresp + 1) ** 2
    Y = real_harmonics(lresp, dirs)                # [nang, L2]
    c4 = chi0.reshape(nrad, nang, nrad, nang)
    # chi0_{lm;l'm'}(r_j, r_j'), index (j, lm)
    A = np.einsum("al,jakb,bm->jlkm", Y * w_a[:, None], c4, Y * w_a[:, None]).reshape(nrad * L2, nrad * L2)
    C = np.zeros((nrad * L2, nrad * L2))
    for l in range(lresp + 1):
        cl = radial_coulomb(radii, l)
        for m in range(-l, l + 1):
            idx = np.arange(nrad) * L2 + l * l + l + m
            C[np.ix_(idx, idx)] = cl
    Wr = np.kron(np.diag(w_r), np.eye(L2))
    S = np.eye(nrad * L2) - A @ Wr @ C @ Wr
    chi = np.linalg.solve(S, A)
    u = np.zeros(nrad * L2)
    u[np.arange(nrad) * L2] = np.sqrt(4.0 * np.pi) * short_range_potential(radii, q, rs)
    rho = chi @ Wr @ u
    vind = C @ Wr @ rho
    return radii, rho.reshape(nrad, L2), vind.reshape(nrad, L2)


def on_grid(coeff_lm, pts, nang):
    """sum_lm f_lm(r_j) Y_lm(Omega_a) on the product grid (f given per shell)."""
    pts = np.asarray(pts, float)
    radii = np.linalg.norm(pts[::nang], axis=1)
    lmax = int(round(np.sqrt(coeff_lm.shape[1]))) - 1
    Y = real_harmonics(lmax, pts[:nang] / radii[0])
    return (coeff_lm @ Y.T).reshape(-1)
