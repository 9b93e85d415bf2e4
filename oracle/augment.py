"""Augmentation of site orbitals with all-electron character (Sec. VI.C,
Eq. (eq-aug1) and (eq-aug2)).

TEST INFRASTRUCTURE ONLY (see the package header).

  psi_ae(r) = psi_ps(r) + sum_lm sum_{nu,nu'} Y_lm(r^) [phi_ae_{nu l}(r) - phi_ps_{nu l}(r)]
                                    (A_l^-1)_{nu nu'} <phi_ps_{nu' l} Y_lm | psi_ps>
  A_{nu nu'; l} = int_0^{r_a} dr r^2 phi_ps_{nu l}(r) phi_ps_{nu' l}(r)

on the site's product grid: the radial integral is the grid's radial
quadrature over the shells with r_j <= r_a, the projection
<phi Y_lm | psi> = sum_{j: r_j <= r_a} sum_a w[(j,a)] phi(r_j) Y_lm(a) psi(j,a),
and the correction is applied on those shells.  Radial functions are given on
the shells: phi[l][nu][j].
"""
import numpy as np

from oracle.induced import real_harmonics


def augment(psi, pts, wts, nrad, nang, phi_ae, phi_ps, r_aug):
    """psi [npts, ncol] complex -> augmented copy."""
    pts = np.asarray(pts, float)
    wts = np.asarray(wts, float)
    radii = np.linalg.norm(pts[::nang], axis=1)
    inside = radii <= r_aug
    w = wts.reshape(nrad, nang)
    w_r = w.sum(axis=1) / (4.0 * np.pi)
    lmax = len(phi_ps) - 1
    Y = real_harmonics(lmax, pts[:nang] / radii[0])            # [nang, (lmax+1)^2]
    out = np.array(psi, dtype=np.complex128, copy=True)
    p3 = np.asarray(psi).reshape(nrad, nang, -1)
    o3 = out.reshape(nrad, nang, -1)
    for l in range(lmax + 1):
        fps = np.asarray(phi_ps[l], float) * inside[None, :]   # [nnu, nrad]
        fae = np.asarray(phi_ae[l], float) * inside[None, :]
        A = (fps * w_r[None, :]) @ fps.T
        Ainv = np.linalg.inv(A)
        for m in range(-l, l + 1):
            y = Y[:, l * l + l + m]
            # <phi_ps_{nu l} Y_lm | psi>: [nnu, ncol]
            proj = np.einsum("nj,ja,a,jac->nc", fps, w, y, p3)
            coef = Ainv @ proj
            o3 += np.einsum("nj,a,nc->jac", fae - fps, y, coef)
    return out
