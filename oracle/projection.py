"""Orbitals on a site grid by direct Fourier summation.

Eq. (bloch): psi_bk(r) = exp(i k.r) sum_G C_bk(G) exp(i G.r).  Sec. VI.B,
method 1: build the phase matrix P_k(r, G) = exp(i (k+G).r) and multiply by
the coefficient matrix C_k(G, b).  The normalisation Omega^-1/2 makes
int_cell |psi|^2 = 1 when sum_G |C(G)|^2 = 1 (coefficients of the Q factor of
a QR decomposition), and the k-sum of Sec. VI.D then carries weights w_k.
"""
import numpy as np


def reciprocal(cell):
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(cell, float)).T


def project_direct(cell, kpts, gvec, coeff, center, pts):
    """Return psi[p, k, b] at absolute positions center + pts[p].

    cell [3,3] (rows a1..a3), kpts [nk,3] cartesian, gvec [ng,3] integers,
    coeff [nk, ng, nb] complex, center [3], pts [npts,3].
    """
    cell = np.asarray(cell, float)
    omega = abs(np.linalg.det(cell))
    g = np.asarray(gvec, float) @ reciprocal(cell)             # [ng,3]
    r = np.asarray(center, float)[None, :] + np.asarray(pts, float)
    nk, ng, nb = coeff.shape
    out = np.empty((r.shape[0], nk, nb), np.complex128)
    for k in range(nk):
        phase = np.exp(1j * (r @ (kpts[k][None, :] + g).T))  # P_k(r, G)
        out[:, k, :] = (phase @ coeff[k]) / np.sqrt(omega)
    return out


def split_occupied(psi, energies, nocc, kweights):
    """Columns grouped as (k outer, band inner): occupied and unoccupied sets.

    Returns psi_o [npts, Ko], psi_u [npts, Ku], e_o, e_u, w_o, w_u where w_* is
    the k-weight of each column.
    """
    npts, nk, nb = psi.shape
    po, pu, eo, eu, wo, wu = [], [], [], [], [], []
    for k in range(nk):
        n = int(nocc[k])
        po.append(psi[:, k, :n]); pu.append(psi[:, k, n:])
        eo.append(energies[k, :n]); eu.append(energies[k, n:])
        wo.append(np.full(n, kweights[k])); wu.append(np.full(nb - n, kweights[k]))
    return (np.concatenate(po, 1), np.concatenate(pu, 1), np.concatenate(eo),
            np.concatenate(eu), np.concatenate(wo), np.concatenate(wu))
