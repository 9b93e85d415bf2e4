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


# ----------------------------------------------------------------------------
# Sec. VI.B, method 2: FFT to a real-space grid over the cell, cubic Lagrange
# interpolation to the site points, then the Bloch phase.
# ----------------------------------------------------------------------------

def lagrange3_weights(t):
    """Weights of the 4-point (3rd-degree) Lagrange interpolant through nodes
    -1, 0, 1, 2 evaluated at t (the point lies between nodes 0 and 1)."""
    t = np.asarray(t, float)
    return np.stack([-t * (t - 1.0) * (t - 2.0) / 6.0,
                     (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0,
                     -(t + 1.0) * t * (t - 2.0) / 2.0,
                     (t + 1.0) * t * (t - 1.0) / 6.0], axis=-1)


def periodic_part_on_grid(gvec, coeff_k, grid):
    """u_k(x) = sum_G C_k(G) exp(i G.x) at the nodes x = sum_i (m_i / N_i) a_i.

    With G = sum n_i b_i, G.x = 2 pi sum_i n_i m_i / N_i: an inverse DFT of the
    coefficients placed at n mod N.  Returns [N1, N2, N3, nb].
    """
    n1, n2, n3 = grid
    nb = coeff_k.shape[1]
    c = np.zeros((n1, n2, n3, nb), np.complex128)
    g = np.asarray(gvec)
    c[g[:, 0] % n1, g[:, 1] % n2, g[:, 2] % n3, :] = coeff_k
    return np.fft.ifftn(c, axes=(0, 1, 2)) * (n1 * n2 * n3)


def project_fft_lagrange(cell, kpts, gvec, coeff, center, pts, grid):
    """psi[p, k, b] by method 2: FFT of the periodic part to the cell grid,
    3rd-degree Lagrange interpolation in each lattice direction (nodes
    i0 - 1 .. i0 + 2 around the point, i0 = floor of its grid coordinate,
    indices periodic), then exp(i k.r) / sqrt(Omega)."""
    cell = np.asarray(cell, float)
    omega = abs(np.linalg.det(cell))
    n = np.asarray(grid, int)
    g = np.asarray(gvec)
    for d in range(3):
        if n[d] < 2 * np.abs(g[:, d]).max() + 1:
            raise ValueError("FFT grid does not hold every G without aliasing")
    r = np.asarray(center, float)[None, :] + np.asarray(pts, float)
    s = (r @ np.linalg.inv(cell)) * n[None, :]      # grid coordinates
    i0 = np.floor(s).astype(int)
    w = lagrange3_weights(s - i0)                   # [npts, 3, 4]
    nk, ng, nb = coeff.shape
    out = np.empty((r.shape[0], nk, nb), np.complex128)
    for k in range(nk):
        u = periodic_part_on_grid(g, coeff[k], n)
        acc = np.zeros((r.shape[0], nb), np.complex128)
        for a in range(4):
            ia = (i0[:, 0] + a - 1) % n[0]
            for b in range(4):
                ib = (i0[:, 1] + b - 1) % n[1]
                for c in range(4):
                    ic = (i0[:, 2] + c - 1) % n[2]
                    wt = w[:, 0, a] * w[:, 1, b] * w[:, 2, c]
                    acc += wt[:, None] * u[ia, ib, ic, :]
        out[:, k, :] = acc * np.exp(1j * (r @ kpts[k]))[:, None] / np.sqrt(omega)
    return out
