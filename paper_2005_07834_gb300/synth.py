"""Seeded synthetic inputs for local real-space screening (Vinson & Shirley).

This module draws inputs only: plane-wave coefficients and band energies of a
periodic cell (the data a DFT code hands to the screening step, Sec. VI.A-B,
Eq. (bloch)), k-points and their weights, site-centred product grids
(Gauss-Legendre radial shells times a Lebedev angular set, App. D.1) and the
weights of a scalar loss.  It holds none of the method's arithmetic (no
projection, Green's function, quadrature, Coulomb operator or Dyson solve), so
that both the FP64 CPU oracle and the CUDA path can consume the same arrays.

Recipe (per workload):
  * G set: integer triples n with |2 pi n / a| <= gmax, lexicographic order.
  * per k, in ascending k order: Re C ~ N(0,1) [ng x nb], Im C ~ N(0,1),
    occupied energies ~ U[-1.0, -0.1] Ha sorted, unoccupied ~ U[0.1, 3.0] Ha
    sorted; C <- (Re + i Im) * exp(-|G|^2 / 2) row-wise, then the Q factor of a
    reduced QR, so that sum_G |C_b(G)|^2 = 1 and the bands are orthonormal.
  * site grid: n-point Gauss-Legendre on [0, R] (r = R (x+1)/2, radial weight
    (R/2) w r^2) times a Lebedev rule; radial-major point order; the point
    weight is radial weight x angular weight (angular weights sum to 4 pi).
  * Coulomb multipole cutoff lmax = floor(degree / 2) of the Lebedev rule.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Lebedev set size -> polynomial degree it integrates exactly.
LEBEDEV_DEGREE = {6: 3, 14: 5, 26: 7, 38: 9, 50: 11, 74: 13, 86: 15, 110: 17,
                  146: 19, 170: 21, 194: 23}


@dataclass
class Orbitals:
    cell: np.ndarray          # [3,3] bohr, rows are lattice vectors a1, a2, a3
    kpts: np.ndarray          # [nk,3] cartesian, bohr^-1
    kweights: np.ndarray      # [nk], sums to 1
    gvec: np.ndarray          # [ng,3] int32, multiples of the reciprocal vectors
    coeff: np.ndarray         # [nk, ng, nb] complex128
    energies: np.ndarray      # [nk, nb] Ha, occupied bands first
    nocc: np.ndarray          # [nk] int32

    @property
    def nk(self):
        return self.coeff.shape[0]

    @property
    def ng(self):
        return self.coeff.shape[1]

    @property
    def nbands(self):
        return self.coeff.shape[2]


@dataclass
class SiteGrid:
    center: np.ndarray        # [3] bohr
    pts: np.ndarray           # [npts,3] offsets from the centre, bohr
    wts: np.ndarray           # [npts] integration weights (include r^2)
    lmax: int                 # Coulomb multipole cutoff
    nrad: int
    nang: int

    @property
    def npts(self):
        return self.pts.shape[0]


@dataclass
class Workload:
    name: str
    orbitals: Orbitals
    sites: list = field(default_factory=list)
    nfreq: int = 16
    fft_grid: tuple = (0, 0, 0)   # cell grid of the method-2 projection (0: automatic)


def cubic_cell(a: float) -> np.ndarray:
    return np.eye(3) * float(a)


def g_sphere(cell: np.ndarray, gmax: float) -> np.ndarray:
    """Integer triples n with |n . B| <= gmax (B = reciprocal rows), lexicographic."""
    recip = 2.0 * np.pi * np.linalg.inv(cell).T
    nmax = int(np.ceil(gmax / np.min(np.linalg.norm(recip, axis=1)))) + 1
    r = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    g = n @ recip
    keep = np.linalg.norm(g, axis=1) <= gmax + 1e-12
    return n[keep].astype(np.int32)


def gamma_centred_kmesh(cell: np.ndarray, m: int):
    recip = 2.0 * np.pi * np.linalg.inv(cell).T
    r = np.arange(m) / m
    f = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    return f @ recip, np.full(f.shape[0], 1.0 / f.shape[0])


def draw_orbitals(cell, kpts, kweights, gmax, nocc, nunocc, seed=0) -> Orbitals:
    rng = np.random.default_rng(seed)
    gvec = g_sphere(cell, gmax)
    recip = 2.0 * np.pi * np.linalg.inv(cell).T
    gnorm = np.linalg.norm(gvec @ recip, axis=1)
    env = np.exp(-gnorm ** 2 / 2.0)
    nk, ng, nb = len(kpts), len(gvec), nocc + nunocc
    coeff = np.empty((nk, ng, nb), np.complex128)
    energies = np.empty((nk, nb))
    for k in range(nk):
        re = rng.standard_normal((ng, nb))
        im = rng.standard_normal((ng, nb))
        eo = np.sort(rng.uniform(-1.0, -0.1, nocc))
        eu = np.sort(rng.uniform(0.1, 3.0, nunocc))
        c = (re + 1j * im) * env[:, None]
        q, _ = np.linalg.qr(c)
        coeff[k] = q
        energies[k, :nocc] = eo
        energies[k, nocc:] = eu
    return Orbitals(np.asarray(cell, float), np.asarray(kpts, float),
                    np.asarray(kweights, float), gvec, coeff, energies,
                    np.full(nk, nocc, np.int32))


def site_grid(center, nrad, nang, radius) -> SiteGrid:
    from scipy.integrate import lebedev_rule
    deg = LEBEDEV_DEGREE[nang]
    omega, wang = lebedev_rule(deg)          # [3,nang], sum 4 pi
    x, w = np.polynomial.legendre.leggauss(nrad)
    r = radius * (x + 1.0) / 2.0
    wrad = (radius / 2.0) * w * r ** 2
    pts = (r[:, None, None] * omega.T[None, :, :]).reshape(-1, 3)
    wts = (wrad[:, None] * wang[None, :]).reshape(-1)
    return SiteGrid(np.asarray(center, float), pts, wts, deg // 2, nrad, nang)


def loss_weights(npts: int, seed: int = 2) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(npts)


# ----------------------------------------------------------------------------
# Workloads with the shapes of the paper's runs (16 imaginary frequencies,
# site grids of a few thousand points, tens of bands per cell).
# ----------------------------------------------------------------------------

def draw_real_orbitals(cell, gmax, nocc, nunocc, seed=0) -> Orbitals:
    """Gamma-point orbitals with time-reversal symmetry (real in real space).

    Draw order: a real matrix R [ng x nb] standard normal, occupied energies
    U[-1,-0.1] sorted, unoccupied U[0.1,3.0] sorted.  The rows of R are the
    coefficients in the real orthonormal basis {1, sqrt(2) cos(G.r), sqrt(2)
    sin(G.r)} (one cos and one sin row per pair +-G, G the lexicographically
    larger of the pair), each times exp(-|G|^2/2); reduced QR keeps Q; then
    C(G) = (a - i b)/sqrt(2), C(-G) = (a + i b)/sqrt(2), C(0) = a, a unitary map,
    so the columns stay orthonormal and C(-G) = conj C(G).
    """
    rng = np.random.default_rng(seed)
    gvec = g_sphere(cell, gmax)
    recip = 2.0 * np.pi * np.linalg.inv(cell).T
    gnorm = np.linalg.norm(gvec @ recip, axis=1)
    env = np.exp(-gnorm ** 2 / 2.0)
    ng, nb = len(gvec), nocc + nunocc
    index = {tuple(g): i for i, g in enumerate(gvec)}
    zero = index[(0, 0, 0)]
    pos = [i for i, g in enumerate(gvec) if tuple(g) > (0, 0, 0)]
    neg = [index[tuple(-gvec[i])] for i in pos]
    r = rng.standard_normal((ng, nb))
    eo = np.sort(rng.uniform(-1.0, -0.1, nocc))
    eu = np.sort(rng.uniform(0.1, 3.0, nunocc))
    rows = np.concatenate([[zero], pos, pos])            # basis order: 1, cos rows, sin rows
    q, _ = np.linalg.qr(r * env[rows][:, None])
    coeff = np.empty((ng, nb), np.complex128)
    npair = len(pos)
    a, b = q[1:1 + npair], q[1 + npair:]
    coeff[zero] = q[0]
    coeff[pos] = (a - 1j * b) / np.sqrt(2.0)
    coeff[neg] = (a + 1j * b) / np.sqrt(2.0)
    energies = np.concatenate([eo, eu])[None, :]
    return Orbitals(np.asarray(cell, float), np.zeros((1, 3)), np.ones(1), gvec, coeff[None], energies,
                    np.full(1, nocc, np.int32))


def gamma_site_260(seed=0) -> Workload:
    """Gamma-point real orbitals: a = 10 bohr, |G| <= 3, 64 occ + 192 unocc, 10 GL x 26 Lebedev, 12 freq."""
    cell = cubic_cell(10.0)
    orb = draw_real_orbitals(cell, 3.0, 64, 192, seed)
    site = site_grid(np.full(3, 5.0), 10, 26, 4.0)
    return Workload("gamma-site-260pt-b256", orb, [site], nfreq=12, fft_grid=(16, 16, 16))


def gamma_site_3520(seed=0) -> Workload:
    """Gamma-point real orbitals: a = 20 bohr, |G| <= 4, 1024 occ + 4096 unocc, 32 GL x 110 Lebedev, 16 freq."""
    cell = cubic_cell(20.0)
    orb = draw_real_orbitals(cell, 4.0, 1024, 4096, seed)
    site = site_grid(np.full(3, 10.0), 32, 110, 6.0)
    return Workload("gamma-site-3520pt-b5120", orb, [site], nfreq=16, fft_grid=(48, 48, 48))


def single_site_260(seed=0) -> Workload:
    """a = 10 bohr, |G| <= 3, 2x2x2 k, 8 occ + 24 unocc per k, 10 GL x 26 Lebedev, 12 freq."""
    cell = cubic_cell(10.0)
    k, w = gamma_centred_kmesh(cell, 2)
    orb = draw_orbitals(cell, k, w, 3.0, 8, 24, seed)
    site = site_grid(np.full(3, 5.0), 10, 26, 4.0)
    return Workload("single-site-260pt-k8-b32", orb, [site], nfreq=12, fft_grid=(16, 16, 16))


def single_site_3520(seed=0) -> Workload:
    """a = 20 bohr, |G| <= 4, 2x2x2 k, 128 occ + 512 unocc per k, 32 GL x 110 Lebedev, 16 freq."""
    cell = cubic_cell(20.0)
    k, w = gamma_centred_kmesh(cell, 2)
    orb = draw_orbitals(cell, k, w, 4.0, 128, 512, seed)
    site = site_grid(np.full(3, 10.0), 32, 110, 6.0)
    return Workload("single-site-3520pt-k8-b640", orb, [site], nfreq=16, fft_grid=(48, 48, 48))


def batched_sites(orbitals: Orbitals, nsites=64, seed=1, radius=4.0) -> list:
    """Uneven sites: centres uniform in the cell, 16..48 radial shells, Lebedev 50/110/194."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, (nsites, 3)) @ orbitals.cell
    nrad = rng.integers(16, 49, nsites)
    nang = rng.choice(np.array([50, 110, 194]), nsites)
    return [site_grid(centres[i], int(nrad[i]), int(nang[i]), radius) for i in range(nsites)]


def batched_64_sites(seed=0) -> Workload:
    base = single_site_260(seed)
    return Workload("batched-64-sites-k8-b32", base.orbitals, batched_sites(base.orbitals), nfreq=16,
                    fft_grid=(16, 16, 16))


def large_cell_16_sites(seed=0) -> Workload:
    """a = 40 bohr, |G| <= 4, Gamma + (1/8,2/8,3/8), 1024 occ + 3072 unocc, 16 sites 48 GL x 194, 20 freq."""
    cell = cubic_cell(40.0)
    recip = 2.0 * np.pi * np.linalg.inv(cell).T
    k = np.array([[0.0, 0.0, 0.0], [1 / 8, 2 / 8, 3 / 8]]) @ recip
    orb = draw_orbitals(cell, k, np.array([0.5, 0.5]), 4.0, 1024, 3072, seed)
    rng = np.random.default_rng(1)
    centres = rng.uniform(0.0, 1.0, (16, 3)) @ cell
    sites = [site_grid(c, 48, 194, 6.0) for c in centres]
    return Workload("large-cell-16-sites-k2-b4096", orb, sites, nfreq=20, fft_grid=(96, 96, 96))


def tiny(nk=1, nocc=3, nunocc=5, gmax=2.0, a=6.0, nrad=3, nang=14, seed=0) -> Workload:
    """Small case for brute-force checks (one or a few k-points)."""
    cell = cubic_cell(a)
    if nk == 1:
        k, w = np.zeros((1, 3)), np.ones(1)
    else:
        k, w = gamma_centred_kmesh(cell, 2)
    orb = draw_orbitals(cell, k, w, gmax, nocc, nunocc, seed)
    site = site_grid(np.full(3, a / 2), nrad, nang, 2.0)
    return Workload("tiny", orb, [site], nfreq=12)
