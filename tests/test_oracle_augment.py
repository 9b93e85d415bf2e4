"""Pins of the augmentation oracle (Eq. eq-aug1, eq-aug2) (CPU only)."""
import numpy as np
import pytest

from oracle import augment, induced
from paper_2005_07834_gb300 import synth


def radial_set(radii, lmax, nnu, r_aug, seed=0):
    """Synthetic partial waves: smooth pseudo waves r^l exp(-a r^2) and
    all-electron waves that differ from them only inside r_aug."""
    rng = np.random.default_rng(seed)
    ps, ae = [], []
    for l in range(lmax + 1):
        a = rng.uniform(0.3, 1.5, nnu)
        b = rng.uniform(-0.5, 0.5, nnu)
        f = radii[None, :] ** l * np.exp(-a[:, None] * radii[None, :] ** 2)
        bump = np.where(radii < r_aug, np.sin(np.pi * radii / r_aug) ** 2, 0.0)
        ps.append(f)
        ae.append(f + b[:, None] * bump[None, :] * (1.0 + radii[None, :]))
    return ae, ps


@pytest.fixture(scope="module")
def site():
    return synth.site_grid(np.zeros(3), 12, 50, 3.0)                 # L = 5


def test_partial_waves_are_mapped_to_all_electron_waves(site):
    """A pseudo orbital that inside r_a is a combination of pseudo partial waves
    becomes the same combination of all-electron waves (the A^-1 of Eq. eq-aug2
    makes the discrete projection exact)."""
    s = site
    radii = np.linalg.norm(s.pts[::s.nang], axis=1)
    r_aug = 1.8
    ae, ps = radial_set(radii, 2, 3, r_aug)
    Y = induced.real_harmonics(2, s.pts[:s.nang] / radii[0])
    rng = np.random.default_rng(1)
    ncol = 4
    psi = np.zeros((s.nrad, s.nang, ncol), complex)
    want = np.zeros_like(psi)
    inside = radii <= r_aug
    for l in range(3):
        for m in range(-l, l + 1):
            alpha = rng.standard_normal((3, ncol)) + 1j * rng.standard_normal((3, ncol))
            y = Y[:, l * l + l + m]
            psi += np.einsum("nj,a,nc->jac", ps[l], y, alpha)
            want += np.einsum("nj,a,nc->jac", np.where(inside[None, :], ae[l], ps[l]), y, alpha)
    got = augment.augment(psi.reshape(s.npts, ncol), s.pts, s.wts, s.nrad, s.nang, ae, ps, r_aug)
    # A_l of nearby Gaussians is ill-conditioned (cond ~1e5): rounding, not the method, sets the bar
    assert np.max(np.abs(got - want.reshape(s.npts, ncol))) < 1e-9 * np.max(np.abs(want))


def test_identical_partial_waves_change_nothing(site):
    s = site
    radii = np.linalg.norm(s.pts[::s.nang], axis=1)
    _, ps = radial_set(radii, 3, 2, 2.0)
    psi = np.random.default_rng(2).standard_normal((s.npts, 3)) + 0j
    got = augment.augment(psi, s.pts, s.wts, s.nrad, s.nang, ps, ps, 2.0)
    assert np.array_equal(got, psi)


def test_only_shells_inside_the_radius_change(site):
    s = site
    radii = np.linalg.norm(s.pts[::s.nang], axis=1)
    ae, ps = radial_set(radii, 2, 2, 1.5)
    psi = np.random.default_rng(3).standard_normal((s.npts, 5)) * (1 + 0.5j)
    got = augment.augment(psi, s.pts, s.wts, s.nrad, s.nang, ae, ps, 1.5)
    outside = np.repeat(radii > 1.5, s.nang)
    assert np.array_equal(got[outside], psi[outside])
    assert np.max(np.abs(got[~outside] - psi[~outside])) > 1e-3
