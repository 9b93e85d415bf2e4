"""Pins of the method-2 projection oracle (Sec. VI.B: FFT to the cell grid,
3rd-degree Lagrange interpolation, Bloch phase) against the direct Fourier sum,
polynomial exactness and the interpolation order (CPU only)."""
import numpy as np
import pytest

from oracle import projection
from paper_2005_07834_gb300 import synth


@pytest.fixture(scope="module")
def orb():
    return synth.tiny(nk=8, nocc=3, nunocc=5, gmax=3.5).orbitals   # |n_i| <= 3: 7 points needed


def test_lagrange_weights_reproduce_cubics():
    """Through nodes -1, 0, 1, 2 the weights reproduce 1, m, m^2, m^3 at t."""
    t = np.random.default_rng(3).uniform(0.0, 1.0, 50)
    w = projection.lagrange3_weights(t)
    m = np.array([-1.0, 0.0, 1.0, 2.0])
    for p in range(4):
        assert np.max(np.abs(w @ m ** p - t ** p)) < 1e-14
    # at a node the interpolant returns the node value
    assert np.allclose(projection.lagrange3_weights(0.0), [0.0, 1.0, 0.0, 0.0], atol=0, rtol=0)


def test_nodes_reproduce_the_direct_sum(orb):
    """At FFT-grid nodes (t = 0 in every direction) interpolation returns the
    node value, which is the exact Fourier sum when the grid holds every G:
    pins the FFT sign, normalisation, index wrap, the phase and Omega^-1/2."""
    o = orb
    n = (12, 12, 12)
    rng = np.random.default_rng(4)
    m = rng.integers(0, 12, (40, 3))
    nodes = (m / np.array(n)) @ o.cell
    ref = projection.project_direct(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), nodes)
    got = projection.project_fft_lagrange(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), nodes, n)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_lattice_translation_gives_the_bloch_factor(orb):
    """psi(r + a_i) = exp(i k.a_i) psi(r): checks the periodic stencil across the cell edge."""
    o = orb
    n = (12, 12, 12)
    rng = np.random.default_rng(5)
    r = rng.uniform(0.0, 1.0, (30, 3)) @ o.cell
    base = projection.project_fft_lagrange(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), r, n)
    for i in range(3):
        moved = projection.project_fft_lagrange(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), r + o.cell[i], n)
        phase = np.exp(1j * (o.kpts @ o.cell[i]))
        assert np.max(np.abs(moved - base * phase[None, :, None])) < 1e-12


def test_interpolation_error_is_fourth_order():
    """One plane wave exp(i G.r) sampled on N and 2N points per direction:
    the cubic interpolant's error falls by about 2^4."""
    cell = synth.cubic_cell(6.0)
    gvec = np.array([[1, 0, 0], [0, 1, 1], [1, -1, 0]])
    coeff = np.zeros((1, 3, 1), complex)
    coeff[0, :, 0] = [0.6, 0.5j, -0.4]
    kpts = np.zeros((1, 3))
    r = np.random.default_rng(6).uniform(0.0, 1.0, (200, 3)) @ cell
    ref = projection.project_direct(cell, kpts, gvec, coeff, np.zeros(3), r)
    err = []
    for n in (12, 24, 48):
        got = projection.project_fft_lagrange(cell, kpts, gvec, coeff, np.zeros(3), r, (n, n, n))
        err.append(np.max(np.abs(got - ref)))
    assert 12.0 < err[0] / err[1] < 20.0
    assert 12.0 < err[1] / err[2] < 20.0


def test_grid_too_small_is_rejected(orb):
    with pytest.raises(ValueError):
        projection.project_fft_lagrange(orb.cell, orb.kpts, orb.gvec, orb.coeff, np.zeros(3),
                                        np.zeros((1, 3)), (6, 12, 12))
