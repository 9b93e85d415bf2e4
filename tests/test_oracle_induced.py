"""Pins of the induced-potential oracle (Sec. VI.E core-hole response with the
v1 of Eq. (eq-partition)) against the full-grid Dyson solution, closed forms
of the real harmonics and reductions (CPU only)."""
import numpy as np
import pytest
from scipy import special

from oracle import chi0 as ochi0, coulomb, dyson, induced
from paper_2005_07834_gb300 import synth
from tests.oracle_problem import OracleProblem


@pytest.fixture(scope="module")
def prob():
    wl = synth.tiny(nk=8, nocc=3, nunocc=5, nrad=6, nang=26)      # L = 3, 156 points
    pr = OracleProblem(wl)
    chi = ochi0.chi0_pairs(*pr.args(), pr.t, pr.W)
    return pr, chi


def test_real_harmonics_orthonormal_and_addition_theorem():
    from scipy.integrate import lebedev_rule
    x, w = lebedev_rule(11)                                          # 50 points, degree 11
    Y = induced.real_harmonics(5, x.T)
    assert np.max(np.abs((Y * w[:, None]).T @ Y - np.eye(36))) < 1e-13
    # sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b)
    cosg = x.T @ x
    for l in range(6):
        blk = Y[:, l * l:(l + 1) ** 2]
        assert np.max(np.abs(blk @ blk.T - (2 * l + 1) / (4 * np.pi) * special.eval_legendre(l, cosg))) < 1e-13


def test_short_range_potential():
    r = np.array([0.5, 1.0, 2.0, 3.0, 3.5])
    v = induced.short_range_potential(r, -1.0, 3.0)
    assert np.allclose(v, [-(1 / 0.5 - 1 / 3.0), -(1 - 1 / 3.0), -(0.5 - 1 / 3.0), 0.0, 0.0])


@pytest.mark.parametrize("q,rs", [(-1.0, 1.5), (2.0, 10.0)])
def test_full_l_equals_the_grid_solution(prob, q, rs):
    """With every l <= L kept, rho_ind = chi Q v1 and v_ind = v Q rho_ind on the
    grid, chi = (I - chi0 Q v Q)^-1 chi0 by a dense solve on the full grid
    (independent route: no lm basis).  The screened interaction of the same
    Dyson equation then gives W Q rho = (W - v) Q v1 ... checked through
    v Q chi Q v = W - v."""
    pr, chi0 = prob
    s = pr.site
    q_w = s.wts
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    chi = np.linalg.solve(np.eye(s.npts) - (chi0 * q_w[None, :]) @ (v * q_w[None, :]), chi0)
    v1 = induced.short_range_potential(np.linalg.norm(s.pts, axis=1), q, rs)
    rho_ref = chi @ (q_w * v1)
    vind_ref = v @ (q_w * rho_ref)
    radii, rho, vind = induced.induced_potential(chi0, s.pts, s.wts, s.nrad, s.nang, q, rs, s.lmax)
    assert np.linalg.norm(induced.on_grid(vind, s.pts, s.nang) - vind_ref) < 1e-10 * np.linalg.norm(vind_ref)
    # the grid density has angular components beyond L (v filters them out of v_ind): compare
    # its l <= L components, sum_a w_a Y_lm(a) rho(r_j, a)
    w_a = s.wts[:s.nang] / (s.wts[:s.nang].sum() / (4.0 * np.pi))
    ylm = induced.real_harmonics(s.lmax, s.pts[:s.nang] / radii[0])
    rho_ref_lm = rho_ref.reshape(s.nrad, s.nang) @ (ylm * w_a[:, None])
    assert np.linalg.norm(rho - rho_ref_lm) < 1e-10 * np.linalg.norm(rho_ref_lm)
    # the grid chi is the one of the oracle's Dyson solution: v Q chi Q v = W - v
    w = dyson.screened_interaction(v, chi0, q_w)
    assert np.linalg.norm((v * q_w) @ (chi * q_w) @ v - (w - v)) < 1e-10 * np.linalg.norm(w - v)


def test_l0_truncation_is_exact_for_isotropic_response(prob):
    """chi0 that does not depend on directions has only an (00;00) block, so
    keeping l = 0 loses nothing."""
    pr, _ = prob
    s = pr.site
    rng = np.random.default_rng(8)
    b = rng.standard_normal((s.nrad, s.nrad))
    k = -(b @ b.T) * 1e-3
    chi = np.kron(k, np.ones((s.nang, s.nang)))
    _, rho0, v0 = induced.induced_potential(chi, s.pts, s.wts, s.nrad, s.nang, -1.0, 1.5, 0)
    _, rhoL, vL = induced.induced_potential(chi, s.pts, s.wts, s.nrad, s.nang, -1.0, 1.5, s.lmax)
    assert np.max(np.abs(vL[:, 1:])) < 1e-14 * np.max(np.abs(vL))
    assert np.allclose(v0[:, 0], vL[:, 0], rtol=1e-12, atol=0)
    assert np.allclose(rho0[:, 0], rhoL[:, 0], rtol=1e-12, atol=0)


def test_no_polarizability_no_induced_potential(prob):
    pr, _ = prob
    s = pr.site
    _, rho, vind = induced.induced_potential(np.zeros((s.npts, s.npts)), s.pts, s.wts, s.nrad, s.nang,
                                             -1.0, 1.5, 2)
    assert not rho.any() and not vind.any()
