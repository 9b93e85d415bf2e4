"""Pins of the ALDA oracle (Eq. chi-alda, kxc_alda) (CPU only)."""
import numpy as np
import pytest

from oracle import alda, chi0 as ochi0, coulomb, dyson, projection
from paper_2005_07834_gb300 import synth
from tests.oracle_problem import OracleProblem


@pytest.fixture(scope="module")
def prob():
    wl = synth.tiny(nk=8, nocc=3, nunocc=5, nrad=4, nang=26)
    pr = OracleProblem(wl)
    chi = ochi0.chi0_pairs(*pr.args(), pr.t, pr.W)
    v = coulomb.coulomb_multipole(pr.site.pts, pr.site.lmax)
    return pr, chi, v


def test_zero_kernel_is_rpa(prob):
    pr, chi, v = prob
    w_rpa = dyson.screened_interaction(v, chi, pr.site.wts)
    w0 = alda.screened_interaction_alda(chi, v, np.zeros(pr.site.npts), pr.site.wts)
    assert np.linalg.norm(w0 - w_rpa) < 1e-12 * np.linalg.norm(w_rpa)


def test_dressed_polarizability_route(prob):
    """chi~ of Eq. (chi-alda) equals the RPA Dyson chain of chi_eff = (I - chi0 D)^-1 chi0:
    W~ from the dense ALDA solve = W of dyson.screened_interaction(v, chi_eff)."""
    pr, chi, v = prob
    s = pr.site
    n = alda.density(pr.po, pr.wo)
    f = alda.fx_exchange(n)
    d = f * s.wts
    chi_eff = np.linalg.solve(np.eye(s.npts) - chi * d[None, :], chi)
    w_a = alda.screened_interaction_alda(chi, v, f, s.wts)
    w_b = dyson.screened_interaction(v, chi_eff, s.wts)
    assert np.linalg.norm(w_a - w_b) < 1e-11 * np.linalg.norm(w_a)
    assert np.linalg.norm(chi_eff - chi_eff.T) < 1e-12 * np.linalg.norm(chi_eff)
    # the exchange kernel is attractive: W~ differs from W by more than rounding
    w_rpa = dyson.screened_interaction(v, chi, s.wts)
    assert np.linalg.norm(w_a - w_rpa) > 1e-6 * np.linalg.norm(w_rpa)


def test_exchange_kernel_is_the_second_derivative_of_the_energy():
    """f_x = d^2 e_x / dn^2, checked by 5-point finite differences (as the paper forms f_xc)."""
    n = np.array([1e-3, 1e-2, 0.1, 1.0])
    h = 1e-3 * n
    e = alda.exchange_energy_density
    d2 = (-e(n + 2 * h) + 16 * e(n + h) - 30 * e(n) + 16 * e(n - h) - e(n - 2 * h)) / (12 * h ** 2)
    assert np.allclose(alda.fx_exchange(n), d2, rtol=1e-6, atol=0)


def test_density_integrates_to_the_electron_count():
    """n from orthonormal orbitals on a uniform cell grid: int_cell n = 2 sum_k w_k nocc_k."""
    wl = synth.tiny(nk=8, nocc=3, nunocc=5)
    o = wl.orbitals
    m = 12
    x = np.arange(m) / m
    grid = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3) @ o.cell
    psi = projection.project_direct(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), grid)
    po, _, _, _, wo, _ = projection.split_occupied(psi, o.energies, o.nocc, o.kweights)
    omega = abs(np.linalg.det(o.cell))
    total = alda.density(po, wo).sum() * omega / m ** 3
    assert abs(total - 2.0 * np.sum(o.kweights * o.nocc)) < 1e-10


def test_exchange_constant_against_the_uniform_gas_values():
    """Pins the Dirac constant (3/pi)^(1/3) that both the energy and the kernel carry, against
    textbook values of the uniform electron gas in Hartree atomic units: the exchange energy per
    electron is -0.458165 / r_s Ha and the exchange potential -0.610887 / r_s Ha, with
    n = 3 / (4 pi r_s^3).  A wrong constant shared by e_x and f_x passes the second-derivative
    check but fails these."""
    for rs in (1.0, 2.0, 5.0):
        n = 3.0 / (4.0 * np.pi * rs ** 3)
        eps_x = float(alda.exchange_energy_density(n)) / n
        assert abs(eps_x - (-0.458165 / rs)) < 1e-6 / rs, (rs, eps_x)
        h = 1e-4 * n
        v_x = float(alda.exchange_energy_density(n + h) - alda.exchange_energy_density(n - h)) / (2 * h)
        assert abs(v_x - (-0.610887 / rs)) < 1e-6 / rs, (rs, v_x)
        # f_x = dv_x/dn = -(1/3) (3/pi)^(1/3) n^(-2/3) = v_x / (3 n) for the n^(1/3) potential
        assert abs(float(alda.fx_exchange(n)) - (-0.610887 / rs) / (3.0 * n)) < 1e-6 / (rs * 3.0 * n)
