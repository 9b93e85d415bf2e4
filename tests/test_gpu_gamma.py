"""Gamma-point real orbitals (Sec. VI.F): detection, and chi0 / W from the
real-operand tensor-core contraction (half the products) vs the oracle and
vs the complex contraction.  Bars: 1e-10 (float64 context), 1e-5 (bf16x3)."""
import numpy as np
import pytest

from paper_2005_07834_gb300 import synth
from tests.gpu_util import max_rel, Reference, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def case():
    wl = synth.gamma_site_260()
    return wl, Reference(wl)


def build(lrs, precision, wl, ref, real_mode=None):
    scr = lrs.Screening(0, precision)
    if real_mode is not None:
        scr.set_option(lrs.LRS_OPT_REAL_ORBITALS, real_mode)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    return scr


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
def test_gamma_real_orbitals(lrs, case, precision, tol):
    wl, ref = case
    scr = build(lrs, precision, wl, ref)
    assert scr.orbitals_are_real()
    chi, w = scr.get_chi0(0), scr.get_w(0)
    e_chi, e_w = rel_fro(chi, ref.chi0), rel_fro(w, ref.w)
    m_chi, m_w = max_rel(chi, ref.chi0), max_rel(w, ref.w)
    print(f"{precision} Gamma real: chi0 {e_chi:.2e} (max {m_chi:.2e}), W {e_w:.2e} (max {m_w:.2e})")
    assert e_chi < tol and e_w < tol and m_chi < tol and m_w < tol
    assert np.array_equal(chi, chi.T)
    scr.close()


@pytest.mark.parametrize("tile_n", [64, 128])
def test_gamma_sites_in_one_launch(lrs, tile_n):
    """Three Gamma-point sites of 260, 700 and 350 points (3, 6 and 3 row tiles of 128, ragged
    last ones) in one chi0 launch: with real orbitals each frequency's product is symmetric and
    only the tiles reaching the lower triangle are computed (q (T + 1) T / 2 of them, q = 128 /
    tile_n).  Each site's chi0 against the oracle (bf16x3 bar 1e-5, element-wise too), and
    exactly symmetric."""
    wl = synth.gamma_site_260()
    c = wl.sites[0].center
    wl.sites = [wl.sites[0], synth.site_grid(c + 0.7, 14, 50, 3.5), synth.site_grid(c - 1.1, 25, 14, 3.0)]
    refs = [Reference(wl, site=i) for i in range(3)]
    scr = lrs.Screening(0, "bf16x3")
    scr.set_option(lrs.LRS_OPT_CHI0_TILE_N, tile_n)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=refs[0].pr.mu, zeta=refs[0].pr.zeta)
    scr.project()
    scr.build_chi0()
    assert scr.orbitals_are_real()
    for i, ref in enumerate(refs):
        chi = scr.get_chi0(i)
        e, m = rel_fro(chi, ref.chi0), max_rel(chi, ref.chi0)
        print(f"tile_n {tile_n}, site {i} ({chi.shape[0]} points): chi0 {e:.2e} (max {m:.2e})")
        assert e < 1e-5 and m < 1e-5
        assert np.array_equal(chi, chi.T)
    scr.close()


def test_real_and_complex_contractions_agree(lrs, case):
    wl, ref = case
    a = build(lrs, "bf16x3", wl, ref)
    b = build(lrs, "bf16x3", wl, ref, lrs.LRS_REAL_OFF)
    d = rel_fro(a.get_chi0(0), b.get_chi0(0))
    print(f"bf16x3 real vs complex contraction: {d:.2e}")
    assert d < 1e-5
    a.close()
    b.close()


def test_complex_orbitals_are_not_real(lrs):
    wl = synth.tiny(nk=1, nocc=3, nunocc=5)          # one k at Gamma, but complex random coefficients
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    assert not scr.orbitals_are_real()
    scr.close()
