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
