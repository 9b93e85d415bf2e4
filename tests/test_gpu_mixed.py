"""Mixed-precision (bf16x3 tensor-core) path vs the FP64 oracle through the C-ABI.

Tolerance: 1e-5 relative Frobenius for chi0 and W (measured ~1e-7 and ~1e-9).
"""
import numpy as np
import pytest

from paper_2005_07834_gb300 import synth
from tests.gpu_util import Reference, public_psi, rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def cfg_260():
    return Reference(synth.single_site_260())


def screening(lrs, wl, precision="bf16x3"):
    scr = lrs.Screening(0, precision)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    return scr


def test_mixed_projection(lrs, cfg_260):
    scr = screening(lrs, synth.single_site_260())
    scr.project()
    psi = scr.get_site_orbitals(0)
    err = rel_fro(psi, public_psi(cfg_260.pr))
    assert err < TOL, err
    scr.close()


def test_mixed_chi0_from_exact_orbitals(lrs, cfg_260):
    scr = screening(lrs, synth.single_site_260())
    scr.set_site_orbitals(0, public_psi(cfg_260.pr))
    scr.build_chi0()
    scr.synchronize()
    chi = scr.get_chi0(0)
    assert rel_fro(chi, cfg_260.chi0) < TOL
    assert np.array_equal(chi, chi.T)
    scr.close()


def test_mixed_full_build(lrs, cfg_260):
    ref = cfg_260
    scr = screening(lrs, synth.single_site_260())
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    assert rel_fro(scr.get_chi0(0), ref.chi0) < TOL
    w = scr.get_w(0)
    assert rel_fro(w, ref.w) < TOL
    assert rel_fro(w - ref.v, ref.w - ref.v) < 1e-3
    scr.close()


def test_mixed_ragged_multisite(lrs):
    wl = synth.tiny(nk=8, nocc=3, nunocc=5)
    wl.sites.append(synth.site_grid(np.array([1.0, 2.0, 0.5]), 5, 14, 2.5))
    scr = screening(lrs, wl)
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    for i in range(2):
        ref = Reference(wl, site=i)
        assert rel_fro(scr.get_chi0(i), ref.chi0) < TOL
        assert rel_fro(scr.get_w(i), ref.w) < TOL
    scr.close()
