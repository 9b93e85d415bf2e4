"""Mixed-precision (bf16x3 tensor-core) path vs the FP64 oracle through the C-ABI.

Tolerance: 1e-5, both relative Frobenius and element-wise (max |d| / max |ref|), for psi,
chi0, W and W - v.
"""
import numpy as np
import pytest

from paper_2005_07834_gb300 import synth
from tests.gpu_util import Reference, max_rel, public_psi, rel_fro

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
    assert max_rel(psi, public_psi(cfg_260.pr)) < TOL
    scr.close()


def test_mixed_chi0_from_exact_orbitals(lrs, cfg_260):
    scr = screening(lrs, synth.single_site_260())
    scr.set_site_orbitals(0, public_psi(cfg_260.pr))
    scr.build_chi0()
    scr.synchronize()
    chi = scr.get_chi0(0)
    assert rel_fro(chi, cfg_260.chi0) < TOL
    assert max_rel(chi, cfg_260.chi0) < TOL
    assert np.array_equal(chi, chi.T)
    scr.close()


def test_mixed_full_build(lrs, cfg_260):
    ref = cfg_260
    scr = screening(lrs, synth.single_site_260())
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    chi = scr.get_chi0(0)
    w = scr.get_w(0)
    e = {"chi0": (rel_fro(chi, ref.chi0), max_rel(chi, ref.chi0)), "w": (rel_fro(w, ref.w), max_rel(w, ref.w)),
         "w-v": (rel_fro(w - ref.v, ref.w - ref.v), max_rel(w - ref.v, ref.w - ref.v))}
    print("bf16x3 260-point site (fro, max):", {k: (f"{a:.2e}", f"{b:.2e}") for k, (a, b) in e.items()})
    for k, (a, b) in e.items():
        assert a < TOL and b < TOL, (k, a, b)
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
        chi, w = scr.get_chi0(i), scr.get_w(i)
        assert rel_fro(chi, ref.chi0) < TOL and max_rel(chi, ref.chi0) < TOL
        assert rel_fro(w, ref.w) < TOL and max_rel(w, ref.w) < TOL
        assert rel_fro(w - ref.v, ref.w - ref.v) < TOL and max_rel(w - ref.v, ref.w - ref.v) < TOL
    scr.close()
