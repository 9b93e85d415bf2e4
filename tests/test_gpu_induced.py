"""Induced density and potential of the screened short-range core-hole
potential (Sec. VI.E, Eq. (eq-partition)) vs the oracle, from the library's
own chi0.  Bars: 1e-10 relative for float64 contexts, 1e-5 for bf16x3
(inherited from the mixed chi0)."""
import numpy as np
import pytest

from oracle import induced as oind
from paper_2005_07834_gb300 import synth
from tests.gpu_util import Reference, max_rel, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def case260():
    wl = synth.single_site_260()
    return wl, Reference(wl)


@pytest.fixture(scope="module")
def case400():
    base = synth.tiny(nk=8, nocc=3, nunocc=5, gmax=2.5)
    wl = synth.Workload("tiny-400", base.orbitals, [synth.site_grid(base.sites[0].center, 8, 50, 2.5)], nfreq=12)
    return wl, Reference(wl)


def built(lrs, precision, wl, ref):
    scr = lrs.Screening(0, precision)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    scr.project()
    scr.build_chi0()
    return scr


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
def test_induced_matches_oracle(lrs, case260, precision, tol):
    wl, ref = case260
    s = wl.sites[0]
    scr = built(lrs, precision, wl, ref)
    assert scr.site_grid_shape(0) == (True, s.nrad, s.nang)
    for lresp in (0, 2, s.lmax):
        for q, rs in ((-1.0, 1.5), (1.0, 3.0)):
            rho, vind, grid = scr.induced_potential(0, q, rs, lresp)
            _, orho, ovind = oind.induced_potential(ref.chi0, s.pts, s.wts, s.nrad, s.nang, q, rs, lresp)
            ogrid = oind.on_grid(ovind, s.pts, s.nang)
            e = (rel_fro(rho, orho), rel_fro(vind, ovind), rel_fro(grid, ogrid),
                 max_rel(rho, orho), max_rel(vind, ovind), max_rel(grid, ogrid))
            print(f"{precision} l_resp {lresp} q {q} R_S {rs}: rho {e[0]:.1e} v_ind {e[1]:.1e} grid {e[2]:.1e}")
            assert max(e) < tol
    scr.close()


def test_induced_higher_multipoles(lrs, case400):
    """L = 5 site (8 shells x 50 directions): every l up to 5."""
    wl, ref = case400
    s = wl.sites[0]
    scr = built(lrs, "fp64", wl, ref)
    for lresp in (1, 5):
        rho, vind, grid = scr.induced_potential(0, -1.0, 2.0, lresp)
        _, orho, ovind = oind.induced_potential(ref.chi0, s.pts, s.wts, s.nrad, s.nang, -1.0, 2.0, lresp)
        assert rel_fro(rho, orho) < 1e-10 and rel_fro(vind, ovind) < 1e-10
    scr.close()


def test_induced_errors(lrs, case260):
    wl, ref = case260
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    with pytest.raises(lrs.LrsError) as e:
        scr.induced_potential(0, -1.0, 1.5, 0)            # no chi0 yet
    assert e.value.code == lrs.LRS_ERR_STATE
    scr.project()
    scr.build_chi0()
    for args in ((0, -1.0, 1.5, 4), (0, -1.0, 0.0, 0), (3, -1.0, 1.5, 0)):
        with pytest.raises(lrs.LrsError) as e:
            scr.induced_potential(*args)
        assert e.value.code == lrs.LRS_ERR_ARG
    scr.close()
    # a grid that is not a radial x angular product
    w2 = synth.tiny(nk=8, nocc=3, nunocc=5)
    s2 = w2.sites[0]
    s2.pts = s2.pts.copy()
    s2.pts[5] *= 1.01
    scr = lrs.Screening(0, "fp64")
    scr.load(w2.orbitals)
    scr.set_sites([s2])
    scr.set_frequency_quadrature(12)
    scr.project()
    scr.build_chi0()
    assert scr.site_grid_shape(0) == (False, 0, 0)
    with pytest.raises(lrs.LrsError) as e:
        scr.induced_potential(0, -1.0, 1.0, 0)
    assert e.value.code == lrs.LRS_ERR_UNSUPPORTED
    scr.close()
