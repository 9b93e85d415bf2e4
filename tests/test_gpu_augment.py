"""All-electron augmentation (Eq. eq-aug1, eq-aug2) on the GPU vs the oracle,
and the chi0 and W built from the augmented orbitals.  Bars: 1e-10 (float64
context), 1e-5 (bf16x3)."""
import numpy as np
import pytest

from oracle import augment as oaug, chi0 as ochi0, coulomb, dyson, projection
from paper_2005_07834_gb300 import synth
from tests.gpu_util import public_psi, max_rel, rel_fro
from tests.oracle_problem import OracleProblem
from tests.test_oracle_augment import radial_set

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def case():
    wl = synth.single_site_260()
    s = wl.sites[0]
    pr = OracleProblem(wl)
    radii = np.linalg.norm(s.pts[::s.nang], axis=1)
    ae, ps = radial_set(radii, 2, 2, 2.2, seed=4)
    psi_aug = oaug.augment(public_psi(pr), s.pts, s.wts, s.nrad, s.nang, ae, ps, 2.2)
    return wl, pr, np.array(ae), np.array(ps), psi_aug


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
def test_augmented_orbitals_match_oracle(lrs, case, precision, tol):
    wl, pr, ae, ps, psi_aug = case
    scr = lrs.Screening(0, precision)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.project()
    before = scr.get_site_orbitals(0)
    scr.augment(0, ae, ps, 2.2)
    got = scr.get_site_orbitals(0)
    err = rel_fro(got, psi_aug)
    print(f"{precision}: augmented orbitals vs oracle {err:.2e} (max {max_rel(got, psi_aug):.2e}); change by "
          f"augmentation {rel_fro(psi_aug, public_psi(pr)):.2e}")
    assert err < tol and max_rel(got, psi_aug) < tol
    assert rel_fro(got, before) > 1e-3
    scr.close()


def test_screening_from_augmented_orbitals(lrs, case):
    wl, pr, ae, ps, psi_aug = case
    s = wl.sites[0]
    o = wl.orbitals
    po, pu, eo, eu, wo, wu = projection.split_occupied(psi_aug.reshape(s.npts, o.nk, o.nbands), o.energies,
                                                         o.nocc, o.kweights)
    chi_ref = ochi0.chi0_pairs(po, pu, eo, eu, wo, wu, pr.mu, pr.t, pr.W)
    w_ref = dyson.screened_interaction(coulomb.coulomb_multipole(s.pts, s.lmax), chi_ref, s.wts)
    scr = lrs.Screening(0, "fp64")
    scr.load(o)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=pr.mu, zeta=pr.zeta)
    scr.project()
    scr.augment(0, ae, ps, 2.2)
    scr.build_chi0()
    scr.solve_w()
    assert rel_fro(scr.get_chi0(0), chi_ref) < 1e-10
    assert rel_fro(scr.get_w(0), w_ref) < 1e-10
    scr.close()


def test_augment_errors(lrs, case):
    wl, pr, ae, ps, _ = case
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    with pytest.raises(lrs.LrsError) as e:
        scr.augment(0, ae, ps, 2.2)                     # not projected yet
    assert e.value.code == lrs.LRS_ERR_STATE
    scr.project()
    with pytest.raises(lrs.LrsError) as e:
        scr.augment(0, ae, ps, -1.0)
    assert e.value.code == lrs.LRS_ERR_ARG
    big = np.zeros((5,) + ae.shape[1:])                   # l_aug = 4 > L = 3
    with pytest.raises(lrs.LrsError) as e:
        scr.augment(0, big, big, 2.2)
    assert e.value.code == lrs.LRS_ERR_ARG
    with pytest.raises(lrs.LrsError) as e:
        scr.augment(0, ae, np.zeros_like(ps), 2.2)      # zero pseudo waves: singular overlap
    assert e.value.code == lrs.LRS_ERR_NUMERIC
    scr.close()
