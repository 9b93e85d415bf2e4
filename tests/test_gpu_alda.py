"""ALDA vertex (Eq. chi-alda, kxc_alda) on the GPU vs the oracle: site density,
exchange-only kernel, the ALDA screened interaction in both Dyson bases, a
caller-supplied kernel, the induced core-hole response with the vertex, and
the return to RPA.  Bars: 1e-10 (FP64 contexts), 1e-5 (bf16x3)."""
import numpy as np
import pytest

from oracle import alda as oalda, induced as oind
from paper_2005_07834_gb300 import synth
from tests.gpu_util import Reference, max_rel, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def case():
    wl = synth.single_site_260()
    ref = Reference(wl)
    n = oalda.density(ref.pr.po, ref.pr.wo)
    return wl, ref, n


def built(lrs, precision, wl, ref, basis=None):
    scr = lrs.Screening(0, precision)
    if basis is not None:
        scr.set_option(lrs.LRS_OPT_DYSON_BASIS, basis)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    scr.project()
    scr.build_chi0()
    return scr


@pytest.mark.parametrize("basis", ["lm", "full"])
def test_exchange_alda_matches_oracle(lrs, case, basis):
    wl, ref, n = case
    s = wl.sites[0]
    scr = built(lrs, "fp64", wl, ref, lrs.LRS_DYSON_LM if basis == "lm" else lrs.LRS_DYSON_FULL)
    assert rel_fro(scr.get_density(0), n) < 1e-12
    scr.set_fxc(0, lrs.LRS_FXC_ALDA_X)
    f = oalda.fx_exchange(n)
    assert rel_fro(scr.get_fxc(0), f) < 1e-12
    scr.solve_w()
    w_ref = oalda.screened_interaction_alda(ref.chi0, ref.v, f, s.wts)
    err = rel_fro(scr.get_w(0), w_ref)
    shift = rel_fro(w_ref, ref.w)
    print(f"{basis}: ALDA W~ vs oracle {err:.2e} (W~ differs from the RPA W by {shift:.2e})")
    assert err < 1e-10
    assert rel_fro(scr.get_chi0(0), ref.chi0) < 1e-10          # chi0 itself is unchanged
    scr.set_fxc(0, lrs.LRS_FXC_NONE)
    scr.solve_w()
    assert rel_fro(scr.get_w(0), ref.w) < 1e-10
    scr.close()


def test_user_kernel_and_mixed_context(lrs, case):
    wl, ref, _ = case
    s = wl.sites[0]
    f = -np.random.default_rng(21).uniform(0.5, 3.0, s.npts)
    scr = built(lrs, "bf16x3", wl, ref)
    scr.set_fxc(0, lrs.LRS_FXC_USER, f)
    assert np.array_equal(scr.get_fxc(0), f)
    scr.solve_w()
    w_ref = oalda.screened_interaction_alda(ref.chi0, ref.v, f, s.wts)
    w = scr.get_w(0)
    err = rel_fro(w, w_ref)
    print(f"bf16x3, caller kernel: W~ vs oracle {err:.2e} (max {max_rel(w, w_ref):.2e}, "
          f"W~ - v {rel_fro(w - ref.v, w_ref - ref.v):.2e})")
    assert err < 1e-5 and max_rel(w, w_ref) < 1e-5 and rel_fro(w - ref.v, w_ref - ref.v) < 1e-5
    scr.close()


def test_induced_response_with_the_vertex(lrs, case):
    wl, ref, n = case
    s = wl.sites[0]
    f = oalda.fx_exchange(n)
    d = f * s.wts
    chi_eff = np.linalg.solve(np.eye(s.npts) - ref.chi0 * d[None, :], ref.chi0)
    scr = built(lrs, "fp64", wl, ref)
    scr.set_fxc(0, lrs.LRS_FXC_ALDA_X)
    rho, vind, _ = scr.induced_potential(0, -1.0, 1.5, s.lmax)
    _, orho, ovind = oind.induced_potential(chi_eff, s.pts, s.wts, s.nrad, s.nang, -1.0, 1.5, s.lmax)
    _, _, ovind_rpa = oind.induced_potential(ref.chi0, s.pts, s.wts, s.nrad, s.nang, -1.0, 1.5, s.lmax)
    print(f"ALDA induced potential vs oracle {rel_fro(vind, ovind):.2e}; "
          f"|v_ind,00| ALDA / RPA at the first shell {abs(ovind[0, 0] / ovind_rpa[0, 0]):.3f}")
    assert rel_fro(rho, orho) < 1e-10 and rel_fro(vind, ovind) < 1e-10
    with pytest.raises(lrs.LrsError) as e:
        scr.backward(0, grad_w=np.eye(s.npts))
    assert e.value.code == lrs.LRS_ERR_UNSUPPORTED
    scr.close()
