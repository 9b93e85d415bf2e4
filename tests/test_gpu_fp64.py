"""FP64 CUDA path vs the FP64 oracle through the C-ABI (tolerance 1e-10 relative Frobenius)."""
import numpy as np
import pytest

from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys
from paper_2005_07834_gb300 import synth
from tests.gpu_util import max_rel, Reference, public_psi, rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def cfg_260():
    return Reference(synth.single_site_260())


def run_fp64(lrs, workload, nfreq):
    scr = lrs.Screening(0, "fp64")
    scr.load(workload.orbitals)
    scr.set_sites(workload.sites)
    mu, zeta = scr.set_frequency_quadrature(nfreq)
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    return scr, mu, zeta


def test_single_site_260_forward(lrs, cfg_260):
    ref = cfg_260
    scr, mu, zeta = run_fp64(lrs, synth.single_site_260(), 12)
    pr = ref.pr
    assert mu == pytest.approx(pr.mu, abs=1e-15) and zeta == pytest.approx(pr.zeta, rel=1e-14)
    t, W = scr.get_frequency_quadrature()
    assert np.max(np.abs(t / pr.t - 1)) < 1e-13 and np.max(np.abs(W / pr.W - 1)) < 1e-13
    psi = scr.get_site_orbitals(0)
    assert rel_fro(psi, public_psi(pr)) < 1e-12
    assert rel_fro(scr.get_v(0), ref.v) < 1e-13
    chi = scr.get_chi0(0)
    assert rel_fro(chi, ref.chi0) < TOL
    assert np.max(np.abs(chi - ref.chi0)) < TOL * np.max(np.abs(ref.chi0))
    assert np.array_equal(chi, chi.T)
    w = scr.get_w(0)
    assert rel_fro(w, ref.w) < TOL
    assert rel_fro(w - ref.v, ref.w - ref.v) < 1e-8
    st = scr.stats()
    assert st["kernel_launches"] > 0 and st["status_word"] == 0
    scr.close()


def test_ragged_multisite(lrs):
    """Two sites whose sizes are not multiples of the tiles, odd band counts."""
    wl = synth.tiny(nk=8, nocc=3, nunocc=5)
    extra = synth.site_grid(np.array([1.0, 2.0, 0.5]), 5, 14, 2.5)      # 70 points
    wl.sites.append(extra)
    scr, mu, zeta = run_fp64(lrs, wl, 12)
    for i in range(2):
        ref = Reference(wl, site=i)
        assert rel_fro(scr.get_chi0(i), ref.chi0) < TOL
        assert rel_fro(scr.get_w(i), ref.w) < TOL
    scr.close()


def test_set_site_orbitals_bypasses_projection(lrs, cfg_260):
    ref = cfg_260
    wl = synth.single_site_260()
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(12)
    scr.set_site_orbitals(0, public_psi(ref.pr))
    scr.build_chi0([0])
    scr.solve_w([0])
    assert rel_fro(scr.get_chi0(0), ref.chi0) < TOL
    assert rel_fro(scr.get_w(0), ref.w) < TOL
    scr.close()


def test_zeta_override_and_more_frequencies(lrs):
    wl = synth.tiny(nk=1, nocc=2, nunocc=6)
    ref_pr = Reference(wl, nfreq=24).pr
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    mu, zeta = scr.set_frequency_quadrature(24, mu=ref_pr.mu, zeta=0.3)
    assert zeta == 0.3
    scr.project()
    scr.build_chi0()
    from oracle import quadrature as oq
    t, W = oq.frequency_grid(24, 0.3)
    chi = ochi0.chi0_pairs(*ref_pr.args(), t, W)
    assert rel_fro(scr.get_chi0(0), chi) < TOL
    scr.close()


def test_state_and_argument_errors(lrs):
    wl = synth.tiny()
    scr = lrs.Screening(0, "fp64")
    with pytest.raises(lrs.LrsError) as e:
        scr.set_frequency_quadrature(12)
    assert e.value.code == lrs.LRS_ERR_STATE
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(8)
    with pytest.raises(lrs.LrsError) as e:
        scr.build_chi0()
    assert e.value.code == lrs.LRS_ERR_STATE
    with pytest.raises(lrs.LrsError) as e:
        scr.solve_w()
    assert e.value.code == lrs.LRS_ERR_STATE
    with pytest.raises(lrs.LrsError) as e:
        scr.set_frequency_quadrature(8, mu=5.0)      # mu above every level
    assert e.value.code == lrs.LRS_ERR_ARG
    with pytest.raises(lrs.LrsError) as e:
        scr.build_chi0([7])
    assert e.value.code == lrs.LRS_ERR_ARG
    scr.close()


@pytest.mark.parametrize("basis", ["full", "lm-lu", "lm-lu-tc", "lm-spd", "lm-spd-tc"])
def test_dyson_bases_match_oracle(lrs, cfg_260, basis):
    ref = cfg_260
    wl = synth.single_site_260()
    scr = lrs.Screening(0, "fp64")
    scr.set_option(lrs.LRS_OPT_DYSON_BASIS, lrs.LRS_DYSON_FULL if basis == "full" else lrs.LRS_DYSON_LM)
    if basis != "full":
        scr.set_option(lrs.LRS_OPT_DYSON_SOLVER,
                       lrs.LRS_SOLVER_LU if basis.startswith("lm-lu") else lrs.LRS_SOLVER_SPD)
    if basis.endswith("-tc"):     # float64-accurate basis changes and updates from bf16 slices on the tensor cores
        scr.set_option(lrs.LRS_OPT_DYSON_UPDATE, lrs.LRS_UPDATE_TC)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(12)
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    w = scr.get_w(0)
    assert rel_fro(w, ref.w) < TOL
    assert rel_fro(w - ref.v, ref.w - ref.v) < 1e-8
    scr.close()


def test_non_product_grid_uses_full_basis(lrs):
    wl = synth.tiny(nk=8, nocc=3, nunocc=5)
    s = wl.sites[0]
    s.pts = s.pts.copy()
    s.pts[5] *= 1.01                       # breaks the radial x angular product structure
    ref = Reference(wl)
    scr, mu, zeta = run_fp64(lrs, wl, 12)  # automatic basis: full grid
    assert rel_fro(scr.get_w(0), ref.w) < TOL
    scr.set_option(lrs.LRS_OPT_DYSON_BASIS, lrs.LRS_DYSON_LM)
    with pytest.raises(lrs.LrsError) as e:
        scr.solve_w()
    assert e.value.code == lrs.LRS_ERR_ARG
    scr.close()


def test_spd_and_lu_dyson_agree_on_a_large_site(lrs):
    """Symmetric (Gauss-Jordan) and LU lm-basis solvers on a 48-shell x 110-point
    site (r = 48 * 81 = 3888, several pivot blocks and a ragged last one) from the
    same chi0: the two float64 solutions of one linear system agree to 1e-11."""
    wl = synth.single_site_260()
    wl.sites = [synth.site_grid(wl.sites[0].center, 48, 110, 4.0)]
    scr = lrs.Screening(0, "bf16x3")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(8)
    scr.project()
    scr.build_chi0()
    ws = []
    for solver in (lrs.LRS_SOLVER_LU, lrs.LRS_SOLVER_SPD):
        scr.set_option(lrs.LRS_OPT_DYSON_SOLVER, solver)
        scr.solve_w()
        ws.append(scr.get_w(0))
    v = scr.get_v(0)
    err = rel_fro(ws[1] - v, ws[0] - v)
    print(f"SPD vs LU lm-basis W - v: {err:.2e}")
    assert err < 1e-11
    scr.close()


def test_tensor_core_update_is_float64_accurate(lrs):
    """SPD inverse of the 48 x 110 site (r = 3888) with the basis changes and the
    trailing updates on the tensor cores vs float64 FMAs, from the same chi0
    (FP64 context): W - v agrees to 1e-12, i.e. the sliced products carry
    float64 accuracy."""
    wl = synth.single_site_260()
    wl.sites = [synth.site_grid(wl.sites[0].center, 48, 110, 4.0)]
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(8)
    scr.project()
    scr.build_chi0()
    ws = []
    for mode in (lrs.LRS_UPDATE_FP64, lrs.LRS_UPDATE_TC):
        scr.set_option(lrs.LRS_OPT_DYSON_UPDATE, mode)
        scr.solve_w()
        ws.append(scr.get_w(0))
    v = scr.get_v(0)
    err = rel_fro(ws[1] - v, ws[0] - v)
    print(f"tensor-core vs float64 trailing updates, W - v: {err:.2e}")
    assert err < 1e-12
    scr.close()


def test_tensor_core_basis_change_over_several_k_segments(lrs):
    """12 shells x 194 directions (L = 11: 144 harmonics, r = 1728): the basis
    changes contract over K = 194 and 144, more than one exactly accumulated
    segment of 128, and 144 output columns span three tiles with a ragged one.
    Tensor-core vs float64-FMA arithmetic from the same chi0: W - v agrees to 1e-12."""
    wl = synth.single_site_260()
    wl.sites = [synth.site_grid(wl.sites[0].center, 12, 194, 3.0)]
    scr = lrs.Screening(0, "bf16x3")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(8)
    scr.project()
    scr.build_chi0()
    ws = []
    for solver in (lrs.LRS_SOLVER_SPD, lrs.LRS_SOLVER_LU):
        scr.set_option(lrs.LRS_OPT_DYSON_SOLVER, solver)
        for mode in (lrs.LRS_UPDATE_FP64, lrs.LRS_UPDATE_TC):
            scr.set_option(lrs.LRS_OPT_DYSON_UPDATE, mode)
            scr.solve_w()
            ws.append(scr.get_w(0))
    v = scr.get_v(0)
    for name, (a, b) in (("SPD", (ws[0], ws[1])), ("LU", (ws[2], ws[3]))):
        err = rel_fro(b - v, a - v)
        print(f"{name}: tensor-core vs float64 arithmetic, W - v: {err:.2e}")
        assert err < 1e-12
    scr.close()


@pytest.mark.parametrize("nrad,nang", [(70, 14), (130, 6)])
def test_tensor_core_radial_products_over_several_tiles(lrs, nrad, nang):
    """The four radial-block products around the SPD inverse (M = I - F^T X F, Z = F M^-1 F^T)
    as per-lm GEMMs on the tensor cores: 70 shells x 14 directions (r = 630; 70 output columns
    span two tiles, K = 70 three chunks with a ragged one) and 130 shells x 6 directions (r = 520;
    K = 130 two exactly accumulated segments, so the identity of M is added once).  Tensor-core vs
    float64-FMA arithmetic from the same chi0: W - v agrees to 1e-12 (Frobenius), and element by
    element the tensor-core route is within twice the float64 route's own distance from the dense
    float64 LU of the same Dyson equation."""
    wl = synth.single_site_260()
    wl.sites = [synth.site_grid(wl.sites[0].center, nrad, nang, 4.0)]
    scr = lrs.Screening(0, "bf16x3")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(8)
    scr.project()
    scr.build_chi0()
    scr.set_option(lrs.LRS_OPT_DYSON_SOLVER, lrs.LRS_SOLVER_SPD)
    ws = []
    for mode in (lrs.LRS_UPDATE_FP64, lrs.LRS_UPDATE_TC):
        scr.set_option(lrs.LRS_OPT_DYSON_UPDATE, mode)
        scr.solve_w()
        ws.append(scr.get_w(0))
    v = scr.get_v(0)
    err = rel_fro(ws[1] - v, ws[0] - v)
    # element-wise, both routes against the dense float64 LU of the full-grid Dyson equation on the
    # same chi0: M = I - F^T X F has condition number up to |C| |X|, which scales rounding in
    # single elements of either route alike
    ref = odys.screened_interaction(v, scr.get_chi0(0), wl.sites[0].wts)
    e64, etc = max_rel(ws[0] - v, ref - v), max_rel(ws[1] - v, ref - v)
    print(f"{nrad} x {nang}: tensor-core vs float64 radial products, W - v: {err:.2e}; max element against "
          f"the dense LU: float64 route {e64:.2e}, tensor-core route {etc:.2e}")
    assert err < 1e-12
    assert etc < 2.0 * e64 + 1e-13
    scr.close()


def test_128_wide_pivot_blocks_match_32_wide(lrs):
    """The SPD inverse exchanging 128-wide pivot blocks (each inverted by 32-wide steps, then
    D = C P and the rank-128 trailing update on the float64-accurate tensor-core GEMM) against the
    32-wide exchange, from the same chi0 on the 48 x 110 site (r = 3888: 30 full blocks and a
    ragged one of 48) and on a 7 x 110 site (r = 567: four full blocks and one of 55): W - v agrees to
    1e-12; the blocked solve rewrites the trailing matrix once per 128 pivots."""
    wl = synth.single_site_260()
    for nrad in (48, 7):
        wl.sites = [synth.site_grid(wl.sites[0].center, nrad, 110, 4.0)]
        scr = lrs.Screening(0, "bf16x3")
        scr.load(wl.orbitals)
        scr.set_sites(wl.sites)
        scr.set_frequency_quadrature(8)
        scr.project()
        scr.build_chi0()
        ws, launches = [], []
        for panel in (32, 128, 0):
            scr.set_option(lrs.LRS_OPT_DYSON_PANEL, panel)
            scr.solve_w()
            ws.append(scr.get_w(0))
            launches.append(scr.stats()["w_main_launches"])
        v = scr.get_v(0)
        r = nrad * 81
        err = rel_fro(ws[1] - v, ws[0] - v)
        print(f"r = {r}: 128- vs 32-wide pivot blocks, W - v: {err:.2e}; update launches {launches}")
        assert err < 1e-12
        assert np.array_equal(ws[0], ws[2])               # the default takes 32-wide blocks
        assert launches[1] == (r + 127) // 128 and launches[0] == (r + 31) // 32
        with pytest.raises(lrs.LrsError) as e:
            scr.set_option(lrs.LRS_OPT_DYSON_PANEL, 64)
        assert e.value.code == lrs.LRS_ERR_ARG
        scr.close()
