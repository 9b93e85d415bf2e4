"""Several uneven sites in one persistent tensor-core launch, replayed from a CUDA graph.

Sites of 130, 260, 350 and 440 points (radial shells x Lebedev 26/50/110)
share the orbitals of the 260-point workload; chi0 and W of every site are
compared with the FP64 oracle (Green's-function route, itself pinned to the
pair sum) at the mixed-precision tolerance 1e-5, relative Frobenius and element-wise
(max |d| / max |ref|), W - v included.
"""
import numpy as np
import pytest

from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys
from paper_2005_07834_gb300 import synth
from tests.gpu_util import max_rel, rel_fro
from tests.oracle_problem import OracleProblem

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def workload():
    wl = synth.single_site_260()
    wl.sites = [synth.site_grid(np.array([1.0, 2.0, 3.0]), 5, 26, 3.0), wl.sites[0],
                synth.site_grid(np.array([7.0, 4.0, 2.0]), 7, 50, 4.0),
                synth.site_grid(np.array([3.0, 8.0, 6.0]), 4, 110, 3.5)]
    refs = []
    for i in range(len(wl.sites)):
        pr = OracleProblem(wl, site=i)
        chi = ochi0.chi0_green(*pr.args(), pr.t, pr.W)
        v = ocoul.coulomb_multipole(pr.site.pts, pr.site.lmax)
        refs.append((chi, odys.screened_interaction(v, chi, pr.site.wts), v))
    return wl, refs


def make(lrs, wl, stream=None):
    scr = lrs.Screening(0, "bf16x3", stream)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    return scr


def test_batched_sites_one_launch(lrs, workload):
    wl, refs = workload
    scr = make(lrs, wl)
    scr.project()
    scr.build_chi0()            # all sites: one persistent launch
    scr.solve_w()
    scr.synchronize()
    for i, (chi, w, v) in enumerate(refs):
        c, g = scr.get_chi0(i), scr.get_w(i)
        e = (rel_fro(c, chi), max_rel(c, chi), rel_fro(g, w), max_rel(g, w), rel_fro(g - v, w - v),
             max_rel(g - v, w - v))
        print(f"site {i} ({wl.sites[i].npts} points): chi0 {e[0]:.2e} max {e[1]:.2e}, W {e[2]:.2e} "
              f"max {e[3]:.2e}, W-v {e[4]:.2e} max {e[5]:.2e}")
        assert max(e) < TOL, (i, e)
    scr.close()


def test_graph_replay_matches_eager(lrs, workload):
    import torch
    wl, refs = workload
    stream = torch.cuda.Stream()
    scr = make(lrs, wl, stream.cuda_stream)
    scr.graph_capture()
    scr.synchronize()
    eager = [(scr.get_chi0(i), scr.get_w(i)) for i in range(len(wl.sites))]
    for _ in range(3):
        scr.graph_launch()
    scr.synchronize()
    for i, (chi, w) in enumerate(eager):
        assert np.array_equal(scr.get_chi0(i), chi)
        assert np.array_equal(scr.get_w(i), w)
        assert rel_fro(w, refs[i][1]) < TOL and max_rel(w, refs[i][1]) < TOL
    scr.close()


def test_autotune_keeps_accuracy(lrs, workload):
    wl, refs = workload
    scr = make(lrs, wl)
    scr.project()
    best = scr.autotune()
    assert best["tile_n"] in (64, 128) and best["segment"] in (2, 4) and best["ms_chi0"] > 0
    scr.build_chi0()
    scr.solve_w()
    for i, (chi, w, v) in enumerate(refs):
        assert rel_fro(scr.get_chi0(i), chi) < TOL and max_rel(scr.get_chi0(i), chi) < TOL
    for tn in (64, 128):
        scr.set_option(lrs.LRS_OPT_CHI0_TILE_N, tn)
        scr.build_chi0()
        assert rel_fro(scr.get_chi0(1), refs[1][0]) < TOL
    scr.close()


@pytest.mark.parametrize("lanes", [2, 3, 8])
def test_concurrent_dyson_lanes_match_one_lane(lrs, workload, lanes):
    """The sites of one solve spread over concurrent lanes (own streams and
    workspace) give W bit for bit equal to one lane, also when replayed from a
    recorded graph; more lanes than sites is allowed."""
    import torch
    wl, refs = workload
    scr = make(lrs, wl)
    scr.project()
    scr.build_chi0()
    scr.set_option(lrs.LRS_OPT_DYSON_LANES, 1)
    scr.solve_w()
    one = [scr.get_w(i) for i in range(len(wl.sites))]
    scr.set_option(lrs.LRS_OPT_DYSON_LANES, lanes)
    scr.solve_w()
    for i in range(len(wl.sites)):
        assert np.array_equal(scr.get_w(i), one[i]), i
    scr.close()
    stream = torch.cuda.Stream()
    scr = make(lrs, wl, stream.cuda_stream)
    scr.set_option(lrs.LRS_OPT_DYSON_LANES, lanes)
    scr.graph_capture()
    scr.graph_launch()
    scr.synchronize()
    for i in range(len(wl.sites)):
        assert np.array_equal(scr.get_w(i), one[i]), i
        assert rel_fro(scr.get_w(i), refs[i][1]) < TOL and max_rel(scr.get_w(i), refs[i][1]) < TOL
    with pytest.raises(lrs.LrsError) as e:
        scr.set_option(lrs.LRS_OPT_DYSON_LANES, 9)
    assert e.value.code == lrs.LRS_ERR_ARG
    scr.close()


def test_four_lanes_on_large_sites_match_one_lane(lrs):
    """Four sites of the 64-site workload (800 to 9118 points, r up to 6768) solved on four
    concurrent lanes, whose side streams then compete for the GPU: W bit for bit equal to one
    lane.  (Before the gather of a panel's other rows waited for the exchange write-back of the
    block two steps back, this case read stale values under contention: W - v off by 6e-5.)"""
    from paper_2005_07834_gb300 import synth as _synth
    wl = _synth.batched_64_sites()
    sites = [wl.sites[i] for i in (4, 5, 17, 59)]
    scr = lrs.Screening(0, "bf16x3")
    scr.load(wl.orbitals)
    scr.set_sites(sites)
    scr.set_frequency_quadrature(wl.nfreq)
    scr.project()
    scr.build_chi0()
    scr.set_option(lrs.LRS_OPT_DYSON_LANES, 1)
    scr.solve_w()
    one = [scr.get_w(i) for i in range(4)]
    for lanes in (4, 3, 2):
        scr.set_option(lrs.LRS_OPT_DYSON_LANES, lanes)
        for _ in range(2):
            scr.solve_w()
            for i in range(4):
                assert np.array_equal(scr.get_w(i), one[i]), (lanes, i)
    scr.close()
