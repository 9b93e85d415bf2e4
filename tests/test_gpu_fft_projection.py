"""Method-2 projection (Sec. VI.B: FFT to the cell grid, 3rd-degree Lagrange
interpolation, Bloch phase) on the GPU vs the oracle of the same method.

Bars: float64 contexts 1e-10 relative (Frobenius over all points and
columns); fp32 transforms of the mixed contexts 1e-5 (fp32 rounding through
three transform passes and a 64-point gather).  The oracle's own distance to
the exact projection (the method's interpolation error) is printed, not gated.
"""
import dataclasses

import numpy as np
import pytest

from oracle import projection as oproj
from paper_2005_07834_gb300 import synth
from tests.gpu_util import max_rel, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


def oracle_psi(o, site, grid):
    psi = oproj.project_fft_lagrange(o.cell, o.kpts, o.gvec, o.coeff, site.center, site.pts, grid)
    return psi.reshape(site.npts, -1)


def run(lrs, precision, o, sites, grid):
    scr = lrs.Screening(0, precision)
    scr.load(o)
    scr.set_sites(sites)
    scr.set_fft_grid(*grid)
    scr.project(mode=lrs.LRS_PROJ_FFT_LAGRANGE3)
    return scr


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
@pytest.mark.parametrize("grid", [(16, 16, 16), (18, 24, 12)])
def test_fft_projection_matches_oracle(lrs, precision, tol, grid):
    wl = synth.single_site_260()
    o, s = wl.orbitals, wl.sites[0]
    scr = run(lrs, precision, o, [s], grid)
    got = scr.get_site_orbitals(0)
    ref = oracle_psi(o, s, grid)
    err = rel_fro(got, ref)
    exact = oproj.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts).reshape(s.npts, -1)
    print(f"{precision} grid {grid}: vs oracle {err:.2e} (max {max_rel(got, ref):.2e}); method error vs exact "
          f"{rel_fro(ref, exact):.2e}")
    assert err < tol and max_rel(got, ref) < tol
    scr.close()


def test_sheared_cell_and_several_sites(lrs):
    """A non-orthogonal cell (fractional coordinates through the inverse cell
    matrix), k-points off the mesh, three sites of different sizes placed
    across the cell edge; one transform per k serves all sites."""
    base = synth.tiny(nk=8, nocc=3, nunocc=5, gmax=3.5)
    o = base.orbitals
    cell = np.array([[6.0, 0.0, 0.0], [1.5, 5.5, 0.0], [0.7, -0.9, 6.3]])
    recip = 2.0 * np.pi * np.linalg.inv(cell).T
    frac = np.random.default_rng(11).uniform(-0.5, 0.5, (o.nk, 3))
    o = dataclasses.replace(o, cell=cell, kpts=frac @ recip)
    sites = [synth.site_grid(c, nr, na, 2.5) for c, nr, na in
             [(np.array([0.1, 0.2, 0.3]), 3, 14), (cell[0] + cell[1] - 0.2, 4, 26), (0.5 * cell.sum(0), 2, 50)]]
    grid = (18, 16, 24)
    scr = run(lrs, "fp64", o, sites, grid)
    for i, s in enumerate(sites):
        err = rel_fro(scr.get_site_orbitals(i), oracle_psi(o, s, grid))
        assert err < 1e-10, (i, err)
    scr.close()


def test_full_size_sampled(lrs):
    """3520-point site, 8709 G, 640 bands per k on the 48^3 grid (bf16x3
    context, as the large workloads run): 64 seeded points x 24 seeded bands
    per k against the oracle evaluated on those only."""
    wl = synth.single_site_3520()
    o, s = wl.orbitals, wl.sites[0]
    grid = (48, 48, 48)
    scr = run(lrs, "bf16x3", o, [s], grid)
    got = scr.get_site_orbitals(0).reshape(s.npts, o.nk, o.nbands)
    rng = np.random.default_rng(12)
    pts = np.sort(rng.choice(s.npts, 64, replace=False))
    bands = np.sort(rng.choice(o.nbands, 24, replace=False))
    sub = dataclasses.replace(o, coeff=o.coeff[:, :, bands])
    ref = oproj.project_fft_lagrange(sub.cell, sub.kpts, sub.gvec, sub.coeff, s.center, s.pts[pts], grid)
    err = rel_fro(got[pts][:, :, bands], ref)
    print(f"3520-point site, 48^3 grid, sampled: {err:.2e} (max {max_rel(got[pts][:, :, bands], ref):.2e})")
    assert err < 1e-5 and max_rel(got[pts][:, :, bands], ref) < 1e-5
    scr.close()


def test_grid_selection_and_errors(lrs):
    wl = synth.single_site_260()            # |n_i| <= 4: 9 points needed per direction
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    assert scr.get_fft_grid() == (18, 18, 18)   # smallest 2^a 3^b >= 2 x 9
    with pytest.raises(lrs.LrsError) as e:
        scr.set_fft_grid(20, 16, 16)             # 20 = 2^2 5
    assert e.value.code == lrs.LRS_ERR_ARG
    scr.set_fft_grid(8, 16, 16)                  # 8 < 9: aliasing
    with pytest.raises(lrs.LrsError) as e:
        scr.project(mode=lrs.LRS_PROJ_FFT_LAGRANGE3)
    assert e.value.code == lrs.LRS_ERR_ARG
    with pytest.raises(lrs.LrsError) as e:
        scr.project(mode=7)
    assert e.value.code == lrs.LRS_ERR_UNSUPPORTED
    scr.close()


def test_graph_replay_with_fft_projection(lrs):
    """A recorded build whose projection is method 2 replays to the eager result bit for bit."""
    wl = synth.tiny(nk=8, nocc=3, nunocc=5, gmax=3.5)
    import torch
    stream = torch.cuda.Stream()
    scr = lrs.Screening(0, "bf16x3", stream.cuda_stream)
    scr.load(wl.orbitals)
    sites = [synth.site_grid(np.array([1.0, 2.0, 3.0]), 3, 14, 2.0), synth.site_grid(np.array([3.0, 3.0, 3.0]), 4, 26, 2.0)]
    scr.set_sites(sites)
    scr.set_frequency_quadrature(12)
    scr.set_fft_grid(16, 16, 16)
    scr.project(mode=lrs.LRS_PROJ_FFT_LAGRANGE3)
    scr.build_chi0()
    scr.solve_w()
    eager = [scr.get_w(i) for i in range(2)]
    scr.set_option(lrs.LRS_OPT_GRAPH_PROJECTION, lrs.LRS_PROJ_FFT_LAGRANGE3)
    scr.graph_capture()
    scr.graph_launch()
    scr.synchronize()
    for i in range(2):
        assert np.array_equal(scr.get_w(i), eager[i])
        assert rel_fro(scr.get_site_orbitals(i), oracle_psi(wl.orbitals, sites[i], (16, 16, 16))) < 1e-5
    scr.close()
