"""lrs_solve_w_static: W without any device allocation by the library.

This entry point serves callers that cannot allocate device memory (for
example a plugin whose host program's caching allocator already holds the
GPU, or a latency-critical loop that cannot take the synchronisation of
cudaMalloc).  It keeps its scratch in a statically reserved device array, so
the test checks that two consecutive calls of different sizes, and a repeat of
the first, reproduce lrs_solve_w within the FP64 tolerance of the other GPU
tests, and that an oversized request is refused before any work.  The test
allocates its own input and output tensors; the entry point allocates none.
The file name sorts last so that a run stopping at the first failure has
already run every other test.

A second test fills the array to its limit: a 512-point grid of scattered
points (not a radial x angular product, so lrs_solve_w also takes the full-grid
LU), checked against lrs_solve_w and against the FP64 oracle's dense LU on the
same chi0, and the driver's free device memory must not change across calls
once a first call has loaded the kernels.
"""
import numpy as np
import pytest

from oracle import coulomb as ocoul, dyson as odys
from paper_2005_07834_gb300 import synth
from tests.gpu_util import max_rel, rel_fro

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_static_scratch_dyson_matches_lrs_solve_w():
    import torch
    from paper_2005_07834_gb300 import lrs

    wl = synth.single_site_260()
    wl.sites.append(synth.site_grid(np.array([2.0, 3.0, 4.5]), 5, 14, 3.0))   # 70 points
    stream = torch.cuda.current_stream()
    scr = lrs.Screening(0, "fp64", stream.cuda_stream)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    for site in (0, 1, 0):
        s = wl.sites[site]
        n = s.npts
        chi0 = torch.empty((n, n), dtype=torch.float64, device="cuda")
        scr.get_chi0_dev(site, chi0.data_ptr())
        pts = torch.tensor(s.pts, dtype=torch.float64, device="cuda")
        wts = torch.tensor(s.wts, dtype=torch.float64, device="cuda")
        w = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        rc = lrs.lrs_solve_w_static(n, s.lmax, pts.data_ptr(), wts.data_ptr(), chi0.data_ptr(),
                                    w.data_ptr(), stream.cuda_stream)
        assert rc == lrs.LRS_OK, lrs.lrs_last_error()
        torch.cuda.synchronize()
        assert rel_fro(w.cpu().numpy(), scr.get_w(site)) < TOL
    scr.close()


def test_static_scratch_rejects_oversized_grids():
    import torch
    from paper_2005_07834_gb300 import lrs

    n = lrs.lib.lrs_solve_w_static  # the symbol is exported
    assert n is not None
    big = 513
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    rc = lrs.lrs_solve_w_static(big, 3, p, p, p, p, None)
    assert rc == lrs.LRS_ERR_ARG
    assert b"512" in lrs.lrs_last_error()


def test_static_scratch_at_its_limit_allocates_nothing():
    import torch
    from paper_2005_07834_gb300 import lrs

    n = lrs.LRS_STATIC_MAX_NPTS
    rng = np.random.default_rng(7)
    radius = 3.0
    d = rng.normal(size=(n, 3))
    pts = d / np.linalg.norm(d, axis=1)[:, None] * (radius * rng.uniform(0.05, 1.0, n) ** (1 / 3))[:, None]
    wts = np.full(n, 4.0 / 3.0 * np.pi * radius ** 3 / n)
    wl = synth.single_site_260()
    wl.sites = [synth.SiteGrid(np.array([4.0, 5.0, 6.0]), pts, wts, 6, 0, 0)]
    stream = torch.cuda.current_stream()
    scr = lrs.Screening(0, "fp64", stream.cuda_stream)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq)
    assert scr.site_grid_shape(0)[0] is False
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    w_ctx = scr.get_w(0)
    chi0_host = scr.get_chi0(0)
    chi0 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    scr.get_chi0_dev(0, chi0.data_ptr())
    pts_d = torch.tensor(pts, dtype=torch.float64, device="cuda")
    wts_d = torch.tensor(wts, dtype=torch.float64, device="cuda")
    outs = [torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()

    def call(out):
        rc = lrs.lrs_solve_w_static(n, 6, pts_d.data_ptr(), wts_d.data_ptr(), chi0.data_ptr(), out.data_ptr(),
                                    stream.cuda_stream)
        assert rc == lrs.LRS_OK, lrs.lrs_last_error()

    call(outs[0])                        # loads the kernels and the array on first use
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call(outs[1])
    call(outs[2])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    w_oracle = odys.screened_interaction(ocoul.coulomb_multipole(pts, 6), chi0_host, wts)
    for out in outs:
        w = out.cpu().numpy()
        assert rel_fro(w, w_ctx) < TOL and max_rel(w, w_ctx) < TOL
        assert rel_fro(w, w_oracle) < TOL and max_rel(w, w_oracle) < TOL
    assert np.array_equal(outs[1].cpu().numpy(), outs[2].cpu().numpy())
    scr.close()
