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
"""
import numpy as np
import pytest

from paper_2005_07834_gb300 import synth
from tests.gpu_util import rel_fro

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
