"""Two contexts driven from two host threads at once (the end-to-end pipeline of the benchmark),
and site buffers reused across lrs_set_sites calls with sites of other sizes: every W equals the
one a fresh context builds for the same site, bit for bit."""
import threading

import numpy as np
import pytest

from paper_2005_07834_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


def build(scr, wl, site):
    scr.set_sites([site])
    scr.set_frequency_quadrature(wl.nfreq)
    scr.project()
    scr.build_chi0()
    scr.solve_w()
    return scr.get_w(0)


def test_two_threads_and_reused_site_buffers(lrs):
    wl = synth.single_site_260()
    c = wl.sites[0].center
    sites = [wl.sites[0], synth.site_grid(c, 20, 26, 4.0), synth.site_grid(c, 6, 50, 3.0)]   # 260, 520, 300 points
    ref = []
    for s in sites:
        scr = lrs.Screening(0, "bf16x3")
        scr.load(wl.orbitals)
        ref.append(build(scr, wl, s))
        scr.close()
    order = [[0, 1, 2, 1, 0], [2, 0, 1, 2, 1]]
    out = [[], []]
    errors = []

    def drive(t):
        try:
            import torch
            torch.cuda.set_device(0)
            scr = lrs.Screening(0, "bf16x3")
            for i in order[t]:
                scr.load(wl.orbitals)
                out[t].append((i, build(scr, wl, sites[i])))
            scr.close()
        except Exception as ex:
            errors.append(ex)

    threads = [threading.Thread(target=drive, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t in range(2):
        assert [i for i, _ in out[t]] == order[t]
        for i, w in out[t]:
            assert np.array_equal(w, ref[i]), (t, i)


def test_queued_solves_match_waiting_ones(lrs):
    """lrs_solve_w_async queues the Dyson solves and returns; W read afterwards (stream order)
    equals lrs_solve_w's bit for bit, also with two contexts whose builds are queued one behind
    the other from one host thread (the end-to-end pipeline); lrs_synchronize reads the status."""
    wl = synth.single_site_260()
    c = wl.sites[0].center
    sites = [wl.sites[0], synth.site_grid(c, 20, 26, 4.0)]
    scr = lrs.Screening(0, "bf16x3")
    scr.load(wl.orbitals)
    ref = [build(scr, wl, s) for s in sites]
    scr.set_sites([sites[0]])
    scr.set_frequency_quadrature(wl.nfreq)
    scr.project()
    scr.build_chi0()
    scr.solve_w_async()
    assert np.array_equal(scr.get_w(0), ref[0])
    scr.synchronize()
    scr.close()
    ctxs = [lrs.Screening(0, "bf16x3") for _ in range(2)]
    order = [0, 1, 1, 0, 0, 1]

    def queue(c, i):
        c.load(wl.orbitals)
        c.set_sites([sites[i]])
        c.set_frequency_quadrature(wl.nfreq)
        c.project()
        c.build_chi0()
        c.solve_w_async()

    queue(ctxs[0], order[0])
    for k, i in enumerate(order):
        cur = ctxs[k % 2]
        if k + 1 < len(order):
            queue(ctxs[(k + 1) % 2], order[k + 1])
        cur.synchronize()
        assert np.array_equal(cur.get_w(0), ref[i]), k
    for c_ in ctxs:
        c_.close()
