"""Adjoint kernels vs the oracle's pair-form gradient and central finite differences (FP64).

Loss L = q^T W q on the 260-point site, q ~ N(0,1) (seed 2).  Gradients of
all 256 band energies and of the site-grid orbitals; mu and the quadrature
are held fixed.  Tolerances: 1e-9 relative vs the oracle gradient, 1e-6
relative (vector norm) vs central differences with h = 1e-6 Ha.  The
tensor-core adjoint of a bf16x3 context is gated at the mixed-path 1e-5.
"""
import numpy as np
import pytest

from oracle import grad as ograd
from paper_2005_07834_gb300 import synth
from tests.gpu_util import Reference, public_psi, max_rel, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


@pytest.fixture(scope="module")
def case():
    wl = synth.single_site_260()
    ref = Reference(wl)
    q = synth.loss_weights(wl.sites[0].npts, seed=2)
    return wl, ref, q


def oracle_grads(ref, gamma_w=None, gamma_chi0=None):
    pr = ref.pr
    gam = np.zeros_like(ref.w)
    if gamma_w is not None:
        gam += ograd.gamma_chi0(ref.w, pr.site.wts, gamma_w)
    if gamma_chi0 is not None:
        gam += gamma_chi0
    geo, geu, gpo, gpu = ograd.grad_pairs(*pr.args(), pr.t, pr.W, gam)
    o = pr.orbitals
    ge = np.zeros((o.nk, o.nbands))
    gp = np.zeros((pr.site.npts, o.nk, o.nbands), complex)
    io = iu = 0
    for k in range(o.nk):
        n = int(o.nocc[k])
        ge[k, :n] = geo[io:io + n]; ge[k, n:] = geu[iu:iu + o.nbands - n]
        gp[:, k, :n] = gpo[:, io:io + n]; gp[:, k, n:] = gpu[:, iu:iu + o.nbands - n]
        io += n; iu += o.nbands - n
    return ge, gp.reshape(pr.site.npts, -1)


def make_screening(lrs, wl, ref):
    scr = lrs.Screening(0, "fp64")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    scr.set_site_orbitals(0, public_psi(ref.pr))
    return scr


def test_backward_matches_oracle_gradient(lrs, case):
    wl, ref, q = case
    scr = make_screening(lrs, wl, ref)
    scr.build_chi0()
    scr.solve_w()
    ge, gp = scr.backward(0, grad_w=np.outer(q, q))
    oe, op = oracle_grads(ref, gamma_w=np.outer(q, q))
    assert rel_fro(ge, oe) < 1e-9
    assert rel_fro(gp, op) < 1e-9
    scr.close()


def test_backward_general_gradients(lrs, case):
    """A non-symmetric dL/dW together with a direct dL/dchi0."""
    wl, ref, q = case
    rng = np.random.default_rng(7)
    n = wl.sites[0].npts
    gw = rng.standard_normal((n, n))
    gc = rng.standard_normal((n, n)) * 1e-3
    scr = make_screening(lrs, wl, ref)
    scr.build_chi0()
    scr.solve_w()
    ge, gp = scr.backward(0, grad_w=gw, grad_chi0=gc)
    oe, op = oracle_grads(ref, gamma_w=gw, gamma_chi0=gc)
    assert rel_fro(ge, oe) < 1e-9
    assert rel_fro(gp, op) < 1e-9
    ge2, gp2 = scr.backward(0, grad_chi0=gc)
    oe2, op2 = oracle_grads(ref, gamma_chi0=gc)
    assert rel_fro(ge2, oe2) < 1e-9 and rel_fro(gp2, op2) < 1e-9
    scr.close()


def test_backward_central_differences(lrs, case):
    wl, ref, q = case
    scr = make_screening(lrs, wl, ref)
    e0 = wl.orbitals.energies.copy()
    psi0 = public_psi(ref.pr).copy()

    def loss(e=e0, psi=psi0):
        scr.set_energies(e)
        scr.set_site_orbitals(0, psi)
        scr.build_chi0()
        scr.solve_w()
        return q @ scr.get_w(0) @ q

    loss()
    ge, gp = scr.backward(0, grad_w=np.outer(q, q))
    # Central differences carry a round-off error ~ eps_L |L| / h: at h = 1e-6 Ha
    # that floor is a few 1e-6 relative here, at h = 1e-4 it is far below 1e-6.
    for h, tol in ((1e-4, 1e-6), (1e-6, 3e-5)):
        fd = np.zeros_like(e0)
        for idx in np.ndindex(e0.shape):
            ep = e0.copy(); ep[idx] += h
            em = e0.copy(); em[idx] -= h
            fd[idx] = (loss(e=ep) - loss(e=em)) / (2 * h)
        err = rel_fro(ge, fd)
        print(f"energy gradients vs central differences, h = {h:g}: relative error {err:.2e}")
        assert err < tol, (h, err)
    # scissor shift of every unoccupied level: dL/dDelta = sum of unoccupied gradients
    h = 1e-5
    unocc = np.zeros_like(e0, bool)
    for k in range(e0.shape[0]):
        unocc[k, int(wl.orbitals.nocc[k]):] = True
    fd = (loss(e=e0 + h * unocc) - loss(e=e0 - h * unocc)) / (2 * h)
    assert abs(fd - ge[unocc].sum()) < 1e-7 * abs(ge[unocc]).sum()
    rng = np.random.default_rng(11)
    h = 1e-4
    picks = [(int(rng.integers(psi0.shape[0])), int(rng.integers(psi0.shape[1]))) for _ in range(64)]
    fd_re, fd_im, an_re, an_im = [], [], [], []
    for (p, c) in picks:
        for unit, fd_l, an_l, part in ((1.0, fd_re, an_re, np.real), (1j, fd_im, an_im, np.imag)):
            pp = psi0.copy(); pp[p, c] += h * unit
            pm = psi0.copy(); pm[p, c] -= h * unit
            fd_l.append((loss(psi=pp) - loss(psi=pm)) / (2 * h))
            an_l.append(part(gp[p, c]))
    assert rel_fro(np.array(an_re + an_im), np.array(fd_re + fd_im)) < 1e-6
    scr.close()


@pytest.mark.parametrize("own_stream", [False, True])
def test_autograd_function(lrs, case, own_stream):
    """Leaf tensors on the GPU: forward (device setters), loss and backward never leave device
    memory; the library runs on torch's current stream or on a stream of its own."""
    import torch
    from paper_2005_07834_gb300.autograd import screened_interaction

    wl, ref, q = case
    side = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
    scr = lrs.Screening(0, "fp64", side.cuda_stream)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    e = torch.tensor(wl.orbitals.energies, dtype=torch.float64, device="cuda", requires_grad=True)
    psi = torch.tensor(public_psi(ref.pr), dtype=torch.complex128, device="cuda", requires_grad=True)
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    w = screened_interaction(e, psi, scr, 0)
    loss = qt @ w @ qt
    loss.backward()
    assert e.grad.is_cuda and psi.grad.is_cuda
    assert rel_fro(w.detach().cpu().numpy(), ref.w) < 1e-10
    oe, op = oracle_grads(ref, gamma_w=np.outer(q, q))
    assert rel_fro(e.grad.cpu().numpy(), oe) < 1e-9
    assert rel_fro(psi.grad.cpu().numpy(), op) < 1e-9
    # a scissor shift through the device setter: the forward sees the new energies
    shifted = e.detach().clone()
    shifted[:, :] += torch.tensor(np.where(np.arange(wl.orbitals.nbands)[None, :] >= wl.orbitals.nocc[:, None],
                                           0.05, 0.0), device="cuda")
    w2 = screened_interaction(shifted, psi.detach(), scr, 0)
    torch.cuda.synchronize()
    assert rel_fro(w2.cpu().numpy(), ref.w) > 1e-6
    scr.close()


def test_device_setters_match_host_setters(lrs, case):
    """lrs_set_energies_dev / lrs_set_site_orbitals_dev give chi0 and W bit-identical to the host
    setters, and the quadrature rule reads the energies set on the device."""
    import torch
    wl, ref, q = case
    o = wl.orbitals
    e_new = o.energies + np.where(np.arange(o.nbands)[None, :] >= o.nocc[:, None], 0.03, -0.02)
    res = []
    for dev in (False, True):
        scr = lrs.Screening(0, "fp64", torch.cuda.current_stream().cuda_stream)
        scr.load(o)
        scr.set_sites(wl.sites)
        if dev:
            e_t = torch.tensor(e_new, dtype=torch.float64, device="cuda")
            p_t = torch.tensor(public_psi(ref.pr), dtype=torch.complex128, device="cuda")
            scr.set_energies_dev(e_t.data_ptr())
            scr.set_site_orbitals_dev(0, p_t.data_ptr())
        else:
            scr.set_energies(e_new)
            scr.set_site_orbitals(0, public_psi(ref.pr))
        mu, zeta = scr.set_frequency_quadrature(wl.nfreq)
        scr.build_chi0()
        scr.solve_w()
        res.append((mu, zeta, scr.get_chi0(0), scr.get_w(0)))
        scr.close()
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][3], res[1][3])
    with pytest.raises(lrs.LrsError):
        scr = lrs.Screening(0, "fp64")
        try:
            scr.set_energies_dev(0)
        finally:
            scr.close()


def test_mixed_adjoint_on_tensor_cores(lrs, case):
    """bf16x3 context: Green's functions recomputed and H products on tcgen05, gradients in FP64."""
    wl, ref, q = case
    scr = lrs.Screening(0, "bf16x3")
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    scr.set_site_orbitals(0, public_psi(ref.pr))
    scr.build_chi0()
    scr.solve_w()
    ge, gp = scr.backward(0, grad_w=np.outer(q, q))
    oe, op = oracle_grads(ref, gamma_w=np.outer(q, q))
    err_e, err_p = rel_fro(ge, oe), rel_fro(gp, op)
    print(f"mixed adjoint vs oracle gradient: energies {err_e:.2e} (max {max_rel(ge, oe):.2e}), "
          f"orbitals {err_p:.2e} (max {max_rel(gp, op):.2e})")
    assert err_e < 1e-5 and err_p < 1e-5   # mixed-path tolerance (measured 1.4e-6, 1.9e-6)
    assert max_rel(ge, oe) < 1e-5 and max_rel(gp, op) < 1e-5
    scr.close()
