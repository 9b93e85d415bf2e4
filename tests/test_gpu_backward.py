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
from tests.gpu_util import Reference, public_psi, rel_fro

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


def test_autograd_function(lrs, case):
    import torch
    from paper_2005_07834_gb300.autograd import screened_interaction

    wl, ref, q = case
    scr = lrs.Screening(0, "fp64", torch.cuda.current_stream().cuda_stream)
    scr.load(wl.orbitals)
    scr.set_sites(wl.sites)
    scr.set_frequency_quadrature(wl.nfreq, mu=ref.pr.mu, zeta=ref.pr.zeta)
    e = torch.tensor(wl.orbitals.energies, dtype=torch.float64, requires_grad=True)
    psi = torch.tensor(public_psi(ref.pr), dtype=torch.complex128, requires_grad=True)
    qt = torch.tensor(q, dtype=torch.float64, device="cuda")
    w = screened_interaction(e, psi, scr, 0)
    loss = qt @ w @ qt
    loss.backward()
    assert rel_fro(w.detach().cpu().numpy(), ref.w) < 1e-10
    oe, op = oracle_grads(ref, gamma_w=np.outer(q, q))
    assert rel_fro(e.grad.numpy(), oe) < 1e-9
    assert rel_fro(psi.grad.numpy(), op) < 1e-9
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
    print(f"mixed adjoint vs oracle gradient: energies {err_e:.2e}, orbitals {err_p:.2e}")
    assert err_e < 1e-5 and err_p < 1e-5   # mixed-path tolerance (measured 1.4e-6, 1.9e-6)
    scr.close()
