"""torch.autograd.Function for W(band energies, site-grid orbitals) through the C-ABI.

Forward: lrs_set_energies_dev, lrs_set_site_orbitals_dev, lrs_build_chi0,
lrs_solve_w, lrs_get_w_dev.  Backward: lrs_backward_dev (the adjoint kernels
recompute the Green's functions frequency by frequency).  Inputs, W and the
gradients stay in device memory; the library's stream and torch's current
stream are ordered by events, so neither direction synchronises the host.
The frequency quadrature (mu, t_i, W_i) is held fixed, as set on the
Screening context.  Complex gradients follow the PyTorch convention
dL/dRe + i dL/dIm.
"""
import torch


def _library_stream(scr):
    """The context's stream as a torch stream (the legacy default stream when none was given)."""
    if scr.stream:
        return torch.cuda.ExternalStream(scr.stream)
    return torch.cuda.default_stream()


class ScreenedInteraction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, energies, psi, screening, site):
        scr = screening
        lib = _library_stream(scr)
        cur = torch.cuda.current_stream()
        e_dev = energies.detach().to("cuda", torch.float64).contiguous()
        p_dev = psi.detach().to("cuda", torch.complex128).contiguous()
        lib.wait_stream(cur)                 # inputs written on torch's stream
        scr.set_energies_dev(e_dev.data_ptr())
        scr.set_site_orbitals_dev(site, p_dev.data_ptr())
        scr.build_chi0([site])
        scr.solve_w([site])
        n = scr.npts[site]
        w = torch.empty((n, n), dtype=torch.float64, device="cuda")
        scr.get_w_dev(site, w.data_ptr())
        cur.wait_stream(lib)                 # W is read on torch's stream
        for t in (e_dev, p_dev, w):
            t.record_stream(lib)
        ctx.scr, ctx.site = scr, site
        ctx.meta = (energies.shape, energies.device, psi.shape, psi.device)
        return w

    @staticmethod
    def backward(ctx, grad_w):
        eshape, edev, pshape, pdev = ctx.meta
        scr = ctx.scr
        lib = _library_stream(scr)
        cur = torch.cuda.current_stream()
        g = grad_w.detach().to("cuda", torch.float64).contiguous()
        ge = torch.empty(eshape, dtype=torch.float64, device="cuda")
        gp = torch.empty(pshape, dtype=torch.complex128, device="cuda")
        lib.wait_stream(cur)
        scr.backward_dev(ctx.site, g.data_ptr(), 0, ge.data_ptr(), gp.data_ptr())
        cur.wait_stream(lib)
        for t in (g, ge, gp):
            t.record_stream(lib)
        return ge.to(edev), gp.to(pdev), None, None


def screened_interaction(energies, psi, screening, site=0):
    """W of `site` as a differentiable function of energies [nk, nb] and psi [npts, nk*nb]."""
    return ScreenedInteraction.apply(energies, psi, screening, site)
