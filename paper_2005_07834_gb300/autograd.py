"""torch.autograd.Function for W(band energies, site-grid orbitals) through the C-ABI.

Forward: lrs_set_energies, lrs_set_site_orbitals, lrs_build_chi0, lrs_solve_w.
Backward: lrs_backward_dev (the adjoint kernels recompute the Green's
functions frequency by frequency).  The frequency quadrature (mu, t_i, W_i)
is held fixed, as set on the Screening context.  Complex gradients follow the
PyTorch convention dL/dRe + i dL/dIm.
"""
import torch


class ScreenedInteraction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, energies, psi, screening, site):
        scr = screening
        scr.set_energies(energies.detach().to("cpu", torch.float64).numpy())
        scr.set_site_orbitals(site, psi.detach().to("cpu", torch.complex128).numpy())
        scr.build_chi0([site])
        scr.solve_w([site])
        n = scr.npts[site]
        w = torch.empty((n, n), dtype=torch.float64, device="cuda")
        scr.get_w_dev(site, w.data_ptr())
        ctx.scr, ctx.site = scr, site
        ctx.meta = (energies.shape, energies.device, psi.shape, psi.device)
        return w

    @staticmethod
    def backward(ctx, grad_w):
        eshape, edev, pshape, pdev = ctx.meta
        g = grad_w.detach().to("cuda", torch.float64).contiguous()
        ge = torch.empty(eshape, dtype=torch.float64, device="cuda")
        gp = torch.empty(pshape, dtype=torch.complex128, device="cuda")
        ctx.scr.backward_dev(ctx.site, g.data_ptr(), 0, ge.data_ptr(), gp.data_ptr())
        return ge.to(edev), gp.to(pdev), None, None


def screened_interaction(energies, psi, screening, site=0):
    """W of `site` as a differentiable function of energies [nk, nb] and psi [npts, nk*nb]."""
    return ScreenedInteraction.apply(energies, psi, screening, site)
