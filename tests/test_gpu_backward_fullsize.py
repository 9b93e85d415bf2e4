"""Adjoint of L = q^T W q on the 3520-point site (K = 5120, 16 frequencies), through the C-ABI.

The tensor-core adjoint of a bf16x3 context (Green's functions recomputed per frequency, H psi
products on tcgen05, float64 frequency sums) is compared with the float64 adjoint of a plain FP64
context on the same inputs (both contexts take the same site orbitals and the same quadrature), at
the mixed-path tolerance 1e-5 (relative Frobenius and element-wise).  The float64 adjoint is tied
to the loss itself by central differences of eight band energies (two occupied and two unoccupied
of two k-points), h = 1e-4 Ha, each difference quotient from two float64 builds: 1e-6 relative
(the bar of the 260-point differentiation case at this step).
Measured values are printed (pytest -s).
"""
import numpy as np
import pytest

from paper_2005_07834_gb300 import synth
from tests.gpu_util import max_rel, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrs():
    from paper_2005_07834_gb300 import lrs as _lrs
    return _lrs


def test_mixed_adjoint_against_fp64_adjoint_and_differences(lrs):
    wl = synth.single_site_3520()
    o, s = wl.orbitals, wl.sites[0]
    q = synth.loss_weights(s.npts, seed=2)
    gw = np.outer(q, q)
    ref = lrs.Screening(0, "fp64")
    ref.load(o)
    ref.set_sites([s])
    mu, zeta = ref.set_frequency_quadrature(wl.nfreq)
    ref.project()
    psi = ref.get_site_orbitals(0)
    ref.build_chi0()
    ref.solve_w()
    ge64, gp64 = ref.backward(0, grad_w=gw)

    mix = lrs.Screening(0, "bf16x3")
    mix.load(o)
    mix.set_sites([s])
    mix.set_frequency_quadrature(wl.nfreq, mu=mu, zeta=zeta)
    mix.set_site_orbitals(0, psi)
    mix.build_chi0()
    mix.solve_w()
    gem, gpm = mix.backward(0, grad_w=gw)
    mix.close()
    e = {"energies_fro": rel_fro(gem, ge64), "energies_max": max_rel(gem, ge64),
         "orbitals_fro": rel_fro(gpm, gp64), "orbitals_max": max_rel(gpm, gp64)}
    print("mixed vs float64 adjoint, 3520-point site:", {k: f"{v:.2e}" for k, v in e.items()})
    for k, v in e.items():
        assert v < 1e-5, (k, v)

    # central differences of the float64 loss for eight energies (mu and the quadrature held)
    e0 = o.energies.copy()

    def loss(energies):
        ref.set_energies(energies)
        ref.build_chi0()
        ref.solve_w()
        return q @ ref.get_w(0) @ q

    h = 1e-4
    picks = []
    for k in (0, 5):
        n = int(o.nocc[k])
        picks += [(k, n - 1), (k, n - 7), (k, n), (k, n + 9)]
    an, fd = [], []
    for idx in picks:
        ep = e0.copy(); ep[idx] += h
        em = e0.copy(); em[idx] -= h
        fd.append((loss(ep) - loss(em)) / (2 * h))
        an.append(ge64[idx])
    an, fd = np.array(an), np.array(fd)
    err = rel_fro(an, fd)
    print(f"float64 adjoint vs central differences (8 energies, h = {h:g}): {err:.2e}; "
          f"max element {max_rel(an, fd):.2e}")
    assert err < 1e-6, err
    ref.close()
