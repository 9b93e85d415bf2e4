"""Helpers that turn synthetic inputs into oracle arguments (tests only)."""
import numpy as np

from oracle import projection, quadrature


class OracleProblem:
    def __init__(self, workload, site=0, nfreq=None):
        o = workload.orbitals
        s = workload.sites[site]
        self.orbitals, self.site = o, s
        self.psi = projection.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts)
        (self.po, self.pu, self.eo, self.eu, self.wo, self.wu) = projection.split_occupied(
            self.psi, o.energies, o.nocc, o.kweights)
        self.mu = quadrature.chemical_potential_midgap(o.energies, o.nocc)
        self.zeta = quadrature.zeta_rule(o.energies, self.mu)
        self.nfreq = workload.nfreq if nfreq is None else nfreq
        self.t, self.W = quadrature.frequency_grid(self.nfreq, self.zeta)

    def args(self):
        return (self.po, self.pu, self.eo, self.eu, self.wo, self.wu, self.mu)
