"""Shared helpers of the GPU parity tests: oracle references and error norms."""
import numpy as np

from oracle import chi0 as ochi0, coulomb as ocoul, dyson as odys
from tests.oracle_problem import OracleProblem


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def public_psi(pr):
    """Oracle orbitals in the library's public column order [npts][nk*nbands]."""
    npts, nk, nb = pr.psi.shape
    return pr.psi.reshape(npts, nk * nb)


class Reference:
    def __init__(self, workload, site=0, nfreq=None):
        self.pr = OracleProblem(workload, site, nfreq)
        pr = self.pr
        self.chi0 = ochi0.chi0_pairs(*pr.args(), pr.t, pr.W)
        self.v = ocoul.coulomb_multipole(pr.site.pts, pr.site.lmax)
        self.w = odys.screened_interaction(self.v, self.chi0, pr.site.wts)


def max_rel(a, b):
    """Element-wise error scaled by the reference's largest element: max |a - b| / max |b|."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def row_rel(a, b):
    """Largest relative Frobenius error over the rows of a [rows, n] block."""
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))
