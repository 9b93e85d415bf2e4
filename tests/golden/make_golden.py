"""Write oracle reference values for the 42-point tiny workload.

Calls only the oracle and the seeded input generator.  Run from the repository
root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import chi0, coulomb, dyson, projection, quadrature  # noqa: E402
from paper_2005_07834_gb300 import synth  # noqa: E402


def compute():
    w = synth.tiny(nk=8, nocc=3, nunocc=5)
    o, s = w.orbitals, w.sites[0]
    psi = projection.project_direct(o.cell, o.kpts, o.gvec, o.coeff, s.center, s.pts)
    po, pu, eo, eu, wo, wu = projection.split_occupied(psi, o.energies, o.nocc, o.kweights)
    mu = quadrature.chemical_potential_midgap(o.energies, o.nocc)
    zeta = quadrature.zeta_rule(o.energies, mu)
    t, W = quadrature.frequency_grid(12, zeta)
    c = chi0.chi0_pairs(po, pu, eo, eu, wo, wu, mu, t, W)
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    wm = dyson.screened_interaction(v, c, s.wts)
    idx = [(0, 0), (3, 17), (20, 41), (41, 41)]
    return {
        "workload": "tiny: a=6 bohr, |G|<=2, 2x2x2 k, 3 occ + 5 unocc, 3 GL x 14 Lebedev, 12 freq, seed 0",
        "mu": mu, "zeta": zeta,
        "chi0_trace": float(np.trace(c)), "chi0_fro": float(np.linalg.norm(c)),
        "w_trace": float(np.trace(wm)), "w_fro": float(np.linalg.norm(wm)),
        "chi0_entries": {f"{i},{j}": float(c[i, j]) for i, j in idx},
        "w_entries": {f"{i},{j}": float(wm[i, j]) for i, j in idx},
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_oracle.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", out)
