"""Pins of the FP64 oracle against closed forms, brute force and invariants (CPU only)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import chi0, coulomb, dyson, grad, projection, quadrature
from paper_2005_07834_gb300 import synth
from tests.oracle_problem import OracleProblem


@pytest.fixture(scope="module")
def tiny8():
    return OracleProblem(synth.tiny(nk=8, nocc=3, nunocc=5))


@pytest.fixture(scope="module")
def tiny1():
    return OracleProblem(synth.tiny(nk=1, nocc=2, nunocc=3, gmax=1.6))


# ---------------------------------------------------------------- quadrature

def test_kappa_exact_is_the_line_integral():
    # (1/2pi) int_R dt Re[1/((a+it)(b+it))]: 1/(b-a) across the gap, 0 on one side.
    for a, b in [(0.3, -0.2), (1.1, -2.5), (0.05, -0.4)]:
        f = lambda t: ((a * b - t * t) / ((a * a + t * t) * (b * b + t * t))) / (2 * np.pi)
        val, _ = integrate.quad(f, -np.inf, np.inf, epsabs=1e-13, epsrel=1e-12, limit=400)
        assert abs(val - quadrature.kappa_exact(a, b)) < 1e-10
    for a, b in [(0.3, 0.7), (-0.2, -1.5)]:
        f = lambda t: ((a * b - t * t) / ((a * a + t * t) * (b * b + t * t))) / (2 * np.pi)
        val, _ = integrate.quad(f, -np.inf, np.inf, epsabs=1e-13, limit=400)
        assert abs(val) < 1e-10


def test_kappa_quadrature_converges():
    o = synth.single_site_260().orbitals
    mu = quadrature.chemical_potential_midgap(o.energies, o.nocc)
    zeta = quadrature.zeta_rule(o.energies, mu)
    alpha = mu - o.energies[0, :8]
    beta = mu - o.energies[0, 8:]
    ex = quadrature.kappa_exact(alpha[:, None], beta[None, :])
    errs = {}
    for n in (4, 8, 12, 16, 24, 32, 64):
        t, W = quadrature.frequency_grid(n, zeta)
        k = quadrature.kappa_quadrature(alpha[:, None], beta[None, :], t, W)
        errs[n] = np.max(np.abs(k / ex - 1))
    assert errs[4] > errs[8] > errs[12] > errs[16] > errs[24]
    assert errs[16] < 1e-6          # "a 16-point grid was found to be sufficient"
    assert errs[32] < 1e-12 and errs[64] < 1e-12


def test_zeta_rule_and_midgap():
    e = np.array([[-1.0, -0.3, 0.2, 2.0]])
    mu = quadrature.chemical_potential_midgap(e, np.array([2]))
    assert mu == pytest.approx(-0.05)
    zeta = quadrature.zeta_rule(e, mu)
    d = np.abs(mu - e.ravel())
    assert np.min(d) < zeta < np.max(d)
    # metallic limit: the 0.5 eV floor keeps zeta finite
    e0 = np.array([[-1.0, 0.0, 0.0, 1.0]])
    assert quadrature.zeta_rule(e0, 0.0) > 0.1


def test_dkappa_matches_finite_difference():
    t, W = quadrature.frequency_grid(12, 0.7)
    a, b, h = 0.35, -0.8, 1e-4
    da, db = quadrature.dkappa_quadrature(a, b, t, W)
    k = lambda x, y: quadrature.kappa_quadrature(x, y, t, W)
    fa = (-k(a + 2 * h, b) + 8 * k(a + h, b) - 8 * k(a - h, b) + k(a - 2 * h, b)) / (12 * h)
    fb = (-k(a, b + 2 * h) + 8 * k(a, b + h) - 8 * k(a, b - h) + k(a, b - 2 * h)) / (12 * h)
    assert da == pytest.approx(fa, rel=1e-9) and db == pytest.approx(fb, rel=1e-9)


# ---------------------------------------------------------------- projection

def _fft_grid_orbitals(o, n):
    """psi on the uniform cell grid by inverse FFT of the coefficients (independent route)."""
    a = o.cell[0, 0]
    omega = a ** 3
    x = np.arange(n) * a / n
    grid = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    out = np.empty((n ** 3, o.nk, o.nbands), np.complex128)
    for k in range(o.nk):
        box = np.zeros((n, n, n, o.nbands), np.complex128)
        idx = np.mod(o.gvec, n)
        box[idx[:, 0], idx[:, 1], idx[:, 2], :] = o.coeff[k]
        u = np.fft.ifftn(box, axes=(0, 1, 2)) * n ** 3
        out[:, k, :] = np.exp(1j * grid @ o.kpts[k])[:, None] * u.reshape(-1, o.nbands)
    return grid, out / np.sqrt(omega)


def test_projection_matches_fft():
    w = synth.tiny(nk=8, nocc=3, nunocc=5)
    o = w.orbitals
    grid, ref = _fft_grid_orbitals(o, 12)
    psi = projection.project_direct(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), grid)
    assert np.max(np.abs(psi - ref)) < 1e-12 * np.max(np.abs(ref))


def test_projection_orthonormal_over_cell():
    w = synth.tiny(nk=8, nocc=3, nunocc=5)
    o = w.orbitals
    n = 12
    a = o.cell[0, 0]
    x = np.arange(n) * a / n
    grid = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    psi = projection.project_direct(o.cell, o.kpts, o.gvec, o.coeff, np.zeros(3), grid)
    for k in range(o.nk):
        s = psi[:, k, :].conj().T @ psi[:, k, :] * a ** 3 / n ** 3
        assert np.max(np.abs(s - np.eye(o.nbands))) < 1e-12


# ---------------------------------------------------------------- chi0

def test_chi0_brute_force_line_integral(tiny1):
    """Integrate Eq. (chi1) with the full g of Eq. (eq-green) numerically, element by element."""
    pr = tiny1
    o = pr.orbitals
    psi = pr.psi[:, 0, :]                  # one k-point, weight 1
    e = o.energies[0]
    ref = chi0.chi0_pairs(*pr.args(), exact=True)
    for p, q in [(0, 0), (1, 7), (5, 11), (10, 3)]:
        def integrand(t):
            d = 1.0 / (pr.mu + 1j * t - e)
            g_pq = np.sum(np.conj(psi[p]) * psi[q] * d)
            g_qp = np.sum(np.conj(psi[q]) * psi[p] * d)
            return 2.0 * (g_pq * g_qp).real / (2 * np.pi)
        val, _ = integrate.quad(integrand, -np.inf, np.inf, epsabs=1e-14, epsrel=1e-12, limit=500)
        assert abs(val - ref[p, q]) < 1e-9 * np.max(np.abs(ref))


def test_two_level_closed_form_from_green_route():
    rng = np.random.default_rng(5)
    psi_v = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    psi_c = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    ev, ec, mu = -0.4, 0.9, 0.2
    zeta = quadrature.zeta_rule(np.array([ev, ec]), mu)
    t, W = quadrature.frequency_grid(64, zeta)
    got = chi0.chi0_green(psi_v[:, None], psi_c[:, None], np.array([ev]), np.array([ec]),
                          np.ones(1), np.ones(1), mu, t, W)
    a = np.conj(psi_v) * psi_c
    closed = 4.0 * np.real(np.outer(a, np.conj(a))) / (ev - ec)
    assert np.max(np.abs(got - closed)) < 1e-12 * np.max(np.abs(closed))


def test_pair_and_green_routes_agree(tiny8):
    pr = tiny8
    a = chi0.chi0_pairs(*pr.args(), pr.t, pr.W)
    b = chi0.chi0_green(*pr.args(), pr.t, pr.W)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
    rows = [0, 5, 17]
    c = chi0.chi0_pairs(*pr.args(), pr.t, pr.W, rows=rows)
    assert np.max(np.abs(c - a[rows])) < 1e-14 * np.max(np.abs(a))


def test_green_route_rows_match_the_pair_sum(tiny8):
    """The row-restricted Green's-function route (used on the large site grids, where the full
    matrix is too costly for every check) against the independent pair sum, rows in any order,
    repeated and at both ends."""
    pr = tiny8
    npts = pr.po.shape[0]
    rows = [npts - 1, 0, 7, 7, 3]
    a = chi0.chi0_pairs(*pr.args(), pr.t, pr.W, rows=rows)
    b = chi0.chi0_green(*pr.args(), pr.t, pr.W, rows=rows)
    assert b.shape == (len(rows), npts)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
    full = chi0.chi0_green(*pr.args(), pr.t, pr.W)
    assert np.max(np.abs(full[rows] - b)) < 1e-14 * np.max(np.abs(full))


def test_chi0_invariants(tiny8):
    pr = tiny8
    for kw in (dict(exact=True), dict(t=pr.t, W=pr.W)):
        c = chi0.chi0_pairs(*pr.args(), **kw)
        assert np.max(np.abs(c - c.T)) < 1e-14 * np.max(np.abs(c))
        assert np.linalg.eigvalsh(c).max() < 1e-12 * np.max(np.abs(c))
        assert np.all(np.diag(c) < 0)


def test_chi0_quadrature_converges_to_exact(tiny8):
    pr = tiny8
    ex = chi0.chi0_pairs(*pr.args(), exact=True)
    prev = np.inf
    for n in (8, 12, 16, 32):
        t, W = quadrature.frequency_grid(n, pr.zeta)
        err = np.linalg.norm(chi0.chi0_pairs(*pr.args(), t, W) - ex) / np.linalg.norm(ex)
        assert err < prev
        prev = err
    assert prev < 1e-12


# ---------------------------------------------------------------- Coulomb

def test_coulomb_multipole_converges_to_inverse_distance():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((40, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = np.where(np.arange(40) % 2 == 0, 1.0, 2.5)
    pts = u * r[:, None]
    v = coulomb.coulomb_multipole(pts, 60)
    d = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=-1)
    mask = np.not_equal.outer(r, r)
    assert np.max(np.abs(v[mask] - 1.0 / d[mask]) * d[mask]) < 1e-13


def test_coulomb_weighted_psd_and_ball_potential():
    s = synth.single_site_260().sites[0]
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    qh = np.sqrt(s.wts)
    ev = np.linalg.eigvalsh(qh[:, None] * v * qh[None, :])
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(s.wts) == pytest.approx(4 * np.pi * 4.0 ** 3 / 3, rel=1e-12)
    # potential of a uniform unit ball of radius R at radius r: 2 pi (R^2 - r^2/3)
    pot = v @ s.wts
    r = np.linalg.norm(s.pts, axis=1)
    exact = 2 * np.pi * (4.0 ** 2 - r ** 2 / 3)
    assert np.max(np.abs(pot - exact) / exact) < 5e-3


# ---------------------------------------------------------------- Dyson

def test_dyson_without_polarizability_is_bare():
    s = synth.single_site_260().sites[0]
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    w = dyson.screened_interaction(v, np.zeros_like(v), s.wts)
    assert np.max(np.abs(w - v)) == 0.0


def test_dyson_rank_one_sherman_morrison():
    s = synth.tiny().sites[0]
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    u = np.random.default_rng(4).standard_normal(s.npts)
    alpha = 0.37
    w = dyson.screened_interaction(v, -alpha * np.outer(u, u), s.wts)
    y = v @ (s.wts * u)
    ref = v - alpha * np.outer(y, y) / (1.0 + alpha * (u * s.wts) @ y)
    assert np.max(np.abs(w - ref)) < 1e-13 * np.max(np.abs(v))


def test_dyson_invariants(tiny8):
    pr = tiny8
    s = pr.site
    c = chi0.chi0_pairs(*pr.args(), pr.t, pr.W)
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    a = dyson.dyson_matrix(v, c, s.wts)
    ev = np.linalg.eigvals(a)
    assert np.max(np.abs(ev.imag)) < 1e-10 and ev.real.min() > 1 - 1e-10
    w = dyson.screened_interaction(v, c, s.wts)
    assert np.max(np.abs(w - w.T)) < 1e-12 * np.max(np.abs(w))
    qh = np.sqrt(s.wts)
    wt = qh[:, None] * w * qh[None, :]
    vt = qh[:, None] * v * qh[None, :]
    assert np.linalg.eigvalsh(0.5 * (wt + wt.T)).min() > -1e-10
    assert np.linalg.eigvalsh(0.5 * ((vt - wt) + (vt - wt).T)).min() > -1e-10


# ---------------------------------------------------------------- gradients

def _loss(pr, q, v, eo, eu, po, pu, exact=False):
    if exact:
        c = chi0.chi0_pairs(po, pu, eo, eu, pr.wo, pr.wu, pr.mu, exact=True)
    else:
        c = chi0.chi0_pairs(po, pu, eo, eu, pr.wo, pr.wu, pr.mu, pr.t, pr.W)
    return q @ dyson.screened_interaction(v, c, pr.site.wts) @ q


@pytest.mark.parametrize("exact", [False, True])
def test_gradients_match_finite_differences(tiny8, exact):
    pr = tiny8
    s = pr.site
    v = coulomb.coulomb_multipole(s.pts, s.lmax)
    q = synth.loss_weights(s.npts)
    if exact:
        c = chi0.chi0_pairs(*pr.args(), exact=True)
    else:
        c = chi0.chi0_pairs(*pr.args(), pr.t, pr.W)
    wm = dyson.screened_interaction(v, c, s.wts)
    gam = grad.gamma_chi0(wm, s.wts, np.outer(q, q))
    geo, geu, gpo, gpu = grad.grad_pairs(*pr.args(), pr.t, pr.W, gam, exact=exact)
    h = 1e-3

    def fd(f):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    L = lambda eo=pr.eo, eu=pr.eu, po=pr.po, pu=pr.pu: _loss(pr, q, v, eo, eu, po, pu, exact)
    scale = max(np.abs(geo).max(), np.abs(geu).max())
    for i in (0, 7, 23):
        e = np.eye(len(pr.eo))[i]
        assert abs(fd(lambda x: L(eo=pr.eo + x * e)) - geo[i]) < 1e-7 * scale
    for i in (0, 11, 39):
        e = np.eye(len(pr.eu))[i]
        assert abs(fd(lambda x: L(eu=pr.eu + x * e)) - geu[i]) < 1e-7 * scale
    # scissor shift of every unoccupied level
    assert abs(fd(lambda x: L(eu=pr.eu + x)) - geu.sum()) < 1e-7 * scale
    pscale = max(np.abs(gpo).max(), np.abs(gpu).max())
    for (p, b) in [(0, 0), (9, 13), (40, 23)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            m = np.zeros(pr.po.shape, complex); m[p, b] = unit
            assert abs(fd(lambda x: L(po=pr.po + x * m)) - part(gpo[p, b])) < 1e-7 * pscale
            m = np.zeros(pr.pu.shape, complex); m[p, b] = unit
            assert abs(fd(lambda x: L(pu=pr.pu + x * m)) - part(gpu[p, b])) < 1e-7 * pscale
