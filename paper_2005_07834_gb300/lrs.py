"""ctypes binding of liblrs (include/lrs.h).

Two layers:
  * the raw entry points under their C names (``lrs_create``, ``lrs_build_chi0``
    ...), exported from the loaded library with argument types attached;
  * ``Screening``, a small owner of one context that marshals NumPy arrays and
    torch tensors to those entry points and raises ``LrsError`` on a non-zero
    status.
Every step of the computation runs inside the library.  If liblrs.so is
missing the import of this module fails: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LRS_LIBRARY", os.path.join(_HERE, "liblrs.so"))

LRS_OK, LRS_ERR_ARG, LRS_ERR_OOM, LRS_ERR_CUDA, LRS_ERR_STATE = 0, 1, 2, 3, 4
LRS_ERR_TIMEOUT, LRS_ERR_NUMERIC, LRS_ERR_UNSUPPORTED = 5, 6, 7
LRS_FP64, LRS_MIXED_BF16X3, LRS_MIXED_FP16X3 = 0, 1, 2
LRS_PROJ_EXACT, LRS_PROJ_FFT_LAGRANGE3 = 0, 1
LRS_FFT_MAX_N = 256
LRS_OPT_DYSON_BASIS, LRS_OPT_CHI0_SEGMENT, LRS_OPT_PROJ_SEGMENT, LRS_OPT_CHI0_TILE_N = 1, 2, 3, 4
LRS_DYSON_AUTO, LRS_DYSON_FULL, LRS_DYSON_LM = 0, 1, 2
LRS_OPT_WORKSPACE_GB, LRS_OPT_DYSON_SOLVER, LRS_OPT_GRAPH_PROJECTION = 5, 6, 7
LRS_SOLVER_AUTO, LRS_SOLVER_LU, LRS_SOLVER_SPD = 0, 1, 2
LRS_FXC_NONE, LRS_FXC_USER, LRS_FXC_ALDA_X = 0, 1, 2
LRS_OPT_REAL_ORBITALS, LRS_REAL_AUTO, LRS_REAL_OFF = 8, 0, 1
LRS_OPT_DYSON_UPDATE, LRS_UPDATE_AUTO, LRS_UPDATE_FP64, LRS_UPDATE_TC = 9, 0, 1, 2
LRS_OPT_DYSON_LANES = 10
LRS_OPT_DYSON_PANEL = 11
LRS_STATIC_MAX_NPTS = 512
PRECISIONS = {"fp64": LRS_FP64, "bf16x3": LRS_MIXED_BF16X3, "fp16x3": LRS_MIXED_FP16X3}


class lrs_stats_t(C.Structure):
    _fields_ = [("ms_project", C.c_double), ("ms_chi0", C.c_double), ("ms_w", C.c_double),
                ("ms_backward", C.c_double), ("ms_chi0_main", C.c_double), ("flop_chi0", C.c_double),
                ("flop_w", C.c_double), ("kernel_launches", C.c_int64), ("device_bytes", C.c_int64),
                ("device_bytes_peak", C.c_int64), ("status_word", C.c_int), ("flop_w_executed", C.c_double),
                ("ms_w_main", C.c_double), ("flop_w_main", C.c_double), ("w_main_launches", C.c_int64),
                ("w_main_elements", C.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"liblrs.so not found at {LIB_PATH}: run __graft_entry__.build() "
                      "(python -m paper_2005_07834_gb300.build)")
lib = C.CDLL(LIB_PATH)

_P = C.c_void_p
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)
_SIGS = {
    "lrs_last_error": (C.c_char_p, []),
    "lrs_version": (C.c_char_p, []),
    "lrs_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, _P]),
    "lrs_destroy": (C.c_int, [_P]),
    "lrs_set_stream": (C.c_int, [_P, _P]),
    "lrs_set_option": (C.c_int, [_P, C.c_int, C.c_int]),
    "lrs_load_orbitals": (C.c_int, [_P, _DP, C.c_int, _DP, _DP, C.c_int, _IP, C.c_int, _IP, _DP, _DP]),
    "lrs_set_sites": (C.c_int, [_P, C.c_int, _DP, _IP, _DP, _DP, _IP]),
    "lrs_set_energies": (C.c_int, [_P, _DP]),
    "lrs_set_frequency_quadrature": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, _DP, _DP]),
    "lrs_get_frequency_quadrature": (C.c_int, [_P, _DP, _DP]),
    "lrs_project": (C.c_int, [_P, C.c_int, _IP, C.c_int]),
    "lrs_set_fft_grid": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "lrs_induced_potential": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int, _DP, _DP, _DP]),
    "lrs_site_grid_shape": (C.c_int, [_P, C.c_int, _IP, _IP, _IP]),
    "lrs_set_fxc": (C.c_int, [_P, C.c_int, C.c_int, _DP]),
    "lrs_augment": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, _DP, _DP]),
    "lrs_orbitals_are_real": (C.c_int, [_P, _IP]),
    "lrs_get_density": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_get_fxc": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_get_fft_grid": (C.c_int, [_P, _IP]),
    "lrs_set_site_orbitals": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_get_site_orbitals": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_set_energies_dev": (C.c_int, [_P, _P]),
    "lrs_set_site_orbitals_dev": (C.c_int, [_P, C.c_int, _P]),
    "lrs_build_chi0": (C.c_int, [_P, C.c_int, _IP]),
    "lrs_solve_w": (C.c_int, [_P, C.c_int, _IP]),
    "lrs_solve_w_async": (C.c_int, [_P, C.c_int, _IP]),
    "lrs_get_chi0": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_get_w": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_get_v": (C.c_int, [_P, C.c_int, _DP]),
    "lrs_get_chi0_dev": (C.c_int, [_P, C.c_int, _P]),
    "lrs_get_w_dev": (C.c_int, [_P, C.c_int, _P]),
    "lrs_backward": (C.c_int, [_P, C.c_int, _DP, _DP, _DP, _DP]),
    "lrs_backward_dev": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "lrs_solve_w_static": (C.c_int, [C.c_int, C.c_int, _P, _P, _P, _P, _P]),
    "lrs_graph_capture": (C.c_int, [_P, C.c_int, _IP]),
    "lrs_graph_launch": (C.c_int, [_P]),
    "lrs_autotune": (C.c_int, [_P, C.c_int, _IP, _IP, _IP, _DP]),
    "lrs_synchronize": (C.c_int, [_P]),
    "lrs_stats": (C.c_int, [_P, C.POINTER(lrs_stats_t)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class LrsError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what} failed with status {code}: {lrs_last_error().decode()}")
        self.code = code


def _check(code, what):
    if code != LRS_OK:
        raise LrsError(code, what)


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_IP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128_view(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.view(np.float64)


class Screening:
    """One library context: orbitals, site grids, quadrature and results on one device."""

    def __init__(self, device=0, precision="fp64", stream=None):
        self.ctx = _P()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lrs_create(C.byref(self.ctx), int(device), prec, _P(stream or 0)), "lrs_create")
        self.precision = prec
        self.stream = int(stream or 0)
        self.npts = []
        self.nk = self.nb = 0

    # -- lifetime
    def close(self):
        if self.ctx:
            lrs_destroy(self.ctx)
            self.ctx = _P()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lrs_set_stream(self.ctx, _P(stream or 0)), "lrs_set_stream")
        self.stream = int(stream or 0)

    def set_option(self, option, value):
        _check(lrs_set_option(self.ctx, int(option), int(value)), "lrs_set_option")

    # -- inputs
    def load_orbitals(self, cell, kpts, kweights, gvec, coeff, energies, nocc):
        coeff, cview = _c128_view(coeff)
        nk, ng, nb = coeff.shape
        cell, kpts, kw, en = _f64(cell), _f64(kpts), _f64(kweights), _f64(energies)
        g = np.ascontiguousarray(gvec, dtype=np.int32)
        no = np.ascontiguousarray(nocc, dtype=np.int32)
        _check(lrs_load_orbitals(self.ctx, _dp(cell), nk, _dp(kpts), _dp(kw), ng, _ip(g), nb, _ip(no),
                                 _dp(cview), _dp(en)), "lrs_load_orbitals")
        self.nk, self.nb = nk, nb

    def load(self, orbitals):
        o = orbitals
        self.load_orbitals(o.cell, o.kpts, o.kweights, o.gvec, o.coeff, o.energies, o.nocc)

    def set_energies(self, energies):
        e = _f64(energies)
        assert e.size == self.nk * self.nb
        _check(lrs_set_energies(self.ctx, _dp(e)), "lrs_set_energies")

    def set_sites(self, sites):
        centers = _f64(np.stack([s.center for s in sites]))
        npts = np.array([s.npts for s in sites], np.int32)
        pts = _f64(np.concatenate([s.pts for s in sites]))
        wts = _f64(np.concatenate([s.wts for s in sites]))
        lmax = np.array([s.lmax for s in sites], np.int32)
        _check(lrs_set_sites(self.ctx, len(sites), _dp(centers), _ip(npts), _dp(pts), _dp(wts), _ip(lmax)),
               "lrs_set_sites")
        self.npts = [int(n) for n in npts]

    def set_frequency_quadrature(self, nf, mu=float("nan"), zeta=0.0):
        mo, zo = C.c_double(), C.c_double()
        _check(lrs_set_frequency_quadrature(self.ctx, int(nf), float(mu), float(zeta), C.byref(mo), C.byref(zo)),
               "lrs_set_frequency_quadrature")
        self.nf = int(nf)
        return mo.value, zo.value

    def get_frequency_quadrature(self):
        t = np.empty(self.nf)
        w = np.empty(self.nf)
        _check(lrs_get_frequency_quadrature(self.ctx, _dp(t), _dp(w)), "lrs_get_frequency_quadrature")
        return t, w

    # -- stages
    @staticmethod
    def _sites(sites):
        if sites is None:
            return 0, None, None
        arr = np.ascontiguousarray(np.atleast_1d(sites), dtype=np.int32)
        return len(arr), _ip(arr), arr

    def project(self, sites=None, mode=LRS_PROJ_EXACT):
        n, p, _keep = self._sites(sites)
        _check(lrs_project(self.ctx, n, p, mode), "lrs_project")

    def orbitals_are_real(self):
        v = C.c_int()
        _check(lrs_orbitals_are_real(self.ctx, C.byref(v)), "lrs_orbitals_are_real")
        return bool(v.value)

    def augment(self, site, phi_ae, phi_ps, r_aug):
        """phi_ae, phi_ps: [lmax_aug + 1][nnu][nrad] radial functions on the site's shells."""
        ae = _f64(np.asarray(phi_ae, np.float64))
        ps = _f64(np.asarray(phi_ps, np.float64))
        assert ae.shape == ps.shape and ae.ndim == 3
        _check(lrs_augment(self.ctx, int(site), ae.shape[0] - 1, ae.shape[1], float(r_aug), _dp(ae), _dp(ps)),
               "lrs_augment")

    def set_fxc(self, site, kind, fxc=None):
        if fxc is not None:
            fxc = _f64(np.asarray(fxc, np.float64).reshape(-1))
        _check(lrs_set_fxc(self.ctx, int(site), int(kind), _dp(fxc) if fxc is not None else None), "lrs_set_fxc")

    def get_density(self, site):
        out = np.empty(self.npts[site])
        _check(lrs_get_density(self.ctx, int(site), _dp(out)), "lrs_get_density")
        return out

    def get_fxc(self, site):
        out = np.empty(self.npts[site])
        _check(lrs_get_fxc(self.ctx, int(site), _dp(out)), "lrs_get_fxc")
        return out

    def site_grid_shape(self, site):
        """(is a product grid, shells, directions per shell)."""
        p, nr, na = C.c_int(), C.c_int(), C.c_int()
        _check(lrs_site_grid_shape(self.ctx, int(site), C.byref(p), C.byref(nr), C.byref(na)), "lrs_site_grid_shape")
        return bool(p.value), nr.value, na.value

    def induced_potential(self, site, q, shell_radius, lresp=0):
        """Returns (rho_lm [nrad, (lresp+1)^2], vind_lm [nrad, (lresp+1)^2], vind_grid [npts])."""
        _, nrad, _ = self.site_grid_shape(site)
        l2 = (lresp + 1) ** 2
        rho = np.zeros((nrad, l2))
        vind = np.zeros((nrad, l2))
        grid = np.zeros(self.npts[site])
        _check(lrs_induced_potential(self.ctx, int(site), float(q), float(shell_radius), int(lresp), _dp(rho),
                                     _dp(vind), _dp(grid)), "lrs_induced_potential")
        return rho, vind, grid

    def set_fft_grid(self, n1=0, n2=0, n3=0):
        _check(lrs_set_fft_grid(self.ctx, int(n1), int(n2), int(n3)), "lrs_set_fft_grid")

    def get_fft_grid(self):
        n = (C.c_int * 3)()
        _check(lrs_get_fft_grid(self.ctx, n), "lrs_get_fft_grid")
        return tuple(n)

    def set_site_orbitals(self, site, psi):
        psi, view = _c128_view(psi)
        assert psi.shape == (self.npts[site], self.nk * self.nb)
        _check(lrs_set_site_orbitals(self.ctx, int(site), _dp(view)), "lrs_set_site_orbitals")

    def set_energies_dev(self, energies_ptr):
        """Energies [nk][nb] float64 from device memory (stream-ordered on the context stream)."""
        _check(lrs_set_energies_dev(self.ctx, _P(energies_ptr)), "lrs_set_energies_dev")

    def set_site_orbitals_dev(self, site, psi_ptr):
        """Site orbitals [npts][nk*nb] complex128 from device memory (stream-ordered)."""
        _check(lrs_set_site_orbitals_dev(self.ctx, int(site), _P(psi_ptr)), "lrs_set_site_orbitals_dev")

    def get_site_orbitals(self, site):
        out = np.empty((self.npts[site], self.nk * self.nb), np.complex128)
        _check(lrs_get_site_orbitals(self.ctx, int(site), _dp(out.view(np.float64))), "lrs_get_site_orbitals")
        return out

    def build_chi0(self, sites=None):
        n, p, _keep = self._sites(sites)
        _check(lrs_build_chi0(self.ctx, n, p), "lrs_build_chi0")

    def solve_w(self, sites=None):
        n, p, _keep = self._sites(sites)
        _check(lrs_solve_w(self.ctx, n, p), "lrs_solve_w")

    def solve_w_async(self, sites=None):
        n, p, _keep = self._sites(sites)
        _check(lrs_solve_w_async(self.ctx, n, p), "lrs_solve_w_async")

    def _get(self, fn, site, name, out=None):
        n = self.npts[site]
        if out is None:
            out = np.empty((n, n))
        elif out.shape != (n, n) or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"{name}: out must be a C-contiguous float64 array of shape ({n}, {n})")
        _check(fn(self.ctx, int(site), _dp(out)), name)
        return out

    def get_chi0(self, site=0, out=None):
        return self._get(lrs_get_chi0, site, "lrs_get_chi0", out)

    def get_w(self, site=0, out=None):
        """W of a site into a new array, or into `out` (e.g. pinned host memory)."""
        return self._get(lrs_get_w, site, "lrs_get_w", out)

    def get_v(self, site=0):
        return self._get(lrs_get_v, site, "lrs_get_v")

    def get_chi0_dev(self, site, out_ptr):
        _check(lrs_get_chi0_dev(self.ctx, int(site), _P(out_ptr)), "lrs_get_chi0_dev")

    def get_w_dev(self, site, out_ptr):
        _check(lrs_get_w_dev(self.ctx, int(site), _P(out_ptr)), "lrs_get_w_dev")

    def backward(self, site, grad_w=None, grad_chi0=None):
        n = self.npts[site]
        gw = None if grad_w is None else _f64(grad_w)
        gc = None if grad_chi0 is None else _f64(grad_chi0)
        ge = np.empty((self.nk, self.nb))
        gp = np.empty((n, self.nk * self.nb), np.complex128)
        _check(lrs_backward(self.ctx, int(site), None if gw is None else _dp(gw), None if gc is None else _dp(gc),
                            _dp(ge), _dp(gp.view(np.float64))), "lrs_backward")
        return ge, gp

    def backward_dev(self, site, grad_w_ptr, grad_chi0_ptr, grad_e_ptr, grad_psi_ptr):
        _check(lrs_backward_dev(self.ctx, int(site), _P(grad_w_ptr or 0), _P(grad_chi0_ptr or 0),
                                _P(grad_e_ptr), _P(grad_psi_ptr)), "lrs_backward_dev")

    def graph_capture(self, sites=None):
        n, p, _keep = self._sites(sites)
        _check(lrs_graph_capture(self.ctx, n, p), "lrs_graph_capture")

    def graph_launch(self):
        _check(lrs_graph_launch(self.ctx), "lrs_graph_launch")

    def autotune(self, sites=None):
        n, p, _keep = self._sites(sites)
        tn, seg, ms = C.c_int(), C.c_int(), C.c_double()
        _check(lrs_autotune(self.ctx, n, p, C.byref(tn), C.byref(seg), C.byref(ms)), "lrs_autotune")
        return {"tile_n": tn.value, "segment": seg.value, "ms_chi0": ms.value}

    def synchronize(self):
        _check(lrs_synchronize(self.ctx), "lrs_synchronize")

    def stats(self):
        s = lrs_stats_t()
        _check(lrs_stats(self.ctx, C.byref(s)), "lrs_stats")
        return {name: getattr(s, name) for name, _ in lrs_stats_t._fields_}


def exported_symbols():
    return sorted(_SIGS)
