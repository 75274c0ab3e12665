"""Plain FP64 CPU oracle of the DSPS photometry hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package smoke check and
by the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The arithmetic lives in ``oracle.c`` (plain C, double precision, loop by loop,
each function citing the equation of Hearin et al. 2021, arXiv:2112.06830 it
follows).  This module compiles it with gcc on first use and marshals numpy
arrays through ctypes.  Parameters use the structure-of-arrays layout described
in ``oracle.c``: ``params[12, G]`` (sfh0..4, mdf_mu, mdf_sigma, mdf_slope, Av,
delta, logM, z) and gradients ``[11, G]`` (the same rows without z), each with
the grid's optional blocks after them (``Grid.npar``, ``Grid.ngrad``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPAR = 12
NGRAD = 11
SFH_TABLE = 2   # sfh_model: SFR tabulated at the n_t time nodes (the last n_t parameter rows)
AB0 = 1.13492e-13


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("n_age", C.c_int), ("n_z", C.c_int), ("n_lam", C.c_int),
                ("log_age_yr", C.POINTER(C.c_double)), ("lgz", C.POINTER(C.c_double)),
                ("lam", C.POINTER(C.c_double)), ("l_ssp", C.POINTER(C.c_double)),
                ("t0", C.c_double), ("t1", C.c_double), ("n_t", C.c_int),
                ("om0", C.c_double), ("w0", C.c_double), ("h", C.c_double),
                ("sfh_model", C.c_int), ("mdf_kernel", C.c_int),
                ("mdf_mean", C.c_int), ("mdf_x0", C.c_double), ("mdf_h", C.c_double),
                ("dust_bump", C.c_int), ("n_u", C.c_int), ("lgu", C.POINTER(C.c_double)),
                ("dust_law", C.c_int), ("dust_agedep", C.c_int), ("dust_x0", C.c_double),
                ("dust_h", C.c_double)]


class _Filters(C.Structure):
    _fields_ = [("n_filt", C.c_int), ("n_pts", C.POINTER(C.c_int)),
                ("lam", C.POINTER(C.c_double)), ("trans", C.POINTER(C.c_double)), ("rest", C.c_int)]


class _Line(C.Structure):
    _fields_ = [("lam_c", C.c_double), ("half_width", C.c_double), ("cont_width", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            for name in ("orc_triweight_pdf", "orc_triweight_cdf", "orc_gauss_cdf", "orc_gauss_pdf"):
                getattr(lib, name).restype = C.c_double
                getattr(lib, name).argtypes = [C.c_double]
            for name in ("orc_age_gyr", "orc_lum_dist_mpc", "orc_dist_mod"):
                getattr(lib, name).restype = C.c_double
                getattr(lib, name).argtypes = [C.c_double] * 4
            lib.orc_sfr.restype = C.c_double
            lib.orc_sfr.argtypes = [C.c_int, dp, C.c_double, dp]
            lib.orc_cum_mass.restype = C.c_double
            lib.orc_cum_mass.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double, dp]
            lib.orc_age_edges_gyr.argtypes = [C.POINTER(_Grid), dp]
            lib.orc_age_fracs_from_sfr.argtypes = [C.POINTER(_Grid), dp, C.c_double, dp]
            lib.orc_mdf.argtypes = [C.POINTER(_Grid), C.c_double, C.c_double, dp, dp, dp]
            lib.orc_mdf_mean.restype = C.c_double
            lib.orc_mdf_mean.argtypes = [C.POINTER(_Grid), dp, C.c_int, dp, dp]
            lib.orc_dust_trans.restype = C.c_double
            lib.orc_pneb.argtypes = [C.POINTER(_Grid), C.c_double, C.c_double, dp, dp, dp]
            lib.orc_pneb.restype = None
            lib.orc_k0.argtypes = [C.c_double]
            lib.orc_k0.restype = C.c_double
            lib.orc_dust_trans.argtypes = [C.c_double] * 3
            lib.orc_drude.restype = C.c_double
            lib.orc_drude.argtypes = [C.c_double]
            lib.orc_dust_curve.restype = C.c_double
            lib.orc_dust_curve.argtypes = [C.POINTER(_Grid), C.c_double, C.c_double, dp]
            lib.orc_filter_trans.restype = C.c_double
            lib.orc_filter_trans.argtypes = [dp, dp, C.c_int, C.c_double]
            lib.orc_filter_norm.restype = C.c_double
            lib.orc_filter_norm.argtypes = [dp, dp, C.c_int]
            lib.orc_mags_from_weights.argtypes = [C.POINTER(_Grid), C.POINTER(_Filters), dp,
                                                  C.c_double, C.c_double, C.c_double, C.c_double,
                                                  C.c_double, dp]
            lib.orc_weights.argtypes = [C.POINTER(_Grid), C.c_long, dp, dp, C.c_int]
            lib.orc_mags.argtypes = [C.POINTER(_Grid), C.POINTER(_Filters), C.c_long, dp, dp, C.c_int]
            lib.orc_ew_from_spectrum.argtypes = [dp, dp, C.c_int, C.POINTER(_Line), dp]
            lib.orc_ew_from_spectrum.restype = C.c_double
            lib.orc_spectra.argtypes = [C.POINTER(_Grid), C.c_long, dp, dp, C.c_int]
            lib.orc_line_ew.argtypes = [C.POINTER(_Grid), C.POINTER(_Line), C.c_long, dp, dp, dp, dp, C.c_int]
            lib.orc_mags_vjp.argtypes = [C.POINTER(_Grid), C.POINTER(_Filters), C.c_long, dp, dp,
                                         dp, dp, C.c_int]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Grid:
    """SSP grid + SFR time grid + cosmology + model switches, held as float64."""

    def __init__(self, log_age_yr, lgz, lam, l_ssp, t0=0.05, t1=13.8, n_t=200,
                 om0=0.3, w0=-1.0, h=0.7, sfh_model=0, mdf_kernel=0, mdf_mean=0, mdf_x0=9.0, mdf_h=0.5,
                 dust_bump=0, lgu=None, dust_law=0, dust_agedep=0, dust_x0=7.0, dust_h=0.1):
        self.log_age_yr = _f64(log_age_yr)
        self.lgz = _f64(lgz)
        self.lam = _f64(lam)
        self.lgu = _f64(lgu) if lgu is not None and len(lgu) > 1 else None
        nu = len(self.lgu) if self.lgu is not None else 1
        self.l_ssp = _f64(l_ssp).reshape(len(self.log_age_yr), len(self.lgz), nu, len(self.lam))
        self.t0, self.t1, self.n_t = float(t0), float(t1), int(n_t)
        self.om0, self.w0, self.h = float(om0), float(w0), float(h)
        self.sfh_model, self.mdf_kernel = int(sfh_model), int(mdf_kernel)
        self.mdf_mean, self.mdf_x0, self.mdf_h = int(mdf_mean), float(mdf_x0), float(mdf_h)
        self.dust_bump = int(dust_bump)
        self.dust_law = int(dust_law)
        self.dust_agedep, self.dust_x0, self.dust_h = int(dust_agedep), float(dust_x0), float(dust_h)
        self._c = _Grid(len(self.log_age_yr), len(self.lgz), len(self.lam), _dp(self.log_age_yr),
                        _dp(self.lgz), _dp(self.lam), _dp(self.l_ssp), self.t0, self.t1, self.n_t,
                        self.om0, self.w0, self.h, self.sfh_model, self.mdf_kernel,
                        self.mdf_mean, self.mdf_x0, self.mdf_h, self.dust_bump, nu,
                        _dp(self.lgu) if self.lgu is not None else None, self.dust_law,
                        self.dust_agedep, self.dust_x0, self.dust_h)

    @property
    def n_age(self):
        return len(self.log_age_yr)

    @property
    def n_z(self):
        return len(self.lgz)

    @property
    def n_lam(self):
        return len(self.lam)

    @property
    def n_u(self):
        return len(self.lgu) if self.lgu is not None else 1

    # Parameter rows: 0-11, then (nebular axis) log U mean and width, then
    # (age-dependent dust) Av_old and delta_old, then (tabulated SFH) the SFR at
    # the n_t time nodes; gradient rows: 0-10, then the same blocks in order.
    @property
    def row_sfr(self):
        return NPAR + (2 if self.n_u > 1 else 0) + (2 if self.dust_agedep else 0)

    @property
    def grow_sfr(self):
        return NGRAD + (2 if self.n_u > 1 else 0) + (2 if self.dust_agedep else 0)

    @property
    def npar(self):
        return self.row_sfr + (self.n_t if self.sfh_model == SFH_TABLE else 0)

    @property
    def ngrad(self):
        return self.grow_sfr + (self.n_t if self.sfh_model == SFH_TABLE else 0)


class Filters:
    """A list of (lambda [A], transmission) tables; rest=True gives rest-frame
    absolute magnitudes M_Q (Eq. restmag) instead of observer-frame apparent
    ones."""

    def __init__(self, tables, rest=False):
        self.tables = [(_f64(l), _f64(t)) for l, t in tables]
        self.rest = bool(rest)
        self.n_pts = np.array([len(l) for l, _ in self.tables], dtype=np.int32)
        self.lam = _f64(np.concatenate([l for l, _ in self.tables]))
        self.trans = _f64(np.concatenate([t for _, t in self.tables]))
        self._c = _Filters(len(self.tables), self.n_pts.ctypes.data_as(C.POINTER(C.c_int)),
                           _dp(self.lam), _dp(self.trans), 1 if rest else 0)

    @property
    def n_filt(self):
        return len(self.tables)


def _nthreads(n):
    if n is not None:
        return int(n)
    return os.cpu_count() or 1


# ---- scalar functions -------------------------------------------------------

def triweight_pdf(z):
    return _load().orc_triweight_pdf(float(z))


def triweight_cdf(z):
    return _load().orc_triweight_cdf(float(z))


def gauss_cdf(z):
    return _load().orc_gauss_cdf(float(z))


def age_gyr(z, om0=0.3, w0=-1.0, h=0.7):
    return _load().orc_age_gyr(om0, w0, h, float(z))


def lum_dist_mpc(z, om0=0.3, w0=-1.0, h=0.7):
    return _load().orc_lum_dist_mpc(om0, w0, h, float(z))


def dist_mod(z, om0=0.3, w0=-1.0, h=0.7):
    return _load().orc_dist_mod(om0, w0, h, float(z))


def sfr(model, p, t):
    p = _f64(np.resize(np.asarray(p, dtype=np.float64), 5))
    g = np.zeros(5)
    v = _load().orc_sfr(int(model), _dp(p), float(t), _dp(g))
    return v, g


def cum_mass(sfr_nodes, t0, t1, tau):
    s = _f64(sfr_nodes)
    coef = np.zeros(len(s))
    v = _load().orc_cum_mass(_dp(s), len(s), float(t0), float(t1), float(tau), _dp(coef))
    return v, coef


def age_edges_gyr(grid: Grid):
    e = np.zeros(grid.n_age + 1)
    _load().orc_age_edges_gyr(C.byref(grid._c), _dp(e))
    return e


def age_fracs_from_sfr(grid: Grid, sfr_nodes, t_obs):
    s = _f64(sfr_nodes)
    assert len(s) == grid.n_t
    out = np.zeros(grid.n_age)
    _load().orc_age_fracs_from_sfr(C.byref(grid._c), _dp(s), float(t_obs), _dp(out))
    return out


def mdf_mean(grid: Grid, params, i):
    """(mu_i, d mu_i / d p5, d mu_i / d p7) for age bin i of one galaxy's parameters."""
    p = _f64(params)
    d5, d7 = np.zeros(1), np.zeros(1)
    mu = _load().orc_mdf_mean(C.byref(grid._c), _dp(p), int(i), _dp(d5), _dp(d7))
    return mu, float(d5[0]), float(d7[0])


def pneb(grid: Grid, u_mean, u_sigma):
    """(P[n_u], dP/du_mean, dP/du_sigma) of the nebular log U bins (Eq. nebsed)."""
    n = grid.n_u
    P, d1, d2 = np.zeros(n), np.zeros(n), np.zeros(n)
    _load().orc_pneb(C.byref(grid._c), float(u_mean), float(u_sigma), _dp(P), _dp(d1), _dp(d2))
    return P, d1, d2


def mdf(grid: Grid, mu_i, sigma):
    P, dmu, dsig = np.zeros(grid.n_z), np.zeros(grid.n_z), np.zeros(grid.n_z)
    _load().orc_mdf(C.byref(grid._c), float(mu_i), float(sigma), _dp(P), _dp(dmu), _dp(dsig))
    return P, dmu, dsig


def drude(lam):
    return _load().orc_drude(float(lam))


def dust_curve(grid: Grid, lam, delta):
    """(A_lambda / Av, its derivative in delta) under the grid's dust options."""
    d = np.zeros(1)
    c = _load().orc_dust_curve(C.byref(grid._c), float(lam), float(delta), _dp(d))
    return c, float(d[0])


def colour_cut_histogram(mags, band_a, band_b, cut, band_r, lo, hi, n_bins):
    """Sec. 5.1's population statistic: galaxies with colour m_a - m_b > cut,
    counted in n_bins uniform bins of m_r on [lo, hi) (float64, plain
    definition; NaN rows and values outside the range are not counted)."""
    m = np.asarray(mags, dtype=np.float64)
    sel = (m[:, band_a] - m[:, band_b]) > cut
    r = m[sel, band_r]
    r = r[(r >= lo) & (r < hi)]
    return np.histogram(r, bins=n_bins, range=(lo, hi))[0].astype(np.int64)


def k0(lam):
    """The starburst curve k0 of Eq. (kzero) at lam [A]."""
    return _load().orc_k0(float(lam))


def dust_trans(lam, Av, delta):
    return _load().orc_dust_trans(float(lam), float(Av), float(delta))


def filter_trans(lam_tab, tr_tab, x):
    l, t = _f64(lam_tab), _f64(tr_tab)
    return _load().orc_filter_trans(_dp(l), _dp(t), len(l), float(x))


def filter_norm(lam_tab, tr_tab):
    l, t = _f64(lam_tab), _f64(tr_tab)
    return _load().orc_filter_norm(_dp(l), _dp(t), len(l))


def mags_from_weights(grid: Grid, filters: Filters, omega, Av, delta, logM, z, dmod):
    w = _f64(omega).reshape(-1)
    out = np.zeros(filters.n_filt)
    _load().orc_mags_from_weights(C.byref(grid._c), C.byref(filters._c), _dp(w), float(Av),
                                  float(delta), float(logM), float(z), float(dmod), _dp(out))
    return out


# ---- batched entry points ---------------------------------------------------

def _params(grid: Grid, params) -> np.ndarray:
    p = _f64(params)
    if p.ndim != 2 or p.shape[0] < grid.npar:
        raise ValueError(f"params must be [{grid.npar}, G] for this grid, got {p.shape}")
    return p


def weights(grid: Grid, params, nthreads=None):
    """SSP weights in Msun, shape [G, n_age, n_z] (or [G, n_age, n_z, n_u])."""
    p = _params(grid, params)
    G = p.shape[1]
    out = np.zeros((G, grid.n_age, grid.n_z) + ((grid.n_u,) if grid.n_u > 1 else ()))
    _load().orc_weights(C.byref(grid._c), G, _dp(p), _dp(out), _nthreads(nthreads))
    return out


def mags(grid: Grid, filters: Filters, params, nthreads=None):
    """Observer-frame AB magnitudes, shape [G, Q]."""
    p = _params(grid, params)
    G = p.shape[1]
    out = np.zeros((G, filters.n_filt))
    _load().orc_mags(C.byref(grid._c), C.byref(filters._c), G, _dp(p), _dp(out), _nthreads(nthreads))
    return out


def mags_vjp(grid: Grid, filters: Filters, params, mag_bar, nthreads=None):
    """Returns (mags [G, Q], param_bar [ngrad, G]) with param_bar = J^T mag_bar."""
    p = _params(grid, params)
    G = p.shape[1]
    mb = _f64(mag_bar).reshape(G, filters.n_filt)
    m = np.zeros((G, filters.n_filt))
    pb = np.zeros((grid.ngrad, G))
    _load().orc_mags_vjp(C.byref(grid._c), C.byref(filters._c), G, _dp(p), _dp(mb), _dp(m), _dp(pb),
                         _nthreads(nthreads))
    return m, pb


# ---- emission-line equivalent width (Sec. 2.2, Eq. eqw) --------------------

def ew_from_spectrum(lam, L, lam_c, half_width, cont_width):
    """(W [A], dW/dL) of a tabulated spectrum: quadratic continuum fitted on
    half_width < |lam - lam_c| <= half_width + cont_width, trapezoid of
    (L - L0)/L0 over |lam - lam_c| <= half_width."""
    l, v = _f64(lam), _f64(L)
    lb = np.zeros(len(l))
    ln = _Line(float(lam_c), float(half_width), float(cont_width))
    w = _load().orc_ew_from_spectrum(_dp(l), _dp(v), len(l), C.byref(ln), _dp(lb))
    return w, lb


def spectra(grid: Grid, params, nthreads=None):
    """Rest-frame attenuated spectra 10^logM F S, shape [G, n_lam] [Lsun/Hz]."""
    p = _params(grid, params)
    G = p.shape[1]
    out = np.zeros((G, grid.n_lam))
    _load().orc_spectra(C.byref(grid._c), G, _dp(p), _dp(out), _nthreads(nthreads))
    return out


def line_ew(grid: Grid, params, lam_c, half_width, cont_width, nthreads=None):
    """Equivalent widths [G] of the galaxies' rest-frame spectra."""
    p = _params(grid, params)
    G = p.shape[1]
    ew = np.zeros(G)
    ln = _Line(float(lam_c), float(half_width), float(cont_width))
    _load().orc_line_ew(C.byref(grid._c), C.byref(ln), G, _dp(p), None, _dp(ew), None, _nthreads(nthreads))
    return ew


def line_ew_vjp(grid: Grid, params, ew_bar, lam_c, half_width, cont_width, nthreads=None):
    """(ew [G], param_bar [ngrad, G]) with param_bar[k, g] = ew_bar[g] dW_g/dp_k."""
    p = _params(grid, params)
    G = p.shape[1]
    eb = _f64(ew_bar).reshape(G)
    ew = np.zeros(G)
    pb = np.zeros((grid.ngrad, G))
    ln = _Line(float(lam_c), float(half_width), float(cont_width))
    _load().orc_line_ew(C.byref(grid._c), C.byref(ln), G, _dp(p), _dp(eb), _dp(ew), _dp(pb),
                        _nthreads(nthreads))
    return ew, pb
