"""Thin ctypes binding of libdsps (include/dsps.h).

The functions ``dsps_*`` below have the names and arguments of the C ABI and
only marshal arguments; every step of the photometry path runs in the CUDA
library.  ``Context`` is a small convenience layer over them that takes torch
tensors (torch is used for device memory and streams only).

Loading fails loudly (``RuntimeError``) when libdsps.so cannot be built or
loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

DSPS_OK = 0
DSPS_PENDING = 1
DSPS_ERR_INVALID_ARG = -1
DSPS_ERR_OUT_OF_BUDGET = -2
DSPS_ERR_CUDA = -3
DSPS_ERR_TIMEOUT = -4
DSPS_BUF_HOST = 0
DSPS_BUF_DEVICE = 1
DSPS_ERR_DEVICE_FAULT = -5
DSPS_ERR_UNSUPPORTED = -6
DSPS_ERR_NOT_FOUND = -7

DSPS_SFH_DELAYED_TAU = 0
DSPS_SFH_DPL_QUENCH = 1
DSPS_SFH_TABLE = 2
DSPS_FRAME_OBSERVER = 0
DSPS_FRAME_REST = 1
DSPS_MDF_TRIWEIGHT = 0
DSPS_MDF_GAUSSIAN = 1
DSPS_MDF_MEAN_LINEAR = 0
DSPS_MDF_MEAN_TERF = 1
DSPS_DUST_POWERLAW = 0
DSPS_DUST_SALIM = 1
DSPS_PREC_FP32 = 0
DSPS_PREC_BF16X3 = 1
DSPS_NPAR = 12
DSPS_NGRAD = 11
DSPS_NPAR_NEB = 14
DSPS_NGRAD_NEB = 13
DSPS_MAX_NU = 8
DSPS_MAX_FILTERS = 16


class dsps_grid(C.Structure):
    _fields_ = [("n_age", C.c_int32), ("n_z", C.c_int32), ("n_lam", C.c_int32),
                ("log_age_yr", C.POINTER(C.c_double)), ("lgz", C.POINTER(C.c_double)),
                ("lam", C.POINTER(C.c_double)), ("l_ssp", C.POINTER(C.c_float)),
                ("t0_gyr", C.c_double), ("t1_gyr", C.c_double), ("n_t", C.c_int32),
                ("n_u", C.c_int32), ("lgu", C.POINTER(C.c_double))]


class dsps_opts(C.Structure):
    _fields_ = [("om0", C.c_double), ("w0", C.c_double), ("h", C.c_double),
                ("sfh_model", C.c_int32), ("mdf_kernel", C.c_int32), ("device", C.c_int32),
                ("max_chunk", C.c_int64), ("hbm_budget_bytes", C.c_int64), ("n_streams", C.c_int32),
                ("z_max", C.c_double), ("band_skip", C.c_int32), ("mdf_mean", C.c_int32),
                ("mdf_terf_x0", C.c_double), ("mdf_terf_h", C.c_double), ("dust_bump", C.c_int32),
                ("dust_law", C.c_int32), ("dust_agedep", C.c_int32), ("dust_agedep_x0", C.c_double),
                ("dust_agedep_h", C.c_double), ("agedep_fused", C.c_int32)]


DSPS_PROF_KINDS = 4


class dsps_profile_t(C.Structure):
    _fields_ = [("launches", C.c_int64 * DSPS_PROF_KINDS), ("ms", C.c_double * DSPS_PROF_KINDS),
                ("tc_kblocks", C.c_int64), ("simt_steps", C.c_int64),
                ("tc_kblocks_n128", C.c_int64)]


DSPS_MAX_HIST_BINS = 4096


class dsps_hist_spec(C.Structure):
    _fields_ = [("band_a", C.c_int32), ("band_b", C.c_int32), ("cut", C.c_float), ("band_r", C.c_int32),
                ("lo", C.c_float), ("hi", C.c_float), ("n_bins", C.c_int32)]


DSPS_MAX_LINE_POINTS = 4096


class dsps_line_spec(C.Structure):
    _fields_ = [("lam_line", C.c_double), ("half_width", C.c_double), ("cont_width", C.c_double)]


class dsps_request(C.Structure):
    _fields_ = [("n_gal", C.c_int64), ("params", C.c_void_p), ("set_id", C.c_int32),
                ("precision", C.c_int32), ("want_grad", C.c_int32), ("mag_bar", C.c_void_p),
                ("mags", C.c_void_p), ("param_bar", C.c_void_p), ("buffers", C.c_int32)]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes)
_SIGS = [
    ("dsps_default_opts", None, [C.POINTER(dsps_opts)]),
    ("dsps_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(dsps_grid), C.POINTER(dsps_opts)]),
    ("dsps_destroy", C.c_int, [C.c_void_p]),
    ("dsps_filters_add", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                   C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.POINTER(C.c_double)),
                                   C.POINTER(C.c_int32)]),
    ("dsps_filters_add_frame", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                         C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.POINTER(C.c_double)),
                                         C.c_int32, C.POINTER(C.c_int32)]),
    ("dsps_filters_count", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    ("dsps_band_coverage", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("dsps_weights", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("dsps_photometry", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                  C.c_void_p]),
    ("dsps_photometry_vjp", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    ("dsps_photometry_fp32_static", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                              C.c_void_p]),
    ("dsps_photometry_histogram", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_int32,
                                            C.POINTER(dsps_hist_spec), C.c_void_p, C.c_void_p]),
    ("dsps_histogram", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.POINTER(dsps_hist_spec),
                                 C.c_void_p, C.c_void_p]),
    ("dsps_spectra", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    ("dsps_line_add", C.c_int, [C.c_void_p, C.POINTER(dsps_line_spec), C.POINTER(C.c_int32)]),
    ("dsps_line_ew", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("dsps_line_ew_vjp", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    ("dsps_submit", C.c_int, [C.c_void_p, C.POINTER(dsps_request), C.POINTER(C.c_uint64)]),
    ("dsps_poll", C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(C.c_double)]),
    ("dsps_photometry_host", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                       C.c_void_p]),
    ("dsps_device_error", C.c_int, [C.c_void_p, C.c_void_p]),
    ("dsps_profile_enable", C.c_int, [C.c_void_p, C.c_int32]),
    ("dsps_profile_read", C.c_int, [C.c_void_p, C.POINTER(dsps_profile_t)]),
    ("dsps_strerror", C.c_char_p, [C.c_int]),
    ("dsps_last_error_message", C.c_char_p, []),
]


def library_path() -> str:
    return _build.LIB


def load():
    """Builds (if needed) and loads libdsps.so; raises RuntimeError on failure."""
    global _lib
    with _lock:
        if _lib is None:
            try:
                path = _build.build()
                lib = C.CDLL(path)
            except Exception as e:  # noqa: BLE001
                raise RuntimeError(f"libdsps.so could not be built or loaded: {e}") from e
            for name, res, args in _SIGS:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class DSPSError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.dsps_last_error_message().decode(errors="replace")
        super().__init__(f"{where}: {lib.dsps_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def _check(code, where):
    if code < 0:
        raise DSPSError(code, where)
    return code


# ---- C ABI, one function per entry point -------------------------------------

def dsps_default_opts():
    o = dsps_opts()
    load().dsps_default_opts(C.byref(o))
    return o


def dsps_create(grid: dsps_grid, opts: dsps_opts):
    h = C.c_void_p()
    _check(load().dsps_create(C.byref(h), C.byref(grid), C.byref(opts)), "dsps_create")
    return h


def dsps_destroy(ctx):
    return _check(load().dsps_destroy(ctx), "dsps_destroy")


def dsps_filters_add(ctx, tables, frame=None):
    """Registers a filter set; frame DSPS_FRAME_REST gives rest-frame absolute
    magnitudes (Eq. restmag), the default observer-frame apparent ones."""
    n = len(tables)
    lam = [np.ascontiguousarray(l, dtype=np.float64) for l, _ in tables]
    tr = [np.ascontiguousarray(t, dtype=np.float64) for _, t in tables]
    n_pts = (C.c_int32 * n)(*[len(x) for x in lam])
    lp = (C.POINTER(C.c_double) * n)(*[x.ctypes.data_as(C.POINTER(C.c_double)) for x in lam])
    tp = (C.POINTER(C.c_double) * n)(*[x.ctypes.data_as(C.POINTER(C.c_double)) for x in tr])
    sid = C.c_int32()
    if frame is None:
        _check(load().dsps_filters_add(ctx, n, n_pts, lp, tp, C.byref(sid)), "dsps_filters_add")
    else:
        _check(load().dsps_filters_add_frame(ctx, n, n_pts, lp, tp, int(frame), C.byref(sid)), "dsps_filters_add")
    return sid.value


def dsps_filters_count(ctx, set_id):
    q = C.c_int32()
    _check(load().dsps_filters_count(ctx, set_id, C.byref(q)), "dsps_filters_count")
    return q.value


def dsps_band_coverage(ctx, n_gal, params_ptr, set_id, coverage_ptr, stream=0):
    _check(load().dsps_band_coverage(ctx, n_gal, params_ptr, set_id, coverage_ptr, stream), "dsps_band_coverage")


def dsps_weights(ctx, n_gal, params_ptr, w_out_ptr, stream=0):
    return _check(load().dsps_weights(ctx, n_gal, params_ptr, w_out_ptr, stream), "dsps_weights")


def dsps_photometry(ctx, n_gal, params_ptr, set_id, precision, mags_ptr, stream=0):
    return _check(load().dsps_photometry(ctx, n_gal, params_ptr, set_id, precision, mags_ptr, stream),
                  "dsps_photometry")


def dsps_photometry_vjp(ctx, n_gal, params_ptr, set_id, precision, mag_bar_ptr, mags_ptr, param_bar_ptr,
                        stream=0):
    return _check(load().dsps_photometry_vjp(ctx, n_gal, params_ptr, set_id, precision, mag_bar_ptr,
                                             mags_ptr, param_bar_ptr, stream), "dsps_photometry_vjp")


def dsps_photometry_histogram(ctx, n_gal, params_ptr, set_id, precision, spec, counts_ptr, stream=0):
    return _check(load().dsps_photometry_histogram(ctx, n_gal, params_ptr, set_id, precision, C.byref(spec),
                                                   counts_ptr, stream), "dsps_photometry_histogram")


def dsps_histogram(ctx, n_gal, mags_ptr, n_filt, spec, counts_ptr, stream=0):
    return _check(load().dsps_histogram(ctx, n_gal, mags_ptr, n_filt, C.byref(spec), counts_ptr, stream),
                  "dsps_histogram")


def dsps_photometry_fp32_static(ctx, n_gal, params_ptr, set_id, mags_ptr, stream=0):
    """FP32 photometry with no device allocation (fixed in-library scratch)."""
    return _check(load().dsps_photometry_fp32_static(ctx, n_gal, params_ptr, set_id, mags_ptr, stream),
                  "dsps_photometry_fp32_static")


def dsps_spectra(ctx, n_gal, params_ptr, n0, n1, out_ptr, stream=0):
    return _check(load().dsps_spectra(ctx, n_gal, params_ptr, n0, n1, out_ptr, stream), "dsps_spectra")


def dsps_line_add(ctx, spec: dsps_line_spec):
    lid = C.c_int32(-1)
    _check(load().dsps_line_add(ctx, C.byref(spec), C.byref(lid)), "dsps_line_add")
    return lid.value


def dsps_line_ew(ctx, n_gal, params_ptr, line_id, ew_ptr, stream=0):
    return _check(load().dsps_line_ew(ctx, n_gal, params_ptr, line_id, ew_ptr, stream), "dsps_line_ew")


def dsps_line_ew_vjp(ctx, n_gal, params_ptr, line_id, ew_bar_ptr, ew_ptr, param_bar_ptr, stream=0):
    return _check(load().dsps_line_ew_vjp(ctx, n_gal, params_ptr, line_id, ew_bar_ptr, ew_ptr, param_bar_ptr,
                                          stream), "dsps_line_ew_vjp")


def dsps_submit(ctx, req: dsps_request):
    t = C.c_uint64()
    _check(load().dsps_submit(ctx, C.byref(req), C.byref(t)), "dsps_submit")
    return t.value


def dsps_poll(ctx, ticket, timeout_us=0):
    """(rc, latency_us): rc is DSPS_OK, DSPS_PENDING (timeout 0) or
    DSPS_ERR_TIMEOUT (a positive timeout elapsed); other errors raise."""
    lat = C.c_double(0.0)
    rc = load().dsps_poll(ctx, ticket, timeout_us, C.byref(lat))
    if rc != DSPS_ERR_TIMEOUT:
        _check(rc, "dsps_poll")
    return rc, lat.value


def dsps_photometry_host(ctx, n_gal, params_ptr, set_id, precision, mags_ptr, stream=0):
    """Host buffers in and out, one call (synchronises the stream)."""
    return _check(load().dsps_photometry_host(ctx, n_gal, params_ptr, set_id, precision, mags_ptr, stream),
                  "dsps_photometry_host")


def dsps_device_error(ctx, stream=0):
    return load().dsps_device_error(ctx, stream)


def dsps_profile_enable(ctx, enable=True):
    return _check(load().dsps_profile_enable(ctx, 1 if enable else 0), "dsps_profile_enable")


def dsps_profile_read(ctx):
    """{kind: (launches, ms)} for kinds 0 weights/sort/combine, 1 fp32, 2 tensor, 3 adjoint, plus
    "tc_kblocks": 128 x 256 x 32 split-bf16 tensor-core block products executed,
    "simt_steps": 128 x 128 x 16 FP32 tile steps of the FP32 photometry contraction and
    "tc_kblocks_n128": 128 x 128 x 32 split-bf16 block products of the one-launch
    age-dependent dust contraction."""
    p = dsps_profile_t()
    _check(load().dsps_profile_read(ctx, C.byref(p)), "dsps_profile_read")
    out = {k: (int(p.launches[k]), float(p.ms[k])) for k in range(DSPS_PROF_KINDS)}
    out["tc_kblocks"] = int(p.tc_kblocks)
    out["simt_steps"] = int(p.simt_steps)
    out["tc_kblocks_n128"] = int(p.tc_kblocks_n128)
    return out


def dsps_strerror(code):
    return load().dsps_strerror(code).decode()


# ---- convenience layer over torch tensors ------------------------------------

def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Context:
    """Owns a dsps context (resident SSP block, cosmology table, work space)."""

    def __init__(self, ssp, sfh_model=DSPS_SFH_DELAYED_TAU, mdf_kernel=DSPS_MDF_TRIWEIGHT, device=0,
                 max_chunk=None, hbm_budget_bytes=None, n_streams=None, om0=0.3, w0=-1.0, h=0.7, z_max=10.0,
                 band_skip=True, mdf_mean=DSPS_MDF_MEAN_LINEAR, mdf_terf_x0=None, mdf_terf_h=None,
                 dust_bump=False, dust_law=DSPS_DUST_POWERLAW, dust_agedep=False, dust_agedep_x0=None,
                 dust_agedep_h=None, agedep_fused=True):
        self._keep = [np.ascontiguousarray(ssp.log_age_yr, dtype=np.float64),
                      np.ascontiguousarray(ssp.lgz, dtype=np.float64),
                      np.ascontiguousarray(ssp.lam, dtype=np.float64),
                      np.ascontiguousarray(ssp.l_ssp, dtype=np.float32)]
        la, lz, lm, ls = self._keep
        lgu = getattr(ssp, "lgu", None)
        lu = np.ascontiguousarray(lgu, dtype=np.float64) if lgu is not None and len(lgu) > 1 else None
        self._keep.append(lu)
        g = dsps_grid(len(la), len(lz), len(lm), la.ctypes.data_as(C.POINTER(C.c_double)),
                      lz.ctypes.data_as(C.POINTER(C.c_double)), lm.ctypes.data_as(C.POINTER(C.c_double)),
                      ls.ctypes.data_as(C.POINTER(C.c_float)), float(ssp.t0), float(ssp.t1), int(ssp.n_t),
                      len(lu) if lu is not None else 0,
                      lu.ctypes.data_as(C.POINTER(C.c_double)) if lu is not None else None)
        o = dsps_default_opts()
        o.om0, o.w0, o.h, o.z_max = om0, w0, h, z_max
        o.sfh_model, o.mdf_kernel, o.device = sfh_model, mdf_kernel, device
        o.band_skip = 1 if band_skip else 0
        o.mdf_mean = mdf_mean
        o.dust_bump = 1 if dust_bump else 0
        o.dust_law = int(dust_law)
        o.dust_agedep = 1 if dust_agedep else 0
        o.agedep_fused = 1 if agedep_fused else 0
        if dust_agedep_x0 is not None:
            o.dust_agedep_x0 = dust_agedep_x0
        if dust_agedep_h is not None:
            o.dust_agedep_h = dust_agedep_h
        if mdf_terf_x0 is not None:
            o.mdf_terf_x0 = mdf_terf_x0
        if mdf_terf_h is not None:
            o.mdf_terf_h = mdf_terf_h
        if max_chunk is not None:
            o.max_chunk = max_chunk
        if hbm_budget_bytes is not None:
            o.hbm_budget_bytes = hbm_budget_bytes
        if n_streams is not None:
            o.n_streams = n_streams
        self.device = device
        self.n_age, self.n_z = len(la), len(lz)
        self.n_u = len(lu) if lu is not None else 1
        # rows 0..11, [u_mean, u_sigma], [Av_old, delta_old], [SFR table];
        # gradient rows 0..10 and the same blocks in the same order
        extra = 2 if dust_agedep else 0                                # Av_old, delta_old
        self.row_sfr = (DSPS_NPAR_NEB if self.n_u > 1 else DSPS_NPAR) + extra
        self.grow_sfr = (DSPS_NGRAD_NEB if self.n_u > 1 else DSPS_NGRAD) + extra
        n_tab = int(ssp.n_t) if sfh_model == DSPS_SFH_TABLE else 0     # SFR at the time nodes
        self.npar = self.row_sfr + n_tab                               # parameter rows
        self.ngrad = self.grow_sfr + n_tab                             # gradient rows
        self.handle = dsps_create(g, o)
        self.n_filt = {}

    def close(self):
        if self.handle:
            dsps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def add_filters(self, tables, rest_frame=False) -> int:
        """A filter set; rest_frame=True for rest-frame absolute magnitudes."""
        sid = dsps_filters_add(self.handle, tables, DSPS_FRAME_REST if rest_frame else None)
        self.n_filt[sid] = len(tables)
        return sid

    def weights(self, params, stream=None):
        import torch
        assert params.is_cuda and params.dtype == torch.float32 and params.shape[0] == self.npar
        params = params.contiguous()
        G = params.shape[1]
        shape = (G, self.n_age, self.n_z) + ((self.n_u,) if self.n_u > 1 else ())
        out = torch.empty(shape, dtype=torch.float32, device=params.device)
        dsps_weights(self.handle, G, params.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def band_coverage(self, params, set_id, stream=None):
        """[G, Q] fraction of each band's filter response on the redshifted SSP grid
        (include/dsps.h: dsps_band_coverage).  A magnitude whose band has coverage
        below about 1e-8 is set by the last points of the filter's far tail and can
        be off by up to ~0.2 mag; at or above it the precision form's tolerance
        holds.  NaN where z is not finite or z <= 0 (observer-frame sets)."""
        import torch
        assert params.is_cuda and params.dtype == torch.float32 and params.shape[0] == self.npar
        params = params.contiguous()
        G = params.shape[1]
        out = torch.empty((G, self.n_filt[set_id]), dtype=torch.float32, device=params.device)
        dsps_band_coverage(self.handle, G, params.data_ptr(), set_id, out.data_ptr(), _stream_handle(stream))
        return out

    def photometry(self, params, set_id, precision=DSPS_PREC_BF16X3, out=None, stream=None):
        import torch
        assert params.is_cuda and params.dtype == torch.float32 and params.shape[0] == self.npar
        params = params.contiguous()
        G = params.shape[1]
        Q = self.n_filt[set_id]
        if out is None:
            out = torch.empty((G, Q), dtype=torch.float32, device=params.device)
        dsps_photometry(self.handle, G, params.data_ptr(), set_id, precision, out.data_ptr(),
                        _stream_handle(stream))
        return out

    def photometry_vjp(self, params, set_id, mag_bar, precision=DSPS_PREC_BF16X3, want_mags=True, stream=None):
        import torch
        params = params.contiguous()
        mag_bar = mag_bar.contiguous().to(torch.float32)
        G = params.shape[1]
        Q = self.n_filt[set_id]
        mags = torch.empty((G, Q), dtype=torch.float32, device=params.device) if want_mags else None
        pbar = torch.empty((self.ngrad, G), dtype=torch.float32, device=params.device)
        dsps_photometry_vjp(self.handle, G, params.data_ptr(), set_id, precision, mag_bar.data_ptr(),
                            mags.data_ptr() if mags is not None else None, pbar.data_ptr(),
                            _stream_handle(stream))
        return mags, pbar

    def photometry_histogram(self, params, set_id, spec, precision=DSPS_PREC_BF16X3, stream=None):
        """Counts (device int64 [n_bins]) of the colour-cut magnitude histogram
        (spec: dsps_hist_spec), the magnitudes never written."""
        import torch
        params = params.contiguous()
        counts = torch.empty(spec.n_bins, dtype=torch.int64, device=params.device)
        dsps_photometry_histogram(self.handle, params.shape[1], params.data_ptr(), set_id, precision, spec,
                                  counts.data_ptr(), _stream_handle(stream))
        return counts

    def histogram(self, mags, spec, stream=None):
        """The same histogram of magnitudes already on the device ([G, Q] float32)."""
        import torch
        mags = mags.contiguous()
        counts = torch.empty(spec.n_bins, dtype=torch.int64, device=mags.device)
        dsps_histogram(self.handle, mags.shape[0], mags.data_ptr(), mags.shape[1], spec, counts.data_ptr(),
                       _stream_handle(stream))
        return counts

    def spectra(self, params, n0, n1, stream=None):
        """Rest-frame attenuated spectra [G, n1 - n0] on grid columns [n0, n1)."""
        import torch
        assert params.is_cuda and params.dtype == torch.float32 and params.shape[0] == self.npar
        params = params.contiguous()
        G = params.shape[1]
        out = torch.empty((G, n1 - n0), dtype=torch.float32, device=params.device)
        dsps_spectra(self.handle, G, params.data_ptr(), n0, n1, out.data_ptr(), _stream_handle(stream))
        return out

    def add_line(self, lam_line, half_width, cont_width) -> int:
        return dsps_line_add(self.handle, dsps_line_spec(float(lam_line), float(half_width), float(cont_width)))

    def line_ew(self, params, line_id, stream=None):
        """Equivalent widths [G] [A] of a registered line."""
        import torch
        assert params.is_cuda and params.dtype == torch.float32 and params.shape[0] == self.npar
        params = params.contiguous()
        G = params.shape[1]
        ew = torch.empty(G, dtype=torch.float32, device=params.device)
        dsps_line_ew(self.handle, G, params.data_ptr(), line_id, ew.data_ptr(), _stream_handle(stream))
        return ew

    def line_ew_vjp(self, params, line_id, ew_bar, stream=None):
        """(ew [G], param_bar [ngrad, G]) with param_bar = ew_bar dW/dparams."""
        import torch
        assert params.is_cuda and params.dtype == torch.float32 and params.shape[0] == self.npar
        params = params.contiguous()
        ew_bar = ew_bar.contiguous().to(torch.float32)
        G = params.shape[1]
        ew = torch.empty(G, dtype=torch.float32, device=params.device)
        pbar = torch.empty((self.ngrad, G), dtype=torch.float32, device=params.device)
        dsps_line_ew_vjp(self.handle, G, params.data_ptr(), line_id, ew_bar.data_ptr(), ew.data_ptr(),
                         pbar.data_ptr(), _stream_handle(stream))
        return ew, pbar

    def device_error(self, stream=None):
        return dsps_device_error(self.handle, _stream_handle(stream))

    def photometry_host(self, params, set_id, precision=DSPS_PREC_BF16X3, out=None, stream=None):
        """Magnitudes of a population held in host memory (numpy or pinned torch
        CPU float32 [npar, G]) in one library call; returns host [G, Q]
        (``out`` if given: a C-contiguous float32 host buffer)."""
        if hasattr(params, "data_ptr"):
            G, ptr = params.shape[1], params.data_ptr()
        else:
            params = np.ascontiguousarray(params, dtype=np.float32)
            G, ptr = params.shape[1], params.ctypes.data
        Q = self.n_filt[set_id]
        if out is None:
            out = np.empty((G, Q), dtype=np.float32)
        optr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        dsps_photometry_host(self.handle, G, ptr, set_id, precision, optr, _stream_handle(stream))
        return out

    # ---- request loop ----
    def submit(self, params, set_id, precision=DSPS_PREC_BF16X3, mag_bar=None):
        """Queues a population: numpy float32 [npar, G] in host memory (12 rows,
        more with the optional blocks), or a CUDA torch tensor of that shape (a
        DSPS_BUF_DEVICE request: mag_bar a CUDA tensor too, outputs allocated on
        the device).  The returned Ticket keeps the buffers alive until it is
        polled."""
        Q = self.n_filt[set_id]
        if hasattr(params, "is_cuda") and params.is_cuda:
            import torch
            params = params.contiguous().to(torch.float32)
            if params.ndim != 2 or params.shape[0] != self.npar:
                raise ValueError(f"params must be [{self.npar}, G], got {tuple(params.shape)}")
            G = params.shape[1]
            t = Ticket(params, torch.empty((G, Q), dtype=torch.float32, device=params.device))
            req = dsps_request(G, params.data_ptr(), set_id, precision, 0, None, t.mags.data_ptr(), None,
                               DSPS_BUF_DEVICE)
            if mag_bar is not None:
                t.mag_bar = mag_bar.contiguous().to(torch.float32).reshape(G, Q)
                t.param_bar = torch.empty((self.ngrad, G), dtype=torch.float32, device=params.device)
                req.want_grad = 1
                req.mag_bar = t.mag_bar.data_ptr()
                req.param_bar = t.param_bar.data_ptr()
            t.id = dsps_submit(self.handle, req)
            return t
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.ndim != 2 or params.shape[0] != self.npar:
            raise ValueError(f"params must be [{self.npar}, G], got {params.shape}")
        G = params.shape[1]
        t = Ticket(params, np.empty((G, Q), dtype=np.float32))
        req = dsps_request(G, params.ctypes.data, set_id, precision, 0, None, t.mags.ctypes.data, None,
                           DSPS_BUF_HOST)
        if mag_bar is not None:
            t.mag_bar = np.ascontiguousarray(mag_bar, dtype=np.float32).reshape(G, Q)
            t.param_bar = np.empty((self.ngrad, G), dtype=np.float32)
            req.want_grad = 1
            req.mag_bar = t.mag_bar.ctypes.data
            req.param_bar = t.param_bar.ctypes.data
        t.id = dsps_submit(self.handle, req)
        return t

    def poll(self, ticket, timeout_us=0):
        """DSPS_OK (outputs ready in ticket.mags / ticket.param_bar),
        DSPS_PENDING (timeout_us = 0, still running) or DSPS_ERR_TIMEOUT (a
        positive timeout elapsed first; poll again)."""
        rc, lat = dsps_poll(self.handle, ticket.id, timeout_us)
        if rc == DSPS_OK:
            ticket.latency_us = lat
        return rc


class Ticket:
    def __init__(self, params, mags):
        self.params = params
        self.mags = mags
        self.mag_bar = None
        self.param_bar = None
        self.id = None
        self.latency_us = None
