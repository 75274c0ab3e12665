"""The allocation-free FP32 entry point (dsps_photometry_fp32_static), called
through the C ABI, against the regular dsps_photometry FP32 call on the same
inputs, twice in a row with different populations: the second call must not see
anything the first left in the shared static scratch.  The static call runs on
unsorted rows over every wavelength tile, the regular one on sorted rows over
each tile's band, so the two agree to the FP32 tolerance (summation order), and
each is also held to the FP64 oracle directly.  A nebular grid (7 log U values,
a third SSP axis) takes the same entry point with its 14 parameter rows."""
import ctypes
import functools

import numpy as np
import pytest

import oracle

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static(lib, ctx, n, d_p, sid, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.dsps_photometry_fp32_static(ctx.handle, n, ctypes.c_void_p(d_p.data_ptr()), sid,
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_static_scratch_entry_point_matches_regular_call():
    from paper_2112_06830_gb300 import dsps, synth

    ctx = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH)
    f = synth.make_filters(12)
    sid = ctx.add_filters(f)
    F = oracle.Filters(f)
    lib = dsps.load()
    for n, start in ((3000, 0), (1234, 50_000)):
        p = synth.make_population(synth.SFH_DPL_QUENCH, n, 1, start=start)
        p32, p64 = _util.params_f32(p)
        d_p = torch.from_numpy(p32).cuda()
        ref = ctx.photometry(d_p, sid, precision=dsps.DSPS_PREC_FP32)
        out = torch.full_like(ref, float("nan"))
        rc = _static(lib, ctx, n, d_p, sid, out)
        assert rc == dsps.DSPS_OK, lib.dsps_last_error_message()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, want, rtol=0, atol=_util.TOL_FP32)
        idx = np.unique(np.r_[0, n - 1, np.arange(0, n, n // 23)])
        orc = oracle.mags(_util.oracle_grid("full", 1), F, np.ascontiguousarray(p64[:, idx]))
        err = np.abs(got[idx].astype(np.float64) - orc).max()
        print(f"static entry, {n} galaxies: max |dm| vs oracle on {len(idx)} = {err:.2e}")
        assert err <= _util.TOL_FP32
    # a population larger than the static scratch is refused with a clear message
    rc = _static(lib, ctx, 10_000_000, d_p, sid, out)
    assert rc == dsps.DSPS_ERR_INVALID_ARG
    assert b"static scratch" in lib.dsps_last_error_message()
    assert ctx.device_error() == 0
    ctx.close()


@functools.lru_cache(maxsize=None)
def _neb_ssp():
    from paper_2112_06830_gb300 import synth
    return synth.make_ssp_nebular(synth.FULL_GRID, 1)


def test_static_scratch_entry_point_nebular_grid():
    from paper_2112_06830_gb300 import dsps, synth

    g = _neb_ssp()
    ctx = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH, max_chunk=32768)
    f = synth.make_filters(12)
    sid = ctx.add_filters(f)
    lib = dsps.load()
    og = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                     sfh_model=synth.SFH_DPL_QUENCH, lgu=g.lgu)
    for n, start in ((400, 0), (257, 9000)):
        p = synth.with_nebular(synth.make_population(synth.SFH_DPL_QUENCH, n, 41, start), 41, start)
        p32, p64 = _util.params_f32(p)
        d_p = torch.from_numpy(p32).cuda()
        ref = ctx.photometry(d_p, sid, precision=dsps.DSPS_PREC_FP32)
        out = torch.full_like(ref, float("nan"))
        rc = _static(lib, ctx, n, d_p, sid, out)
        assert rc == dsps.DSPS_OK, lib.dsps_last_error_message()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, want, rtol=0, atol=_util.TOL_FP32)
        idx = np.array([0, 1, n // 2, n - 1])
        orc = oracle.mags(og, oracle.Filters(f), np.ascontiguousarray(p64[:, idx]))
        assert np.abs(got[idx].astype(np.float64) - orc).max() <= _util.TOL_FP32
    assert ctx.device_error() == 0
    ctx.close()
