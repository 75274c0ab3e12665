"""The allocation-free FP32 entry point (dsps_photometry_fp32_static), called
through the C ABI, against the regular dsps_photometry FP32 call on the same
inputs, twice in a row with different populations: the second call must not see
anything the first left in the shared static scratch."""
import ctypes

import numpy as np
import pytest

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_scratch_entry_point_matches_regular_call():
    from paper_2112_06830_gb300 import dsps, synth

    ctx = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH)
    sid = ctx.add_filters(synth.make_filters(12))
    lib = dsps.load()
    stream = torch.cuda.current_stream().cuda_stream
    for n, start in ((3000, 0), (1234, 50_000)):
        p = synth.make_population(synth.SFH_DPL_QUENCH, n, 1, start=start).astype(np.float32)
        d_p = torch.from_numpy(p).cuda()
        ref = ctx.photometry(d_p, sid, precision=dsps.DSPS_PREC_FP32)
        out = torch.full_like(ref, float("nan"))
        rc = lib.dsps_photometry_fp32_static(ctx.handle, n, ctypes.c_void_p(d_p.data_ptr()), sid,
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == dsps.DSPS_OK, lib.dsps_last_error_message()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, want, rtol=0, atol=_util.TOL_FP32)
    # a population larger than the static scratch is refused with a clear message
    rc = lib.dsps_photometry_fp32_static(ctx.handle, 10_000_000, ctypes.c_void_p(d_p.data_ptr()), sid,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == dsps.DSPS_ERR_INVALID_ARG
    assert b"static scratch" in lib.dsps_last_error_message()
    assert ctx.device_error() == 0
    ctx.close()
