"""Parity of rest-frame absolute magnitudes (Sec. 2.2, Eq. restmag: filters at
the rest wavelength, no distance terms) between the CUDA path and the FP64
oracle: magnitudes and gradients in both precision forms over several tiles
and a ragged tail, observer and rest-frame sets side by side in one context,
age-dependent dust, batch invariance, the request loop and the
allocation-free entry."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TABLES = synth.make_filters(12)   # 3500-9000 A, FWHM 800 A


@pytest.fixture(scope="module")
def frames():
    from paper_2112_06830_gb300 import dsps
    ctx = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH)
    yield ctx, ctx.add_filters(TABLES, rest_frame=True), ctx.add_filters(TABLES)
    ctx.close()


def _pop(n, seed, start=0):
    return _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start))


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_rest_and_observer_sets_match_the_oracle(frames, prec, tol):
    ctx, rest, obs = frames
    p32, p64 = _pop(700, 31)
    d = torch.from_numpy(p32).cuda()
    idx = np.r_[0:6, 300:306, 690:700]
    grid = _util.oracle_grid("full", synth.SFH_DPL_QUENCH)
    for sid, F in ((rest, oracle.Filters(TABLES, rest=True)), (obs, oracle.Filters(TABLES))):
        m = ctx.photometry(d, sid, precision=prec).cpu().numpy().astype(np.float64)
        ref = oracle.mags(grid, F, p64[:, idx])
        err = np.abs(m[idx] - ref).max()
        print(f"{'rest' if F.rest else 'observer'} frame prec={prec}: max |dm| = {err:.3e}")
        assert err <= tol
    # rest-frame magnitudes are absolute: far brighter than apparent ones
    mr = ctx.photometry(d, rest, precision=prec)
    mo = ctx.photometry(d, obs, precision=prec)
    assert (mo - mr).min().item() > 30.0


@pytest.mark.parametrize("prec", [0, 1])
def test_rest_frame_gradients_match_the_oracle(frames, prec):
    ctx, rest, _ = frames
    n = 150
    p32, p64 = _pop(n, 32, 500)
    mbar = np.random.default_rng(6).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), rest, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    idx = np.r_[0:6, 128:134, 144:150]
    _, ref = oracle.mags_vjp(_util.oracle_grid("full", synth.SFH_DPL_QUENCH), oracle.Filters(TABLES, rest=True),
                             p64[:, idx], mbar[idx])
    floor = {0: 1e-3, 1: 1e-2}[prec]
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb[:, idx] - ref) / scale
    print(f"rest frame prec={prec}: max scaled gradient error {rel.max():.2e}")
    assert rel.max() <= 1e-3


def test_rest_frame_with_age_dependent_dust():
    from paper_2112_06830_gb300 import dsps
    g = _util.ssp("full")
    ctx = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True)
    sid = ctx.add_filters(TABLES, rest_frame=True)
    p = synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, 300, 33), 33)
    p32, p64 = _util.params_f32(p)
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=1)
    idx = np.r_[0:5, 295:300]
    ref = oracle.mags(grid, oracle.Filters(TABLES, rest=True), p64[:, idx])
    for prec, tol in ((0, _util.TOL_FP32), (1, _util.TOL_BF16X3)):
        m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy()
        assert np.abs(m[idx] - ref).max() <= tol
    ctx.close()


def test_batch_invariance_request_loop_and_static_entry(frames):
    from paper_2112_06830_gb300 import dsps
    ctx, rest, _ = frames
    small = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH, max_chunk=256)
    rest_s = small.add_filters(TABLES, rest_frame=True)
    p32, _ = _pop(600, 34)
    p = torch.from_numpy(p32).cuda()
    mb = np.random.default_rng(7).standard_normal((600, 12)).astype(np.float32)
    for prec in (0, 1):
        m1, g1 = ctx.photometry_vjp(p, rest, torch.from_numpy(mb).cuda(), precision=prec)
        m2, g2 = small.photometry_vjp(p, rest_s, torch.from_numpy(mb).cuda(), precision=prec)
        assert torch.equal(m1, m2) and torch.equal(g1, g2)
    t = ctx.submit(p32, rest, precision=1, mag_bar=mb)
    while ctx.poll(t, 100000) in (dsps.DSPS_PENDING, dsps.DSPS_ERR_TIMEOUT):
        pass
    m, g = ctx.photometry_vjp(p, rest, torch.from_numpy(mb).cuda(), precision=1)
    assert np.array_equal(t.mags, m.cpu().numpy()) and np.array_equal(t.param_bar, g.cpu().numpy())
    out = torch.full((600, 12), float("nan"), device="cuda")
    lib = dsps.load()
    rc = lib.dsps_photometry_fp32_static(ctx.handle, 600, ctypes.c_void_p(p.data_ptr()), rest,
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == dsps.DSPS_OK, lib.dsps_last_error_message()
    want = ctx.photometry(p, rest, precision=dsps.DSPS_PREC_FP32)
    assert (out - want).abs().max().item() <= _util.TOL_FP32
    with pytest.raises(dsps.DSPSError):
        dsps.dsps_filters_add(ctx.handle, TABLES, 7)
    small.close()
