"""Parity of the nebular ionisation axis (Sec. 3.3, Eq. nebsed: a triweight
distribution of log U over a third SSP axis) between the CUDA path and the
FP64 oracle: SSP weights, magnitudes and gradients (rows 11, 12 = u_mean,
u_sigma) in both precision forms, the line width whose strength the axis
controls, and exactness of the per-tile log U section skipping."""
import functools

import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LC, HW, CW = synth.EW_LINE


@functools.lru_cache(maxsize=None)
def _ssp():
    return synth.make_ssp_nebular(synth.FULL_GRID, 1)


@functools.lru_cache(maxsize=None)
def _ogrid():
    g = _ssp()
    return oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, lgu=g.lgu)


@pytest.fixture(scope="module")
def neb():
    from paper_2112_06830_gb300 import dsps
    c = dsps.Context(_ssp(), sfh_model=synth.SFH_DPL_QUENCH, max_chunk=32768)
    f = synth.make_filters(12)
    yield c, c.add_filters(f), oracle.Filters(f)
    c.close()


def _pop(n, seed, start=0):
    p = synth.with_nebular(synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start), seed, start)
    return _util.params_f32(p)


def test_context_has_the_nebular_rows(neb):
    ctx, _, _ = neb
    assert (ctx.n_u, ctx.npar, ctx.ngrad) == (7, 14, 13)


def test_weights_match_oracle(neb):
    ctx, _, _ = neb
    p32, p64 = _pop(300, 41)
    w = ctx.weights(torch.from_numpy(p32).cuda()).cpu().numpy().astype(np.float64)
    idx = np.r_[0:6, 128:134, 290:300]
    ref = oracle.weights(_ogrid(), p64[:, idx])
    mass = 10.0 ** p64[10, idx]
    err = np.abs(w[idx] - ref) / (np.abs(ref) + 1e-6 * mass[:, None, None, None])
    print(f"nebular weights: max relative error {err.max():.2e}")
    assert err.max() <= 1e-4
    np.testing.assert_allclose(w[idx].sum(axis=(1, 2, 3)), mass, rtol=2e-5)


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_photometry_matches_oracle(neb, prec, tol):
    ctx, sid, F = neb
    p32, p64 = _pop(600, 42)
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
    idx = np.r_[0:10, 200:210, 590:600]
    ref = oracle.mags(_ogrid(), F, p64[:, idx])
    err = np.abs(m[idx] - ref)
    print(f"nebular prec={prec}: max |dm| = {err.max():.3e}")
    assert err.max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_oracle(neb, prec):
    ctx, sid, F = neb
    n = 200
    p32, p64 = _pop(n, 43, 512)
    mbar = np.random.default_rng(6).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    assert pb.shape == (13, n)
    idx = np.r_[0:8, 128:136, 192:200]
    _, ref = oracle.mags_vjp(_ogrid(), F, p64[:, idx], mbar[idx])
    floor = {0: 1e-3, 1: 1e-2}[prec]
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb[:, idx] - ref) / scale
    where = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"nebular prec={prec}: max scaled gradient error {rel.max():.2e} at {where}; "
          f"u_mean/u_sigma rows {rel[11:].max():.2e}")
    assert rel.max() <= 1e-3


def test_section_skipping_is_exact(neb):
    from paper_2112_06830_gb300 import dsps
    ctx, sid, _ = neb
    p32, _ = _pop(1000, 44)
    p = torch.from_numpy(p32).cuda()
    dense = dsps.Context(_ssp(), sfh_model=synth.SFH_DPL_QUENCH, max_chunk=32768, band_skip=False)
    sd = dense.add_filters(synth.make_filters(12))
    for prec in (0, 1):
        assert torch.equal(ctx.photometry(p, sid, precision=prec), dense.photometry(p, sd, precision=prec))
    dsps.dsps_profile_enable(ctx.handle, True)
    dsps.dsps_profile_read(ctx.handle)
    ctx.photometry(p, sid)
    skip = dsps.dsps_profile_read(ctx.handle)["tc_kblocks"]
    dsps.dsps_profile_enable(ctx.handle, False)
    dsps.dsps_profile_enable(dense.handle, True)
    dsps.dsps_profile_read(dense.handle)
    dense.photometry(p, sd)
    full = dsps.dsps_profile_read(dense.handle)["tc_kblocks"]
    print(f"nebular: executed {skip} of {full} dense block products ({skip / full:.3f})")
    assert skip < 0.5 * full
    dense.close()


def test_section_ranges_at_the_support_edges(neb):
    # Log U distributions whose support ends exactly on a section edge
    # (edges at the midpoints -3.75, -3.25, .., -1.25), very narrow and very
    # wide ones, means off the grid, and invalid log U rows among valid
    # galaxies: the skipping context equals the dense one bit for bit, and
    # the valid galaxies match the oracle.
    from paper_2112_06830_gb300 import dsps
    ctx, sid, F = neb
    n = 700
    p32, p64 = _pop(n, 45)
    cases = [(-2.5, 0.25), (-3.0, 0.25), (-2.25, 1e-3), (-3.25, 1e-6), (-2.5, 10.0),
             (-8.0, 0.25), (2.0, 0.25), (-1.0 - 0.75, 0.25), (np.nan, 0.25), (-2.5, 0.0), (-2.5, -0.1),
             (-2.5, np.inf)]
    for k, (um, us) in enumerate(cases):
        p32[12, k::len(cases)] = um
        p32[13, k::len(cases)] = us
    p64 = p32.astype(np.float64)
    bad = ~(np.isfinite(p64[12]) & np.isfinite(p64[13]) & (p64[13] > 0))
    d = torch.from_numpy(p32).cuda()
    dense = dsps.Context(_ssp(), sfh_model=synth.SFH_DPL_QUENCH, max_chunk=32768, band_skip=False)
    sd = dense.add_filters(synth.make_filters(12))
    for prec in (0, 1):
        a = ctx.photometry(d, sid, precision=prec).cpu().numpy()
        b = dense.photometry(d, sd, precision=prec).cpu().numpy()
        assert np.array_equal(a, b, equal_nan=True)
        assert np.all(np.isnan(a[bad])) and np.all(np.isfinite(a[~bad]))
    assert ctx.device_error() == dsps.DSPS_ERR_INVALID_ARG
    assert ctx.device_error() == 0
    # the adjoint contraction skips the column blocks outside each tile's log U
    # sections and the reference section: the same gradients as the dense path
    mbar = np.random.default_rng(17).standard_normal((n, 12))
    mb = torch.from_numpy(mbar.astype(np.float32)).cuda()
    _, ga = ctx.photometry_vjp(d, sid, mb, precision=1)
    _, gb = dense.photometry_vjp(d, sd, mb, precision=1)
    ga, gb = ga.cpu().numpy().astype(np.float64), gb.cpu().numpy().astype(np.float64)
    scale = np.abs(gb[:, ~bad]).max(axis=1, keepdims=True)
    assert np.abs(ga[:, ~bad] - gb[:, ~bad]).max(axis=1).max() <= 1e-5 * scale.max()
    assert (np.abs(ga[:, ~bad] - gb[:, ~bad]) <= 1e-5 * scale).all()
    ctx.device_error()
    dense.device_error()
    dense.close()
    idx = np.array([k for k in range(0, 96) if not bad[k]] + [n - 4, n - 3])
    idx = idx[~bad[idx]]
    ref = oracle.mags(_ogrid(), F, p64[:, idx])
    err = np.abs(a[idx].astype(np.float64) - ref).max()
    print(f"nebular support edges: max |dm| = {err:.2e} over {len(idx)} galaxies")
    assert err <= _util.TOL_BF16X3
    sub = idx[:24]
    _, gref = oracle.mags_vjp(_ogrid(), F, p64[:, sub], mbar[sub])
    sc = np.maximum(np.abs(gref), 1e-2 * np.abs(gref).max(axis=0, keepdims=True))
    rel = np.abs(ga[:, sub] - gref) / np.where(sc > 0, sc, 1.0)
    print(f"nebular support edges: max scaled gradient error {rel.max():.2e}")
    assert rel.max() <= 1e-3


def test_line_width_and_its_u_gradient(neb):
    ctx, _, _ = neb
    lid = ctx.add_line(LC, HW, CW)
    n = 64
    p32, p64 = _pop(n, 45)
    eb = np.ones(n)
    ew, pb = ctx.line_ew_vjp(torch.from_numpy(p32).cuda(), lid, torch.ones(n, device="cuda"))
    ew, pb = ew.cpu().numpy().astype(np.float64), pb.cpu().numpy().astype(np.float64)
    idx = np.r_[0:6, 58:64]
    ref_ew, ref = oracle.line_ew_vjp(_ogrid(), p64[:, idx], eb[idx], LC, HW, CW)
    assert np.all(np.abs(ew[idx] - ref_ew) <= 2e-5 * (2 * HW + np.abs(ref_ew)))
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb[:, idx] - ref) / scale
    print(f"nebular EW: max |dW| {np.abs(ew[idx] - ref_ew).max():.2e}, gradient {rel.max():.2e}")
    assert rel.max() <= 1e-3
    assert np.all(pb[11] > 0.0)        # [OIII] strengthens with the ionisation parameter


def test_request_loop_takes_the_nebular_rows(neb):
    ctx, sid, _ = neb
    p32, _ = _pop(700, 46)
    mb = np.random.default_rng(7).standard_normal((700, 12)).astype(np.float32)
    t = ctx.submit(p32, sid, precision=1, mag_bar=mb)
    from paper_2112_06830_gb300 import dsps
    while ctx.poll(t, 100000) in (dsps.DSPS_PENDING, dsps.DSPS_ERR_TIMEOUT):
        pass
    m, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mb).cuda(), precision=1)
    assert np.array_equal(t.mags, m.cpu().numpy())
    assert t.param_bar.shape == (13, 700)
    assert np.array_equal(t.param_bar, pb.cpu().numpy())
