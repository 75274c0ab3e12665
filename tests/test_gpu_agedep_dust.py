"""Parity of age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp: each age bin
attenuated with Av and delta moving from young-star to old-star values along
T_erf in log age) between the CUDA path and the FP64 oracle: magnitudes and
gradients (rows 11, 12 = Av_old, delta_old) in both precision forms, the
equal-values limit, batch invariance and the request loop; spectra and the
emission-line width with its gradient."""
import functools

import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {"birthcloud": dict(x0=7.0, h=0.1, law=0, bump=0), "wide_salim": dict(x0=8.0, h=0.3, law=1, bump=1)}


def _ctx(case, **kw):
    from paper_2112_06830_gb300 import dsps
    c = CASES[case]
    return dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True, dust_agedep_x0=c["x0"],
                        dust_agedep_h=c["h"], dust_law=c["law"], dust_bump=bool(c["bump"]), **kw)


def _ogrid(case):
    c = CASES[case]
    g = _util.ssp("full")
    return oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=1, dust_x0=c["x0"], dust_h=c["h"],
                       dust_law=c["law"], dust_bump=c["bump"])


@pytest.fixture(scope="module", params=list(CASES))
def agedep(request):
    c = _ctx(request.param)
    f = synth.make_filters(12)
    yield request.param, c, c.add_filters(f), oracle.Filters(f), _ogrid(request.param)
    c.close()


def _pop(n, seed, start=0):
    p = synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start), seed, start)
    return _util.params_f32(p)


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_photometry_matches_oracle(agedep, prec, tol):
    case, ctx, sid, F, grid = agedep
    assert (ctx.npar, ctx.ngrad) == (14, 13)
    p32, p64 = _pop(400, 61)
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
    idx = np.r_[0:8, 200:206, 390:400]
    ref = oracle.mags(grid, F, p64[:, idx])
    err = np.abs(m[idx] - ref)
    print(f"age-dependent dust {case} prec={prec}: max |dm| = {err.max():.3e}")
    assert err.max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_oracle(agedep, prec):
    case, ctx, sid, F, grid = agedep
    n = 160
    p32, p64 = _pop(n, 62, 700)
    mbar = np.random.default_rng(8).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    assert pb.shape == (13, n)
    idx = np.r_[0:6, 128:134, 154:160]
    _, ref = oracle.mags_vjp(grid, F, p64[:, idx], mbar[idx])
    floor = {0: 1e-3, 1: 1e-2}[prec]
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb[:, idx] - ref) / scale
    where = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"age-dependent dust {case} prec={prec}: max scaled gradient error {rel.max():.2e} at {where}")
    assert rel.max() <= 1e-3


def test_equal_young_and_old_values_match_one_curve():
    from paper_2112_06830_gb300 import dsps
    ctx = _ctx("birthcloud")
    plain = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH)
    f = synth.make_filters(12)
    s1, s0 = ctx.add_filters(f), plain.add_filters(f)
    p32, _ = _pop(300, 63)
    p32[12], p32[13] = p32[8], p32[9]
    p = torch.from_numpy(p32).cuda()
    mb = torch.from_numpy(np.random.default_rng(9).standard_normal((300, 12)).astype(np.float32)).cuda()
    for prec, tol in ((0, 2e-5), (1, 2e-4)):
        m1, g1 = ctx.photometry_vjp(p, s1, mb, precision=prec)
        m0, g0 = plain.photometry_vjp(p[:12].contiguous(), s0, mb, precision=prec)
        assert (m1 - m0).abs().max().item() <= tol
        gsum = g1[:11].clone()
        gsum[8] += g1[11]
        gsum[9] += g1[12]
        scale = torch.clamp(g0.abs(), min=1e-3 * g0.abs().max().item())
        assert ((gsum - g0).abs() / scale).max().item() <= 2e-3
    ctx.close()
    plain.close()


def test_batch_invariance_and_request_loop():
    from paper_2112_06830_gb300 import dsps
    big, small = _ctx("birthcloud"), _ctx("birthcloud", max_chunk=256)
    f = synth.make_filters(8)
    sb, ss = big.add_filters(f), small.add_filters(f)
    p32, _ = _pop(900, 64)
    p = torch.from_numpy(p32).cuda()
    mb = np.random.default_rng(10).standard_normal((900, 8)).astype(np.float32)
    for prec in (0, 1):
        m1, g1 = big.photometry_vjp(p, sb, torch.from_numpy(mb).cuda(), precision=prec)
        m2, g2 = small.photometry_vjp(p, ss, torch.from_numpy(mb).cuda(), precision=prec)
        assert torch.equal(m1, m2) and torch.equal(g1, g2)
        # the forward sums the groups' attenuated spectra on chip (one
        # launch), the gradient path sums per-group fluxes: the same terms in
        # another order
        fwd = big.photometry(p, sb, precision=prec)
        assert (fwd - m1).abs().max().item() <= (1e-5 if prec == 0 else 1e-4)
    t = big.submit(p32, sb, precision=1, mag_bar=mb)
    while big.poll(t, 100000) in (dsps.DSPS_PENDING, dsps.DSPS_ERR_TIMEOUT):
        pass
    m, g = big.photometry_vjp(p, sb, torch.from_numpy(mb).cuda(), precision=1)
    assert np.array_equal(t.mags, m.cpu().numpy()) and np.array_equal(t.param_bar, g.cpu().numpy())
    big.close()
    small.close()


def test_static_entry_is_refused(agedep):
    from paper_2112_06830_gb300 import dsps
    _, ctx, sid, _, _ = agedep
    p = torch.zeros((14, 4), device="cuda")
    out = torch.empty((4, 12), device="cuda")
    rc = dsps.load().dsps_photometry_fp32_static(ctx.handle, 4, p.data_ptr(), sid, out.data_ptr(), None)
    assert rc == dsps.DSPS_ERR_UNSUPPORTED


# ---- spectra and the line width (Sec. 2.2, Eq. eqw) under age-dependent dust ----
# Tolerances as in test_gpu_ew.py: the spectra's FP32 rounding (2e-5 relative),
# the width's 2e-5 (2 hw + |W|) A, and gradients within 1e-3 of max(|g|,
# 1e-2 max|g|).

LC, HW, CW = synth.EW_LINE


@functools.lru_cache(maxsize=None)
def _ssp_line():
    return synth.with_emission_line(_util.ssp("full"))


@pytest.fixture(scope="module", params=list(CASES))
def agedep_line(request):
    from paper_2112_06830_gb300 import dsps
    c = CASES[request.param]
    g = _ssp_line()
    ctx = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True, dust_agedep_x0=c["x0"],
                       dust_agedep_h=c["h"], dust_law=c["law"], dust_bump=bool(c["bump"]))
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=1, dust_x0=c["x0"], dust_h=c["h"],
                       dust_law=c["law"], dust_bump=c["bump"])
    yield request.param, ctx, ctx.add_line(LC, HW, CW), grid
    ctx.close()


def _line_pop(n, seed, start=0):
    p = synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start), seed, start)
    return _util.params_f32(p)


def test_spectra_match_oracle(agedep_line):
    case, ctx, _, grid = agedep_line
    p32, p64 = _line_pop(150, 81)
    n0, n1 = 1703, 2891   # ragged at both ends
    s = ctx.spectra(torch.from_numpy(p32).cuda(), n0, n1).cpu().numpy().astype(np.float64)
    ref = oracle.spectra(grid, p64[:, ::10])[:, n0:n1]
    rel = np.abs(s[::10] - ref) / ref
    print(f"age-dependent dust {case} spectra: max relative error {rel.max():.2e}")
    assert rel.max() <= 2e-5


def test_line_width_matches_oracle(agedep_line):
    case, ctx, lid, grid = agedep_line
    n = 600
    p32, p64 = _line_pop(n, 82)
    ew = ctx.line_ew(torch.from_numpy(p32).cuda(), lid).cpu().numpy().astype(np.float64)
    idx = np.r_[0:8, 128:136, 590:600]
    ref = oracle.line_ew(grid, p64[:, idx], LC, HW, CW)
    err = np.abs(ew[idx] - ref)
    print(f"age-dependent dust {case} EW: max |dW| = {err.max():.3e} A (W in [{ref.min():.1f}, {ref.max():.1f}])")
    assert np.all(err <= 2e-5 * (2 * HW + np.abs(ref)))


def test_line_width_gradient_matches_oracle(agedep_line):
    case, ctx, lid, grid = agedep_line
    n = 150
    p32, p64 = _line_pop(n, 83, 400)
    eb = np.random.default_rng(12).standard_normal(n)
    ew, pb = ctx.line_ew_vjp(torch.from_numpy(p32).cuda(), lid, torch.from_numpy(eb.astype(np.float32)).cuda())
    pb = pb.cpu().numpy().astype(np.float64)
    assert pb.shape == (13, n)
    idx = np.r_[0:10, 128:140, 140:150]
    ref_ew, ref = oracle.line_ew_vjp(grid, p64[:, idx], eb[idx], LC, HW, CW)
    assert np.all(np.abs(ew.cpu().numpy()[idx] - ref_ew) <= 2e-5 * (2 * HW + np.abs(ref_ew)))
    assert np.all(pb[10] == 0.0)    # the mass cancels in W
    rows = [r for r in range(13) if r != 10]
    g, r = pb[rows][:, idx], ref[rows]
    scale = np.maximum(np.abs(r), 1e-2 * np.abs(r).max(axis=0, keepdims=True))
    rel = np.abs(g - r) / scale
    where = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"age-dependent dust {case} EW gradient: max scaled error {rel.max():.2e} at {where}")
    assert rel.max() <= 1e-3


def test_line_width_chunk_invariance_and_forward_agreement():
    from paper_2112_06830_gb300 import dsps
    c = CASES["birthcloud"]
    kw = dict(sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True, dust_agedep_x0=c["x0"], dust_agedep_h=c["h"])
    big, small = dsps.Context(_ssp_line(), **kw), dsps.Context(_ssp_line(), max_chunk=256, **kw)
    lb, ls = big.add_line(LC, HW, CW), small.add_line(LC, HW, CW)
    p32, _ = _line_pop(500, 84)
    p = torch.from_numpy(p32).cuda()
    eb = torch.linspace(-1, 1, 500, device="cuda")
    e1, g1 = big.line_ew_vjp(p, lb, eb)
    e2, g2 = small.line_ew_vjp(p, ls, eb)
    assert torch.equal(e1, e2) and torch.equal(g1, g2)
    assert torch.equal(big.line_ew(p, lb), e1)
    assert torch.equal(big.spectra(p, 100, 900), small.spectra(p, 100, 900))
    big.close()
    small.close()


def test_skipping_is_exact_with_one_age_groups():
    """With tile skipping the one-age groups write only the K blocks of their
    age (the blocks the masked contraction reads); without it every weight is
    written and every block contracted.  The magnitudes keep every bit."""
    from paper_2112_06830_gb300 import dsps
    skip, dense = _ctx("birthcloud"), _ctx("birthcloud", band_skip=False)
    f = synth.make_filters(12)
    s1, s0 = skip.add_filters(f), dense.add_filters(f)
    p32, _ = _pop(700, 65)
    # invalid galaxies among them (a NaN row, a redshift out of range, no
    # formation time): NaN on both sides, through the cached age fractions too
    p32[10, 5] = np.nan
    p32[11, 300] = -1.0
    p32[0, 650] = 0.0
    p = torch.from_numpy(p32).cuda()
    mb = torch.from_numpy(np.random.default_rng(15).standard_normal((700, 12)).astype(np.float32)).cuda()
    mb[[5, 300, 650]] = 0.0
    m1 = skip.photometry(p, s1, precision=dsps.DSPS_PREC_BF16X3)
    m0 = dense.photometry(p, s0, precision=dsps.DSPS_PREC_BF16X3)
    assert np.array_equal(m1.cpu().numpy(), m0.cpu().numpy(), equal_nan=True)
    bad = torch.isnan(m1).all(dim=1)
    assert bad[[5, 300, 650]].all() and int(bad.sum()) == 3
    skip.device_error()
    dense.device_error()
    keep = ~bad
    g1 = skip.photometry_vjp(p, s1, mb, precision=dsps.DSPS_PREC_BF16X3)[1]
    g0 = dense.photometry_vjp(p, s0, mb, precision=dsps.DSPS_PREC_BF16X3)[1]
    # (the adjoint's own band skipping need not keep every bit; a stale block
    # would show as an O(1) error)
    g1, g0 = g1[:, keep], g0[:, keep]
    assert ((g1 - g0).abs() <= 1e-5 * g0.abs().amax(dim=0, keepdim=True)).all()
    skip.device_error()
    dense.device_error()
    skip.close()
    dense.close()


# ---------------------------------------------------------------- fused groups

PRECS = {1: (_util.TOL_BF16X3, 1e-4), 0: (_util.TOL_FP32, 1e-5)}   # oracle tolerance, fused vs per-group


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("case", list(CASES))
def test_fused_groups_match_per_group_launches_and_oracle(case, prec):
    """The forward that contracts every dust group in one launch (each
    group's attenuated spectrum summed on chip -- in TMEM-fed registers for
    split-bf16, in registers beside the FP32 accumulators -- then one filter
    integral) against one launch per group, and against the oracle: the two
    GPU forms differ only in summation order."""
    tol, tol_pg = PRECS[prec]
    f = synth.make_filters(12)
    a = _ctx(case)
    b = _ctx(case, agedep_fused=False)
    sa, sb = a.add_filters(f), b.add_filters(f)
    for n, start in ((1, 0), (129, 300), (3000, 5000)):
        p32, p64 = _pop(n, 63, start)
        x = torch.from_numpy(p32).cuda()
        ma = a.photometry(x, sa, precision=prec).cpu().numpy().astype(np.float64)
        mb = b.photometry(x, sb, precision=prec).cpu().numpy().astype(np.float64)
        d = np.abs(ma - mb).max()
        idx = np.unique(np.r_[0, n - 1, np.arange(0, n, max(1, n // 17))])
        ref = oracle.mags(_ogrid(case), oracle.Filters(f), np.ascontiguousarray(p64[:, idx]))
        err = np.abs(ma[idx] - ref).max()
        print(f"{case} prec={prec} n={n}: fused vs per-group {d:.2e}, fused vs oracle {err:.2e}")
        assert np.isfinite(ma).all()
        assert d <= tol_pg
        assert err <= tol
    assert a.device_error() == 0 and b.device_error() == 0
    a.close()
    b.close()


@pytest.mark.parametrize("prec", list(PRECS))
def test_fused_groups_batch_invariance_and_chunks(prec):
    """A galaxy's magnitudes do not depend on the batch it rides in, nor on how
    the call is cut into chunks (fixed-order sums)."""
    f = synth.make_filters(8)
    a = _ctx("birthcloud")
    small = _ctx("birthcloud", max_chunk=256)
    sa, ss = a.add_filters(f), small.add_filters(f)
    p32, _ = _pop(900, 64, 20_000)
    whole = a.photometry(torch.from_numpy(p32).cuda(), sa, precision=prec).cpu().numpy()
    part = a.photometry(torch.from_numpy(np.ascontiguousarray(p32[:, 400:437])).cuda(), sa,
                        precision=prec).cpu().numpy()
    np.testing.assert_array_equal(whole[400:437], part)
    chunked = small.photometry(torch.from_numpy(p32).cuda(), ss, precision=prec).cpu().numpy()
    np.testing.assert_array_equal(whole, chunked)
    assert a.device_error() == 0
    a.close()
    small.close()


@pytest.mark.parametrize("prec", list(PRECS))
def test_fused_groups_extreme_transitions_and_invalid_rows(prec):
    """Transitions beyond both ends of the age grid (one group of all ages with
    T = 0 or T = 1) and a wide one, with invalid galaxies among the rows: NaN
    where the parameters are out of range, the oracle elsewhere."""
    from paper_2112_06830_gb300 import dsps
    tol = PRECS[prec][0]
    f = synth.make_filters(6)
    g = _util.ssp("full")
    for x0, h in ((4.0, 0.1), (12.0, 0.1), (8.5, 1.5)):
        ctx = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True, dust_agedep_x0=x0, dust_agedep_h=h)
        sid = ctx.add_filters(f)
        p = synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, 200, 65), 65)
        p[11, 7] = -1.0
        p[6, 50] = 0.0
        p32, p64 = _util.params_f32(p)
        m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
        assert np.isnan(m[[7, 50]]).all()
        idx = np.array([0, 1, 100, 199])
        og = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                         sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=1, dust_x0=x0, dust_h=h)
        ref = oracle.mags(og, oracle.Filters(f), np.ascontiguousarray(p64[:, idx]))
        err = np.abs(m[idx] - ref).max()
        print(f"x0={x0} h={h} prec={prec}: max |dm| vs oracle {err:.2e}")
        assert err <= tol
        assert ctx.device_error() == dsps.DSPS_ERR_INVALID_ARG
        ctx.close()


@pytest.mark.parametrize("x0,h", [(7.0, 0.1), (8.0, 0.3), (4.0, 0.1), (12.0, 0.1), (8.5, 1.5)])
def test_fused_gradient_matches_per_group_gradient(x0, h):
    """The split-bf16 gradient whose fluxes and dust rows come from the
    one-launch contraction (a forward and a gradient pass) against the one
    that runs a gradient-mode contraction per dust group: the same terms in
    another summation order.  Transitions inside the grid and beyond both ends
    (one group of every age, T = 0 or 1) and a wide one."""
    from paper_2112_06830_gb300 import dsps
    f = synth.make_filters(8)
    g = _util.ssp("full")
    kw = dict(sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True, dust_agedep_x0=x0, dust_agedep_h=h)
    a = dsps.Context(g, **kw)
    b = dsps.Context(g, agedep_fused=False, **kw)
    sa, sb = a.add_filters(f), b.add_filters(f)
    p32, _ = _pop(700, 66, 1000)
    p = torch.from_numpy(p32).cuda()
    mb = torch.from_numpy(np.random.default_rng(13).standard_normal((700, 8)).astype(np.float32)).cuda()
    ma, ga = a.photometry_vjp(p, sa, mb, precision=dsps.DSPS_PREC_BF16X3)
    mbb, gb = b.photometry_vjp(p, sb, mb, precision=dsps.DSPS_PREC_BF16X3)
    dm = (ma - mbb).abs().max().item()
    scale = torch.clamp(gb.abs(), min=1e-3 * gb.abs().amax(dim=0, keepdim=True))
    rel = ((ga - gb).abs() / scale).max().item()
    print(f"x0={x0} h={h}: fused vs per-group |dm| {dm:.2e}, scaled gradient difference {rel:.2e}")
    assert torch.isfinite(ga).all() and dm <= 1e-4 and rel <= 2e-3
    assert a.device_error() == 0 and b.device_error() == 0
    a.close()
    b.close()
