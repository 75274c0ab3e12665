"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Tolerances: 1e-4 mag for the FP32 contraction, 1e-3 mag for
the split-bf16 tensor-core contraction; weights to 2e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PREC = {"fp32": (0, _util.TOL_FP32), "bf16x3": (1, _util.TOL_BF16X3)}


def _ctx(kind, sfh_model, mdf_kernel=0, **kw):
    from paper_2112_06830_gb300 import dsps
    return dsps.Context(_util.ssp(kind), sfh_model=sfh_model, mdf_kernel=mdf_kernel, **kw)


@pytest.fixture(scope="module")
def small():
    c = _ctx("small", synth.SFH_DELAYED_TAU)
    f = synth.make_filters(6)
    return c, c.add_filters(f), oracle.Filters(f)


@pytest.fixture(scope="module")
def full():
    c = _ctx("full", synth.SFH_DPL_QUENCH)
    f = synth.make_filters(12)
    return c, c.add_filters(f), oracle.Filters(f)


def _run(ctx, sid, p32, prec):
    out = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_weights_match_oracle_small(small):
    ctx, _, _ = small
    p32, p64 = _util.params_f32(synth.make_population(synth.SFH_DELAYED_TAU, 64, 0))
    w = ctx.weights(torch.from_numpy(p32).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.weights(_util.oracle_grid("small", 0), p64)
    mass = 10.0 ** p64[10]
    err = np.abs(w - ref)
    assert (err <= 2e-5 * np.abs(ref) + 1e-6 * mass[:, None, None]).all(), err.max()
    np.testing.assert_allclose(w.sum(axis=(1, 2)), mass, rtol=1e-5)


@pytest.mark.parametrize("model,kernel", [(1, 0), (1, 1)])
def test_weights_match_oracle_full(full, model, kernel):
    ctx = _ctx("full", model, kernel) if kernel else full[0]
    p32, p64 = _util.params_f32(synth.make_population(model, 37, 9))
    w = ctx.weights(torch.from_numpy(p32).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.weights(_util.oracle_grid("full", model, kernel), p64)
    mass = 10.0 ** p64[10]
    err = np.abs(w - ref)
    assert (err <= 2e-5 * np.abs(ref) + 1e-6 * mass[:, None, None]).all(), err.max()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_photometry_small_matches_oracle(small, prec):
    ctx, sid, F = small
    p32, p64 = _util.params_f32(synth.make_population(synth.SFH_DELAYED_TAU, 64, 0))
    m = _run(ctx, sid, p32, PREC[prec][0])
    ref = oracle.mags(_util.oracle_grid("small", 0), F, p64)
    err = np.abs(m - ref)
    print(f"small {prec}: max |dm| = {err.max():.3e}, p99 = {np.quantile(err, 0.99):.3e}")
    assert err.max() <= PREC[prec][1]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("n", [1, 129, 300])
def test_photometry_full_grid_ragged(full, prec, n):
    ctx, sid, F = full
    p32, p64 = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, n, 1, start=1000))
    m = _run(ctx, sid, p32, PREC[prec][0])
    ref = oracle.mags(_util.oracle_grid("full", 1), F, p64)
    err = np.abs(m - ref)
    print(f"full n={n} {prec}: max |dm| = {err.max():.3e}, p99 = {np.quantile(err, 0.99):.3e}")
    assert err.max() <= PREC[prec][1]


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_photometry_full_size_sampled(full, prec):
    """The 1e5-galaxy workload in the bench's launch configuration; the oracle
    checks a sample of 48 galaxies spread over the batch (first and last
    included)."""
    ctx, sid, F = full
    G = 100_000
    p32, p64 = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, G, 1))
    m = _run(ctx, sid, p32, PREC[prec][0])
    idx = np.unique(np.concatenate([[0, G - 1], np.random.default_rng(5).integers(0, G, 46)]))
    ref = oracle.mags(_util.oracle_grid("full", 1), F, p64[:, idx])
    err = np.abs(m[idx] - ref)
    print(f"full 1e5 {prec}: sampled max |dm| = {err.max():.3e}")
    assert err.max() <= PREC[prec][1]
    assert np.isfinite(m).all()


@pytest.mark.parametrize("prec", [0, 1])
def test_results_do_not_depend_on_the_batch(full, prec):
    ctx, sid, _ = full
    p32, _ = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, 700, 1, start=5000))
    whole = _run(ctx, sid, p32, prec)
    part = _run(ctx, sid, np.ascontiguousarray(p32[:, 300:333]), prec)
    np.testing.assert_array_equal(whole[300:333], part)


@pytest.mark.parametrize("prec", [0, 1])
def test_chunked_launches_equal_one_launch(prec):
    ctx = _ctx("small", synth.SFH_DELAYED_TAU, max_chunk=128)
    f = synth.make_filters(6)
    sid = ctx.add_filters(f)
    p32, _ = _util.params_f32(synth.make_population(synth.SFH_DELAYED_TAU, 333, 3))
    a = _run(ctx, sid, p32, prec)
    ctx1 = _ctx("small", synth.SFH_DELAYED_TAU)
    sid1 = ctx1.add_filters(f)
    b = _run(ctx1, sid1, p32, prec)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_edge_redshifts_and_filter_counts(full, prec):
    """z near 0 and at the top of the range (filters partly off the rest grid),
    Av = 0, one-filter and sixteen-filter sets."""
    ctx, _, _ = full
    p = synth.make_population(synth.SFH_DPL_QUENCH, 6, 8)
    p[11] = [1e-3, 0.02, 1.0, 2.9, 3.0, 6.0]
    p[8, 0] = 0.0
    p32, p64 = _util.params_f32(p)
    for tables in (synth.make_filters(1), synth.make_filters(16, 3300.0, 11000.0)):
        sid = ctx.add_filters(tables)
        m = _run(ctx, sid, p32, PREC[prec][0])
        ref = oracle.mags(_util.oracle_grid("full", 1), oracle.Filters(tables), p64)
        fin = np.isfinite(ref)
        assert (np.isfinite(m) == fin).all()
        # A band whose centre maps blueward of the rest grid is sampled only in
        # the filter's far tail; there the filter resampled on the ln(lambda)
        # grid differs from the oracle's linear-in-lambda table by
        # (dlam^2/8) |T''/T| ~ (5 A)^2/8 * ((lam-c)^2/s^4) ~ 2e-3 at T ~ 1e-15
        # of peak (lam - c = 2800 A, s = 340 A).  Those bands get that bound.
        centres = np.array([np.sum(l * t) / np.sum(t) for l, t in tables])
        tail = (1.0 + p64[11])[:, None] * _util.ssp("full").lam[0] > centres[None, :]
        tol = np.where(tail, 5e-3, PREC[prec][1])
        err = np.abs(m - ref)
        assert (err[fin] <= tol[fin]).all(), err[fin].max()


def test_invalid_parameters_give_nan_and_error(small):
    from paper_2112_06830_gb300 import dsps
    ctx, sid, _ = small
    assert ctx.device_error() == 0
    p = synth.make_population(synth.SFH_DELAYED_TAU, 5, 4)
    p[11, 1] = -0.5      # negative redshift
    p[6, 3] = 0.0        # zero MDF width
    p32, _ = _util.params_f32(p)
    m = _run(ctx, sid, p32, 0)
    assert np.isnan(m[1]).all() and np.isnan(m[3]).all()
    assert np.isfinite(m[[0, 2, 4]]).all()
    assert ctx.device_error() == dsps.DSPS_ERR_INVALID_ARG
    assert ctx.device_error() == 0


def test_empty_batch(small):
    ctx, sid, _ = small
    out = ctx.photometry(torch.zeros((12, 0), dtype=torch.float32, device="cuda"), sid)
    assert out.shape == (0, 6)


def test_band_skipping_is_exact(full):
    """Skipping wavelength tiles outside every redshifted filter changes no bit."""
    ctx, sid, _ = full
    dense = _ctx("full", synth.SFH_DPL_QUENCH, band_skip=False)
    sid_d = dense.add_filters(synth.make_filters(12))
    p32, _ = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, 1500, 1, start=20_000))
    np.testing.assert_array_equal(_run(ctx, sid, p32, 1), _run(dense, sid_d, p32, 1))


def test_young_bins_keep_relative_precision(full):
    """Quenched galaxies observed after t_q: the youngest age bins hold ~1e-8 of
    the formed mass; the GPU must still get them to 1e-4 relative."""
    ctx = full[0]
    p = synth.make_population(synth.SFH_DPL_QUENCH, 24, 17)
    p[3] = 5.0          # quench early
    p[4] = 3.0          # by 3 dex
    p[11] = np.linspace(0.01, 0.4, 24)
    p32, p64 = _util.params_f32(p)
    w = ctx.weights(torch.from_numpy(p32).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.weights(_util.oracle_grid("full", 1), p64)
    mass = (10.0 ** p64[10])[:, None, None]
    # age-bin masses (summed over metallicity): the SFH part alone
    wa, ra = w.sum(axis=2), ref.sum(axis=2)
    big = ra > 1e-12 * mass[:, :, 0]
    rel = np.abs(wa - ra)[big] / ra[big]
    assert rel.max() <= 1e-4, rel.max()
    assert (ra[:, 0] / mass[:, 0, 0] < 1e-5).all()   # the youngest bin is tiny indeed
    # joint weights, including the triweight tails of the MDF
    big = ref > 1e-8 * mass
    rel = np.abs(w - ref)[big] / ref[big]
    assert rel.max() <= 3e-4, rel.max()


@pytest.mark.parametrize("kernel", [0, 1])
def test_metallicity_block_skipping_is_exact(kernel):
    """Skipping K blocks where every row of a tile has zero weight (metallicity-
    major K, tiles sorted by mean metallicity) changes no bit, for MDF widths
    from 0.01 dex (one or two non-zero metallicity bins) to 1.5 dex (all bins),
    steep age slopes, and means beyond both ends of the lgZ grid."""
    f = synth.make_filters(12)
    skip = _ctx("full", synth.SFH_DPL_QUENCH, mdf_kernel=kernel)
    dense = _ctx("full", synth.SFH_DPL_QUENCH, mdf_kernel=kernel, band_skip=False)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 2000, 11, start=40_000)
    rng = np.random.default_rng(5)
    p[6] = np.exp(rng.uniform(np.log(0.01), np.log(1.5), p.shape[1]))
    p[5] = rng.uniform(-2.6, 0.9, p.shape[1])
    p[7] = rng.uniform(-0.6, 0.6, p.shape[1])
    p32, p64 = _util.params_f32(p)
    a = _run(skip, skip.add_filters(f), p32, 1)
    b = _run(dense, dense.add_filters(f), p32, 1)
    np.testing.assert_array_equal(a, b)
    idx = np.arange(0, 2000, 97)
    ref = oracle.mags(_util.oracle_grid("full", 1, kernel), oracle.Filters(f), np.ascontiguousarray(p64[:, idx]))
    assert np.abs(a[idx] - ref).max() <= _util.TOL_BF16X3


def test_block_skipping_removes_work(full):
    """The tensor-core kernel executes well under the dense count of block
    products on the standard population (exact skipping of zero K blocks and
    of wavelength tiles outside the filter band)."""
    from paper_2112_06830_gb300 import dsps
    ctx, sid, _ = full
    n = 20_000
    p32, _ = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, n, 1))
    x = torch.from_numpy(p32).cuda()
    ctx.photometry(x, sid, precision=1)
    torch.cuda.synchronize()
    dsps.dsps_profile_enable(ctx.handle, True)
    ctx.photometry(x, sid, precision=1)
    torch.cuda.synchronize()
    prof = dsps.dsps_profile_read(ctx.handle)
    dsps.dsps_profile_enable(ctx.handle, False)
    g = _util.ssp("full")
    a_pad = -(-g.l_ssp.shape[0] // 4) * 4          # metallicity-major K: ages padded to 4
    kz_pad = -(-g.l_ssp.shape[1] * a_pad // 64) * 64
    N_pad = -(-(g.l_ssp.shape[2] + 1) // 256) * 256
    dense_blocks = -(-n // 128) * (N_pad // 256) * (kz_pad // 32)
    frac = prof["tc_kblocks"] / dense_blocks
    print(f"executed {prof['tc_kblocks']} of {dense_blocks} block products ({frac:.3f})")
    assert 0 < frac < 0.30
    assert prof["simt_steps"] == 0
    # the FP32 form counts its 128 x 128 x 16 tile steps: each tile's band only
    dsps.dsps_profile_enable(ctx.handle, True)
    ctx.photometry(x, sid, precision=0)
    torch.cuda.synchronize()
    prof = dsps.dsps_profile_read(ctx.handle)
    dsps.dsps_profile_enable(ctx.handle, False)
    k_pad = -(-g.l_ssp.shape[0] * g.l_ssp.shape[1] // 64) * 64
    dense_steps = -(-n // 128) * (N_pad // 128) * (k_pad // 16)
    frac32 = prof["simt_steps"] / dense_steps
    print(f"FP32 form: {prof['simt_steps']} of {dense_steps} tile steps ({frac32:.3f})")
    assert prof["tc_kblocks"] == 0 and 0 < frac32 < 0.6


def test_million_galaxy_precision_forms(full):
    """10^6 galaxies of the full workload in both forms; per-galaxy magnitude
    error against the oracle on a 10^3-galaxy subsample (every 1000th
    galaxy), and the split-bf16 form against FP32 on all of them."""
    ctx, sid, F = full
    n = 1_000_000
    p32, p64 = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, n, 1))
    x = torch.from_numpy(p32).cuda()
    m_tc = ctx.photometry(x, sid, precision=1)
    m_32 = ctx.photometry(x, sid, precision=0)
    torch.cuda.synchronize()
    m_tc, m_32 = m_tc.cpu().numpy().astype(np.float64), m_32.cpu().numpy().astype(np.float64)
    idx = np.arange(0, n, 1000)
    ref = oracle.mags(_util.oracle_grid("full", 1), F, np.ascontiguousarray(p64[:, idx]))
    e_tc = np.abs(m_tc[idx] - ref).max(axis=1)
    e_32 = np.abs(m_32[idx] - ref).max(axis=1)
    d = np.abs(m_tc - m_32)
    print(f"1e6 galaxies: per-galaxy max |dm| vs oracle on 1e3: bf16x3 max {e_tc.max():.2e} "
          f"p50 {np.median(e_tc):.2e}; fp32 max {e_32.max():.2e} p50 {np.median(e_32):.2e}; "
          f"bf16x3 - fp32 over 1e6: max {d.max():.2e} p99 {np.percentile(d, 99):.2e}")
    assert np.isfinite(m_tc).all() and np.isfinite(m_32).all()
    assert e_tc.max() <= _util.TOL_BF16X3
    assert e_32.max() <= _util.TOL_FP32
    assert d.max() <= _util.TOL_BF16X3 + _util.TOL_FP32
