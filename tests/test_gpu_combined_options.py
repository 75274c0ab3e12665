"""Every model option at once -- the nebular axis (Sec. 3.3), age-dependent dust
(Sec. 3.4.1) with the paper's attenuation law and the UV bump (Sec. 3.4), and
the T_erf age-dependent MDF (Sec. 3.2) -- against the FP64 oracle: the
parameter rows (16: nebular rows 12, 13, old-star dust rows 14, 15) and the
gradient rows (15: nebular 11, 12, old-star dust 13, 14) line up, and the
magnitudes and gradients agree in both precision forms."""
import functools

import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _ssp():
    return synth.make_ssp_nebular(synth.FULL_GRID, 1)


@pytest.fixture(scope="module")
def combo():
    from paper_2112_06830_gb300 import dsps
    g = _ssp()
    c = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH, max_chunk=16384, mdf_mean=dsps.DSPS_MDF_MEAN_TERF,
                     dust_bump=True, dust_law=dsps.DSPS_DUST_SALIM, dust_agedep=True, dust_agedep_x0=7.5,
                     dust_agedep_h=0.2)
    f = synth.make_filters(12)
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, lgu=g.lgu, mdf_mean=1, dust_bump=1, dust_law=1,
                       dust_agedep=1, dust_x0=7.5, dust_h=0.2)
    yield c, c.add_filters(f), oracle.Filters(f), grid
    c.close()


def _pop(n, seed):
    p = synth.make_population(synth.SFH_DPL_QUENCH, n, seed)
    p = synth.with_agedep_dust(synth.with_nebular(p, seed), seed)
    return _util.params_f32(synth.with_terf_mdf(p, seed))


def test_rows(combo):
    ctx, _, _, grid = combo
    assert (ctx.npar, ctx.ngrad) == (16, 15) == (grid.npar, grid.ngrad)


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_photometry_matches_oracle(combo, prec, tol):
    ctx, sid, F, grid = combo
    p32, p64 = _pop(300, 71)
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
    idx = np.r_[0:5, 150:154, 296:300]
    ref = oracle.mags(grid, F, p64[:, idx])
    err = np.abs(m[idx] - ref)
    print(f"all options prec={prec}: max |dm| = {err.max():.3e}")
    assert err.max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_oracle(combo, prec):
    ctx, sid, F, grid = combo
    n = 140
    p32, p64 = _pop(n, 72)
    mbar = np.random.default_rng(11).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    idx = np.r_[0:5, 128:133, 136:140]
    _, ref = oracle.mags_vjp(grid, F, p64[:, idx], mbar[idx])
    floor = {0: 1e-3, 1: 1e-2}[prec]
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb[:, idx] - ref) / scale
    where = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"all options prec={prec}: max scaled gradient error {rel.max():.2e} at {where}")
    assert pb.shape == (15, n)
    assert rel.max() <= 1e-3


@pytest.fixture(scope="module")
def combo_table():
    from paper_2112_06830_gb300 import dsps
    g = _ssp()
    c = dsps.Context(g, sfh_model=dsps.DSPS_SFH_TABLE, max_chunk=16384, mdf_mean=dsps.DSPS_MDF_MEAN_TERF,
                     dust_bump=True, dust_law=dsps.DSPS_DUST_SALIM, dust_agedep=True, dust_agedep_x0=7.5,
                     dust_agedep_h=0.2)
    f = synth.make_filters(12)
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=oracle.SFH_TABLE, lgu=g.lgu, mdf_mean=1, dust_bump=1, dust_law=1,
                       dust_agedep=1, dust_x0=7.5, dust_h=0.2)
    yield c, c.add_filters(f), oracle.Filters(f), grid
    c.close()


def _pop_table(n, seed):
    p = synth.make_population(synth.SFH_DPL_QUENCH, n, seed)
    p = synth.with_agedep_dust(synth.with_nebular(p, seed), seed)
    p = synth.with_terf_mdf(p, seed)
    return _util.params_f32(synth.with_sfr_table(p, synth.FULL_GRID.n_t, seed))


@pytest.mark.parametrize("prec", [0, 1])
def test_every_option_with_a_tabulated_history(combo_table, prec):
    """Rows 0..11, log U (12, 13), old-star dust (14, 15), then the 200 node
    SFRs; gradient rows 0..10, 11, 12, 13, 14 and the 200 node rows."""
    ctx, sid, F, grid = combo_table
    n_t = synth.FULL_GRID.n_t
    assert (ctx.npar, ctx.ngrad) == (16 + n_t, 15 + n_t) == (grid.npar, grid.ngrad)
    n = 140
    p32, p64 = _pop_table(n, 73)
    mbar = np.random.default_rng(12).standard_normal((n, 12))
    m, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid,
                               torch.from_numpy(mbar.astype(np.float32)).cuda(), precision=prec)
    m, pb = m.cpu().numpy().astype(np.float64), pb.cpu().numpy().astype(np.float64)
    idx = np.r_[0:5, 128:133, 136:140]
    mref, ref = oracle.mags_vjp(grid, F, p64[:, idx], mbar[idx])
    tol = {0: _util.TOL_FP32, 1: _util.TOL_BF16X3}[prec]
    assert np.abs(m[idx] - mref).max() <= tol
    floor = {0: 1e-3, 1: 1e-2}[prec]
    g = pb[:, idx]
    assert np.all(g[:5] == 0.0)
    for rows in (slice(5, 15), slice(15, 15 + n_t)):
        r = ref[rows]
        scale = np.maximum(np.abs(r), floor * np.abs(r).max(axis=0, keepdims=True))
        ok = scale > 0
        rel = np.where(ok, np.abs(g[rows] - r) / np.where(ok, scale, 1.0), np.abs(g[rows]))
        print(f"every option + table prec={prec}: rows {rows.start}-{rows.stop - 1}: max scaled error {rel.max():.2e}")
        assert rel.max() <= 1e-3
