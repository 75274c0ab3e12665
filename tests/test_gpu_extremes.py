"""Parity of the hot path with the FP64 oracle at the edges of the parameter
space, in both precision forms, magnitudes and gradients: redshifts from
1e-3 (distance modulus near 28) to 8 (the bluest filters entirely below the
SSP grid: no flux, m = +inf, no gradient term; one sees the grid only through
its truncated Gaussian tail, 40 mag fainter than the others, where the two
sides' interpolations of the truncation step differ at 1e-2 mag: checked for
finiteness only); MDF widths from 0.01 dex (one
metallicity bin) to 1 dex; no dust and Av = 4 with delta at both ends;
masses 10^6 and 10^13; histories peaking in the first Gyr, still rising at
t_obs, and quenched by 3 dex just before t_obs.  Each extreme is applied on
its own to galaxies of the full workload, spread over several tiles."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXTREMES = {
    "z_low": (11, 1e-3),
    "z_high": (11, 8.0),
    "mdf_narrow": (6, 0.01),
    "mdf_wide": (6, 1.0),
    "no_dust": (8, 0.0),
    "dusty_steep": [(8, 4.0), (9, -0.8)],
    "dusty_flat": [(8, 4.0), (9, 0.6)],
    "mass_low": (10, 6.0),
    "mass_high": (10, 13.0),
    "early_peak": [(0, 0.3), (1, 3.0), (2, -3.0)],
    "still_rising": [(0, 13.0), (1, 1.0), (2, -0.5), (3, 13.8), (4, 0.0)],
    "fresh_quench": [(3, 4.0), (4, 3.0), (11, 1.2)],
}


@pytest.fixture(scope="module")
def full():
    from paper_2112_06830_gb300 import dsps
    ctx = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH)
    f = synth.make_filters(12)
    yield ctx, ctx.add_filters(f), oracle.Filters(f)
    ctx.close()


def _pop(name):
    p = synth.make_population(synth.SFH_DPL_QUENCH, 300, 51)
    sets = EXTREMES[name]
    for row, v in (sets if isinstance(sets, list) else [sets]):
        p[row] = v
    return _util.params_f32(p)


@pytest.mark.parametrize("name", list(EXTREMES))
def test_extreme_parameters_match_the_oracle(full, name):
    ctx, sid, F = full
    p32, p64 = _pop(name)
    d = torch.from_numpy(p32).cuda()
    idx = np.r_[0:4, 130:134, 296:300]
    grid = _util.oracle_grid("full", synth.SFH_DPL_QUENCH)
    mbar = np.random.default_rng(8).standard_normal((300, 12))
    # bands in a filter's truncated tail (see above) get no cotangent on either side
    m0 = oracle.mags(grid, F, p64[:, idx])
    fin0 = np.isfinite(m0)
    tail = fin0 & (m0 >= np.where(fin0, m0, np.inf).min(axis=1, keepdims=True) + 20.0)
    sub = mbar[idx]
    sub[tail] = 0.0
    mbar[idx] = sub
    mref, ref = oracle.mags_vjp(grid, F, p64[:, idx], mbar[idx])
    for prec, tol in ((0, _util.TOL_FP32), (1, _util.TOL_BF16X3)):
        m, pb = ctx.photometry_vjp(d, sid, torch.from_numpy(mbar.astype(np.float32)).cuda(), precision=prec)
        m = m.cpu().numpy().astype(np.float64)
        pb = pb.cpu().numpy().astype(np.float64)
        # a band receiving no flux (filter off the SSP grid at high z) is +inf on both sides;
        # a band more than 20 mag fainter than the galaxy's brightest sees only the truncated
        # tail of its filter (~1e-18 transmission): finite on both sides, not compared
        fin = np.isfinite(mref)
        assert np.array_equal(np.isposinf(m[idx]), np.isposinf(mref)) and np.array_equal(np.isfinite(m[idx]), fin)
        bright = np.where(fin, mref, np.inf).min(axis=1, keepdims=True)
        keep = fin & (mref < bright + 20.0)
        err = np.abs(m[idx][keep] - mref[keep]).max()
        floor = {0: 1e-3, 1: 1e-2}[prec]
        scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
        rel = np.abs(pb[:, idx] - ref) / scale
        print(f"{name} prec={prec}: max |dm| = {err:.2e} ({(~fin).sum()} bands without flux, "
              f"{(fin & ~keep).sum()} in a filter's tail), "
              f"max scaled gradient error {rel.max():.2e}")
        assert np.isfinite(pb).all()
        assert err <= tol
        assert rel.max() <= 1e-3
    assert ctx.device_error() == 0
