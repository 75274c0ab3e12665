"""Parity of the dust law with the 2175 A UV bump (Sec. 3.4, Eq. uvbump: a
Drude profile of amplitude 0.85 - 1.9 delta added to the attenuation curve)
between the CUDA path and the FP64 oracle: magnitudes in both forms and
gradients (Av and delta carry the bump's terms) in both forms."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bump():
    from paper_2112_06830_gb300 import dsps
    c = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH, dust_bump=True)
    f = synth.make_filters(12)
    g = _util.ssp("full")
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, dust_bump=1)
    return c, c.add_filters(f), oracle.Filters(f), grid


def _pop(n, seed, start):
    p = synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start)
    p[11] = np.linspace(0.3, 2.9, n)   # bands over rest-frame 900-7000 A: the bump (2175 A) is seen
    return _util.params_f32(p)


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_photometry_matches_oracle(bump, prec, tol):
    ctx, sid, F, grid = bump
    p32, p64 = _pop(300, 8, 4000)
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
    ref = oracle.mags(grid, F, p64)
    err = np.abs(m - ref)
    print(f"UV bump prec={prec}: max |dm| = {err.max():.3e}")
    assert err.max() <= tol
    # the bump changes the magnitudes (it is not silently off)
    g0 = _util.oracle_grid("full", synth.SFH_DPL_QUENCH)
    assert np.abs(oracle.mags(g0, F, p64[:, :20]) - ref[:20]).max() > 1e-3


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_oracle(bump, prec):
    ctx, sid, F, grid = bump
    n = 120
    p32, p64 = _pop(n, 10, 800)
    mbar = np.random.default_rng(4).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    _, ref = oracle.mags_vjp(grid, F, p64, mbar)
    floor = {0: 1e-3, 1: 1e-2}[prec]
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb - ref) / scale
    where = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"UV bump prec={prec}: max scaled gradient error {rel.max():.2e} at {where}")
    assert rel.max() <= 1e-3
