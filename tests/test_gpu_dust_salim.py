"""Parity of the paper's attenuation law (Sec. 3.4, Eq. salim with the
starburst curve k0 of Eq. kzero: A = Av k0(lam) (lam/5500 A)^delta / 4.05,
optionally with the UV bump) between the CUDA path and the FP64 oracle:
magnitudes and gradients in both precision forms, and the line width."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 1], ids=["nobump", "bump"])
def salim(request):
    from paper_2112_06830_gb300 import dsps
    bump = request.param
    c = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH, dust_bump=bool(bump),
                     dust_law=dsps.DSPS_DUST_SALIM)
    f = synth.make_filters(12)
    g = _util.ssp("full")
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, dust_bump=bump, dust_law=1)
    yield c, c.add_filters(f), oracle.Filters(f), grid
    c.close()


def _pop(n, seed, start):
    p = synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start)
    p[11] = np.linspace(0.3, 2.9, n)   # bands over rest-frame 900-7000 A: both k0 fits are seen
    return _util.params_f32(p)


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_photometry_matches_oracle(salim, prec, tol):
    ctx, sid, F, grid = salim
    p32, p64 = _pop(300, 8, 4000)
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
    idx = np.r_[0:12, 140:150, 290:300]
    ref = oracle.mags(grid, F, p64[:, idx])
    err = np.abs(m[idx] - ref)
    print(f"Salim law prec={prec}: max |dm| = {err.max():.3e}")
    assert err.max() <= tol
    # the law changes the magnitudes (it is not silently the power law)
    g0 = _util.oracle_grid("full", synth.SFH_DPL_QUENCH)
    assert np.abs(oracle.mags(g0, F, p64[:, idx[:6]]) - ref[:6]).max() > 1e-2


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_oracle(salim, prec):
    ctx, sid, F, grid = salim
    n = 120
    p32, p64 = _pop(n, 10, 800)
    mbar = np.random.default_rng(4).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    idx = np.r_[0:10, 60:66, 110:120]
    _, ref = oracle.mags_vjp(grid, F, p64[:, idx], mbar[idx])
    floor = {0: 1e-3, 1: 1e-2}[prec]
    scale = np.maximum(np.abs(ref), floor * np.abs(ref).max(axis=0, keepdims=True))
    rel = np.abs(pb[:, idx] - ref) / scale
    where = np.unravel_index(np.argmax(rel), rel.shape)
    print(f"Salim law prec={prec}: max scaled gradient error {rel.max():.2e} at {where}")
    assert rel.max() <= 1e-3


def test_spectra_match_oracle(salim):
    ctx, _, _, grid = salim
    p32, p64 = _pop(64, 12, 0)
    s = ctx.spectra(torch.from_numpy(p32).cuda(), 0, 3000).cpu().numpy().astype(np.float64)
    ref = oracle.spectra(grid, p64[:, ::8])[:, :3000]
    pos = ref > 0
    rel = np.abs(s[::8][pos] - ref[pos]) / ref[pos]
    print(f"Salim law spectra: max relative error {rel.max():.2e}")
    assert rel.max() <= 2e-5
