"""Pins of the oracle's age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp:
Av and delta move from young-star to old-star values along T_erf in log age,
each age bin attenuated by its own curve): its limits, an independent
restatement from the pinned weights, and central differences."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

_SPEC = synth.GridSpec(26, 4, 700, 1200.0, 9000.0)


def _grids(law=0, bump=0, **kw):
    ssp = synth.make_ssp(_SPEC, 6)
    base = dict(t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t, sfh_model=synth.SFH_DPL_QUENCH, dust_law=law, dust_bump=bump)
    g = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, dust_agedep=1, **base, **kw)
    g0 = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, **base)
    return ssp, g, g0


def _pop(n, seed):
    p = synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, n, seed), seed)
    p[11] = np.linspace(0.02, 0.3, n)
    return p


_F = oracle.Filters(synth.make_filters(5, 3500.0, 7500.0, 600.0))


def test_equal_young_and_old_values_reduce_to_one_curve():
    _, g, g0 = _grids(dust_x0=7.5, dust_h=0.3)
    p = _pop(4, 51)
    p[12], p[13] = p[8], p[9]
    mb = np.random.default_rng(2).standard_normal((4, 5))
    m, pb = oracle.mags_vjp(g, _F, p, mb)
    m0, pb0 = oracle.mags_vjp(g0, _F, p[:12], mb)
    np.testing.assert_allclose(m, m0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(pb[:8], pb0[:8], rtol=1e-10, atol=1e-13 * np.abs(pb0).max())
    np.testing.assert_allclose(pb[8] + pb[11], pb0[8], rtol=1e-10, atol=1e-13 * np.abs(pb0).max())
    np.testing.assert_allclose(pb[9] + pb[12], pb0[9], rtol=1e-10, atol=1e-13 * np.abs(pb0).max())


@pytest.mark.parametrize("x0,side", [(2.0, "old"), (13.0, "young")])
def test_transition_beyond_the_grid_gives_one_population(x0, side):
    _, g, g0 = _grids(dust_x0=x0, dust_h=0.2)
    p = _pop(3, 52)
    q = p[:12].copy()
    if side == "old":
        q[8], q[9] = p[12], p[13]
    m = oracle.mags(g, _F, p)
    np.testing.assert_allclose(m, oracle.mags(g0, _F, q), rtol=0, atol=1e-12)
    _, pb = oracle.mags_vjp(g, _F, p, np.ones((3, 5)))
    unused = (8, 9) if side == "old" else (11, 12)
    assert np.all(pb[list(unused)] == 0.0)


@pytest.mark.parametrize("law,bump", [(0, 0), (1, 1)])
def test_restatement_from_the_weights(law, bump):
    ssp, g, _ = _grids(law=law, bump=bump, dust_x0=7.2, dust_h=0.4)
    p = _pop(3, 53)
    w = oracle.weights(g, p)                                       # pinned weights [G, A, Z]
    spec = oracle.spectra(g, p)
    lam = ssp.lam
    T = np.array([oracle.triweight_cdf((x - 7.2) / 0.4) for x in ssp.log_age_yr])
    for k in range(p.shape[1]):
        Av = (1 - T) * p[8, k] + T * p[12, k]
        dl = (1 - T) * p[9, k] + T * p[13, k]
        curve = np.array([[oracle.dust_curve(g, l, d)[0] for l in lam] for d in dl])   # [A, N], pinned curves
        F = 10.0 ** (-0.4 * Av[:, None] * curve)
        ref = np.einsum("iz,izn,in->n", w[k], ssp.l_ssp.astype(np.float64), F)
        np.testing.assert_allclose(spec[k], ref, rtol=1e-12)


@pytest.mark.parametrize("law,bump", [(0, 0), (1, 1)])
def test_adjoint_matches_central_differences(law, bump):
    _, g, _ = _grids(law=law, bump=bump, dust_x0=7.3, dust_h=0.5)
    p = _pop(3, 54)
    mb = np.random.default_rng(3).standard_normal((3, 5))
    _, pb = oracle.mags_vjp(g, _F, p, mb)
    assert pb.shape == (13, 3)
    rows = list(range(11)) + [12, 13]
    for gi, r in enumerate(rows):
        h = 1e-5 * max(1.0, abs(p[r]).max())
        pp, pm = p.copy(), p.copy()
        pp[r] += h
        pm[r] -= h
        fd = ((oracle.mags(g, _F, pp) - oracle.mags(g, _F, pm)) * mb).sum(axis=1) / (2 * h)
        np.testing.assert_allclose(pb[gi], fd, rtol=2e-4, atol=1e-6 * np.abs(pb).max(), err_msg=f"param row {r}")


def test_young_dust_reddens_a_star_forming_galaxy_more():
    # Sec. 3.4.1: colours respond more to the young stars' dust than to the old.
    _, g, _ = _grids(dust_x0=7.0, dust_h=0.1)
    p = _pop(1, 55)
    p[3, 0], p[4, 0] = 13.8, 0.0                 # still forming stars
    _, pb = oracle.mags_vjp(g, _F, p, np.array([[1.0, 0.0, 0.0, 0.0, -1.0]]))   # bluest - reddest colour
    assert abs(pb[8, 0]) > abs(pb[11, 0])
