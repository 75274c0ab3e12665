"""Pins of the oracle's tabulated star formation history (Sec. 3.1: the SFH
enters only through its values on the cosmic-time grid, Eqs. cspsum and
mstartot): a table holding a parametric model's node values reproduces that
model and, through the chain rule, its gradient; a constant table gives the
closed-form weights; the table fixes the shape and logM the mass; nodes after
t_obs do nothing; and the table gradient agrees with central differences."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

_SPEC = synth.GridSpec(24, 5, 600, 1200.0, 9000.0)
_F = oracle.Filters(synth.make_filters(4, 3500.0, 7500.0, 600.0))


def _grids(model, **kw):
    ssp = synth.make_ssp(_SPEC, 9)
    base = dict(t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t, **kw)
    gt = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, sfh_model=oracle.SFH_TABLE, **base)
    gp = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, sfh_model=model, **base)
    return ssp, gt, gp


def _nodes(grid):
    return grid.t0 + np.arange(grid.n_t) * (grid.t1 - grid.t0) / (grid.n_t - 1)


def _tabulate(grid, model, p):
    """Parametric SFR (and dSFR/dp_k) at the nodes, from the oracle's model."""
    t = _nodes(grid)
    v = np.array([[oracle.sfr(model, p[:, g], tn)[0] for tn in t] for g in range(p.shape[1])])
    d = np.array([[oracle.sfr(model, p[:, g], tn)[1] for tn in t] for g in range(p.shape[1])])
    return v, d          # [G, n_t], [G, n_t, 5]


def _with_table(p, tab):
    out = np.zeros((p.shape[0] + tab.shape[1], p.shape[1]))
    out[:p.shape[0]] = p
    out[:5] = 0.0
    out[p.shape[0]:] = tab.T
    return out


@pytest.mark.parametrize("model", [synth.SFH_DELAYED_TAU, synth.SFH_DPL_QUENCH])
def test_table_of_a_model_reproduces_it(model):
    _, gt, gp = _grids(model)
    p = synth.make_population(model, 4, 31)
    tab, dtab = _tabulate(gp, model, p)
    q = _with_table(p, tab)
    assert (gt.npar, gt.ngrad) == (12 + gt.n_t, 11 + gt.n_t)
    np.testing.assert_allclose(oracle.weights(gt, q), oracle.weights(gp, p), rtol=1e-12, atol=0)
    mb = np.random.default_rng(1).standard_normal((4, 4))
    m_t, pb_t = oracle.mags_vjp(gt, _F, q, mb)
    m_p, pb_p = oracle.mags_vjp(gp, _F, p, mb)
    np.testing.assert_allclose(m_t, m_p, rtol=0, atol=1e-12)
    tol = 1e-10 * np.abs(pb_p).max()
    np.testing.assert_allclose(pb_t[5:11], pb_p[5:11], rtol=1e-10, atol=tol)
    assert np.all(pb_t[:5] == 0.0)                       # unused rows
    # chain rule: sum_n dLoss/dSFR_n dSFR_n/dp_k is the parametric gradient
    chain = np.einsum("ng,gnk->kg", pb_t[11:], dtab)
    np.testing.assert_allclose(chain, pb_p[:5], rtol=1e-9, atol=tol)


def test_constant_table_gives_the_closed_form_weights():
    # Constant SFR on [t0, t_obs]: bin i holds the overlap of its time range
    # [t_obs - e_{i+1}, t_obs - e_i] with [t0, t_obs], over t_obs - t0.
    ssp, gt, _ = _grids(synth.SFH_DELAYED_TAU)
    p = synth.make_population(synth.SFH_DELAYED_TAU, 3, 32)
    q = _with_table(p, np.full((3, gt.n_t), 2.5))
    w = oracle.weights(gt, q)
    e = oracle.age_edges_gyr(gt)
    for g in range(3):
        t_obs = oracle.age_gyr(p[11, g])
        lo = np.clip(t_obs - e[1:], gt.t0, t_obs)
        hi = np.clip(t_obs - e[:-1], gt.t0, t_obs)
        ref = 10.0 ** p[10, g] * (hi - lo) / (t_obs - gt.t0)
        np.testing.assert_allclose(w[g].sum(axis=1), ref, rtol=1e-12, atol=1e-12 * ref.max())


def test_table_sets_the_shape_and_logm_the_mass():
    _, gt, _ = _grids(synth.SFH_DPL_QUENCH)
    p = synth.with_sfr_table(synth.make_population(synth.SFH_DPL_QUENCH, 4, 33), gt.n_t, 33)
    q = p.copy()
    q[12:] *= 37.0
    np.testing.assert_allclose(oracle.mags(gt, _F, q), oracle.mags(gt, _F, p), rtol=0, atol=1e-12)
    w = oracle.weights(gt, p)
    np.testing.assert_allclose(w.sum(axis=(1, 2)), 10.0 ** p[10], rtol=1e-12)
    # scale invariance: sum_n SFR_n dLoss/dSFR_n = 0
    _, pb = oracle.mags_vjp(gt, _F, p, np.ones((4, 4)))
    s = (pb[11:] * p[12:]).sum(axis=0)
    assert np.all(np.abs(s) <= 1e-10 * (np.abs(pb[11:] * p[12:])).sum(axis=0))


def test_nodes_after_the_observation_do_nothing():
    _, gt, _ = _grids(synth.SFH_DPL_QUENCH)
    p = synth.with_sfr_table(synth.make_population(synth.SFH_DPL_QUENCH, 3, 34), gt.n_t, 34)
    p[11] = [2.5, 1.0, 0.3]
    t = _nodes(gt)
    q = p.copy()
    for g in range(3):
        after = t > oracle.age_gyr(p[11, g]) + (t[1] - t[0])
        q[12:, g][after] = 1e3 * (1.0 + np.arange(after.sum()))
    np.testing.assert_allclose(oracle.mags(gt, _F, q), oracle.mags(gt, _F, p), rtol=0, atol=1e-12)
    _, pb = oracle.mags_vjp(gt, _F, p, np.ones((3, 4)))
    for g in range(3):
        after = t > oracle.age_gyr(p[11, g]) + (t[1] - t[0])
        assert np.all(pb[11:, g][after] == 0.0)


def test_table_gradient_matches_central_differences():
    _, gt, _ = _grids(synth.SFH_DPL_QUENCH)
    p = synth.with_sfr_table(synth.make_population(synth.SFH_DPL_QUENCH, 2, 35), gt.n_t, 35)
    p[11] = [0.4, 1.2]
    mb = np.random.default_rng(4).standard_normal((2, 4))
    _, pb = oracle.mags_vjp(gt, _F, p, mb)
    scale = np.abs(pb).max()
    for n in (0, 3, 40, 77, 120):
        h = 1e-6 * max(1.0, np.abs(p[12 + n]).max())
        pp, pm = p.copy(), p.copy()
        pp[12 + n] += h
        pm[12 + n] -= h
        fd = ((oracle.mags(gt, _F, pp) - oracle.mags(gt, _F, pm)) * mb).sum(axis=1) / (2 * h)
        np.testing.assert_allclose(pb[11 + n], fd, rtol=2e-5, atol=1e-7 * scale, err_msg=f"node {n}")
    for r in (5, 6, 7, 8, 9, 10):
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[r] += h
        pm[r] -= h
        fd = ((oracle.mags(gt, _F, pp) - oracle.mags(gt, _F, pm)) * mb).sum(axis=1) / (2 * h)
        np.testing.assert_allclose(pb[r], fd, rtol=2e-4, atol=1e-6 * scale, err_msg=f"row {r}")


def test_rows_with_other_options_and_short_params_are_refused():
    ssp = synth.make_ssp_nebular(_SPEC, 3)
    g = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t,
                    sfh_model=oracle.SFH_TABLE, lgu=ssp.lgu, dust_agedep=1)
    assert (g.row_sfr, g.grow_sfr) == (16, 15)
    assert (g.npar, g.ngrad) == (16 + g.n_t, 15 + g.n_t)
    with pytest.raises(ValueError):
        oracle.mags(g, _F, np.zeros((16, 2)))
