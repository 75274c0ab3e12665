"""A band whose filter lies entirely outside the SSP grid at the galaxy's
redshift receives no flux (L = 0 off the grid): its magnitude is +inf, and it
contributes nothing to the gradient -- the other bands' gradients are those
of the filter set without it."""
import numpy as np

import oracle
from paper_2112_06830_gb300 import synth

_SPEC = synth.GridSpec(20, 4, 1500, 1000.0, 30000.0)


def test_offgrid_band_is_infinite_and_drops_out_of_the_gradient():
    ssp = synth.make_ssp(_SPEC, 2)
    g = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t,
                    sfh_model=synth.SFH_DPL_QUENCH)
    on = synth.make_filters(3, 4000.0, 8000.0, 600.0)
    off = [synth.gaussian_filter(900.0, 100.0)]          # 500-1300 A observed: 333-867 A rest at z = 0.5
    p = synth.make_population(synth.SFH_DPL_QUENCH, 3, 41)
    p[11] = 0.5
    mb = np.random.default_rng(2).standard_normal((3, 4))
    m, pb = oracle.mags_vjp(g, oracle.Filters(on + off), p, mb)
    m0, pb0 = oracle.mags_vjp(g, oracle.Filters(on), p, mb[:, :3])
    assert np.all(np.isposinf(m[:, 3]))
    np.testing.assert_allclose(m[:, :3], m0, rtol=0, atol=1e-12)
    assert np.all(np.isfinite(pb))
    np.testing.assert_allclose(pb, pb0, rtol=1e-12, atol=1e-14 * np.abs(pb0).max())
