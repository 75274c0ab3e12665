"""Pins of the oracle's rest-frame absolute magnitudes (Sec. 2.2, Eq. restmag:
the filter at the rest wavelength, no distance modulus or (1+z) term): a flat
L_nu spectrum's closed form at any redshift; the identity with the pinned
observer frame through a filter stretched by (1+z); and the gradient against
central differences."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

_SPEC = synth.GridSpec(24, 5, 3000, 1000.0, 30000.0)


def _grid(l_ssp=None, **kw):
    ssp = synth.make_ssp(_SPEC, 3)
    L = ssp.l_ssp if l_ssp is None else l_ssp
    return ssp, oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, L, t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t,
                            sfh_model=synth.SFH_DPL_QUENCH, **kw)


def test_flat_spectrum_closed_form_at_any_redshift():
    # Every SSP row L_nu = C: the galaxy's L_nu is 10^logM C at every
    # wavelength, and with Av = 0 M_Q = -2.5 log10(10^logM C / AB0) for every
    # filter and redshift (to the trapezoid's quadrature error, < 1e-5 mag).
    C = 3e-15
    ssp, g = _grid()
    _, g = _grid(l_ssp=np.full_like(ssp.l_ssp, C))
    F = oracle.Filters(synth.make_filters(5, 2500.0, 9000.0, 600.0), rest=True)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 4, 21)
    p[8] = 0.0
    p[11] = [0.05, 0.7, 1.9, 3.0]
    m = oracle.mags(g, F, p)
    ref = -2.5 * np.log10(10.0 ** p[10] * C / oracle.AB0)
    np.testing.assert_allclose(m, np.repeat(ref[:, None], 5, axis=1), rtol=0, atol=1e-5)


def test_rest_frame_is_the_observer_frame_through_a_stretched_filter():
    # T'(lam') = T(lam' / (1+z)) seen in the observer frame at z samples the
    # rest-frame filter at every node, with the same normalisation:
    # M_Q = m'_Q - Dmod(z) + 2.5 log10(1+z) (the observer frame is pinned on
    # its own).
    _, g = _grid()
    tables = synth.make_filters(4, 3000.0, 8000.0, 700.0)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 3, 22)
    p[11] = [0.1, 0.8, 1.6]
    M = oracle.mags(g, oracle.Filters(tables, rest=True), p)
    for k in range(3):
        z = p[11, k]
        stretched = oracle.Filters([(l * (1.0 + z), t) for l, t in tables])
        m = oracle.mags(g, stretched, p[:, k:k + 1])[0]
        np.testing.assert_allclose(M[k], m - oracle.dist_mod(z) + 2.5 * np.log10(1.0 + z), rtol=0, atol=1e-10)


def test_rest_frame_gradient_matches_central_differences():
    _, g = _grid(dust_bump=1)
    F = oracle.Filters(synth.make_filters(4, 3000.0, 8000.0, 700.0), rest=True)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 2, 23)
    mb = np.random.default_rng(5).standard_normal((2, 4))
    _, pb = oracle.mags_vjp(g, F, p, mb)
    scale = np.abs(pb).max()
    for r in range(11):
        h = 1e-5 * max(1.0, abs(p[r]).max())
        pp, pm = p.copy(), p.copy()
        pp[r] += h
        pm[r] -= h
        fd = ((oracle.mags(g, F, pp) - oracle.mags(g, F, pm)) * mb).sum(axis=1) / (2 * h)
        np.testing.assert_allclose(pb[r], fd, rtol=2e-4, atol=1e-6 * scale, err_msg=f"row {r}")
    # the logM row: -2.5 per magnitude, as in the observer frame
    np.testing.assert_allclose(pb[10], -2.5 * mb.sum(axis=1), rtol=1e-12)


def test_rest_frame_magnitudes_see_the_redshift_only_through_the_age():
    # Same galaxy at two redshifts: the rest-frame magnitudes differ only by
    # the SED's evolution (t_obs); with a constant-in-time SSP block (every
    # age row equal) and a metallicity-free grid they coincide.
    ssp, _ = _grid()
    L = np.repeat(ssp.l_ssp[:1], ssp.l_ssp.shape[0], axis=0)
    L = np.repeat(L[:, :1], ssp.l_ssp.shape[1], axis=1)
    _, g = _grid(l_ssp=L)
    F = oracle.Filters(synth.make_filters(4, 3000.0, 8000.0, 700.0), rest=True)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 1, 24)
    q = np.repeat(p, 2, axis=1)
    q[11] = [0.2, 2.0]
    m = oracle.mags(g, F, q)
    np.testing.assert_allclose(m[0], m[1], rtol=0, atol=1e-10)
