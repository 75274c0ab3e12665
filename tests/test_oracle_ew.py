"""Pins of the oracle's rest-frame spectrum and emission-line equivalent width
(Sec. 2.2, Eq. eqw) against closed forms, library routines and finite
differences -- independent of the oracle's own fit and adjoint code."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

LC, HW, CW = synth.EW_LINE


def _compact_line(x, s):
    """(1 - (x/s)^2)^3 on |x| < s, zero outside: a line with compact support."""
    u = np.clip(x / s, -1.0, 1.0)
    return (1.0 - u * u) ** 3 * (np.abs(x) < s)


def test_quadratic_spectrum_has_zero_width():
    lam = np.geomspace(4000.0, 6000.0, 4001)
    x = lam - LC
    L = 3.0 + 1e-3 * x + 2e-6 * x * x
    w, _ = oracle.ew_from_spectrum(lam, L, LC, HW, CW)
    assert abs(w) < 1e-10


def test_compact_line_on_quadratic_continuum():
    # The continuum windows see the exact quadratic, so the fit recovers it and
    # W is the integral of the line profile: A s 32/35 for (1 - u^2)^3.
    lam = np.geomspace(4000.0, 6000.0, 40001)
    x = lam - LC
    cont = 3.0 + 1e-3 * x + 2e-6 * x * x
    A, s = 2.0, 10.0
    L = cont * (1.0 + A * _compact_line(x, s))
    w, _ = oracle.ew_from_spectrum(lam, L, LC, HW, CW)
    m = np.abs(x) <= HW
    assert w == pytest.approx(np.trapezoid(A * _compact_line(x, s)[m], lam[m]), rel=1e-10)
    assert w == pytest.approx(A * s * 32.0 / 35.0, rel=1e-7)


def test_absorption_line_is_negative_and_scale_free():
    lam = np.geomspace(4000.0, 6000.0, 8001)
    x = lam - LC
    L = (2.0 - 1e-4 * x) * (1.0 - 0.5 * _compact_line(x, 12.0))
    w, _ = oracle.ew_from_spectrum(lam, L, LC, HW, CW)
    w2, _ = oracle.ew_from_spectrum(lam, 1e-17 * L, LC, HW, CW)
    assert w < 0.0
    assert w == pytest.approx(-0.5 * 12.0 * 32.0 / 35.0, rel=1e-5)
    assert w2 == pytest.approx(w, rel=1e-12)


def test_fit_matches_numpy_polyfit():
    # A noisy continuum: the least-squares quadratic is numpy's polyfit.
    rng = np.random.default_rng(0)
    lam = np.geomspace(4500.0, 5500.0, 600)
    x = lam - LC
    L = (1.0 + 1e-4 * x) * np.exp(0.05 * rng.standard_normal(len(lam))) * (1.0 + 3.0 * _compact_line(x, 15.0))
    w, _ = oracle.ew_from_spectrum(lam, L, LC, HW, CW)
    cm = (np.abs(x) > HW) & (np.abs(x) <= HW + CW)
    lm = np.abs(x) <= HW
    c = np.polyfit(x[cm], L[cm], 2)
    L0 = np.polyval(c, x[lm])
    assert w == pytest.approx(np.trapezoid((L[lm] - L0) / L0, lam[lm]), rel=1e-10)


def test_too_few_points_give_nan():
    lam = np.geomspace(1000.0, 1e5, 200)   # ~110 A apart at 5000 A
    w, _ = oracle.ew_from_spectrum(lam, np.ones(200), LC, HW, CW)
    assert np.isnan(w)


def test_spectrum_adjoint_matches_finite_differences():
    rng = np.random.default_rng(1)
    lam = np.geomspace(4700.0, 5300.0, 300)
    x = lam - LC
    L = (1.0 + 2e-4 * x + 1e-6 * x * x) * np.exp(0.03 * rng.standard_normal(len(lam))) * (
        1.0 + 1.5 * _compact_line(x, 14.0))
    _, lb = oracle.ew_from_spectrum(lam, L, LC, HW, CW)
    used = np.nonzero(np.abs(x) <= HW + CW)[0]
    assert np.all(lb[np.abs(x) > HW + CW] == 0.0)
    for k in used[:: max(1, len(used) // 25)]:
        h = 1e-6 * L[k]
        Lp, Lm = L.copy(), L.copy()
        Lp[k] += h
        Lm[k] -= h
        fd = (oracle.ew_from_spectrum(lam, Lp, LC, HW, CW)[0] - oracle.ew_from_spectrum(lam, Lm, LC, HW, CW)[0]) / (2 * h)
        assert lb[k] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.max(np.abs(lb)))


# ---- galaxy level ------------------------------------------------------------

_SPEC = synth.GridSpec(30, 5, 800, 3000.0, 8000.0)


def _grid(line=True, **kw):
    ssp = synth.make_ssp(_SPEC, 5)
    if line:
        ssp = synth.with_emission_line(ssp)
    return ssp, oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t,
                            sfh_model=synth.SFH_DPL_QUENCH, **kw)


def test_spectrum_is_weights_times_ssp_times_dust():
    ssp, g = _grid(line=False)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 6, 11)
    spec = oracle.spectra(g, p)
    w = oracle.weights(g, p)                               # Msun, pinned separately
    ref = np.einsum("gij,ijn->gn", w, ssp.l_ssp.astype(np.float64))
    dust = 10.0 ** (-0.4 * p[8][:, None] * (ssp.lam[None, :] / 5500.0) ** (p[9][:, None] - 0.7))
    np.testing.assert_allclose(spec, ref * dust, rtol=1e-12)


def test_galaxy_ew_matches_polyfit_of_spectrum():
    ssp, g = _grid()
    p = synth.make_population(synth.SFH_DPL_QUENCH, 8, 12)
    ew = oracle.line_ew(g, p, LC, HW, CW)
    spec = oracle.spectra(g, p)
    x = ssp.lam - LC
    cm = (np.abs(x) > HW) & (np.abs(x) <= HW + CW)
    lm = np.abs(x) <= HW
    for k in range(p.shape[1]):
        c = np.polyfit(x[cm], spec[k, cm], 2)
        L0 = np.polyval(c, x[lm])
        assert ew[k] == pytest.approx(np.trapezoid((spec[k, lm] - L0) / L0, ssp.lam[lm]), rel=1e-9, abs=1e-9)
    assert np.all(ew > 0.0)   # the emission line of the young populations


def test_quenching_weakens_the_line():
    _, g = _grid()
    p = synth.make_population(synth.SFH_DPL_QUENCH, 2, 13)
    p[:, 1] = p[:, 0]
    p[3, 0], p[4, 0] = 13.8, 0.0       # still forming stars at t_obs
    p[3, 1], p[4, 1] = 5.0, 3.0        # quenched 1000x at 5 Gyr
    p[11] = 0.1
    ew = oracle.line_ew(g, p, LC, HW, CW)
    assert ew[0] > ew[1] > 0.0


@pytest.mark.parametrize("bump", [0, 1])
def test_galaxy_ew_adjoint_matches_finite_differences(bump):
    _, g = _grid(dust_bump=bump)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 3, 14)
    eb = np.array([1.0, -0.5, 2.0])
    ew, pb = oracle.line_ew_vjp(g, p, eb, LC, HW, CW)
    np.testing.assert_allclose(ew, oracle.line_ew(g, p, LC, HW, CW), rtol=1e-14)
    for r in range(oracle.NGRAD):
        h = 1e-5 * max(1.0, abs(p[r]).max())
        pp, pm = p.copy(), p.copy()
        pp[r] += h
        pm[r] -= h
        fd = eb * (oracle.line_ew(g, pp, LC, HW, CW) - oracle.line_ew(g, pm, LC, HW, CW)) / (2 * h)
        scale = np.abs(pb).max(axis=0)
        np.testing.assert_allclose(pb[r], fd, rtol=2e-4, atol=1e-6 * scale.max(), err_msg=f"row {r}")
    # W is a ratio of spectra: the mass drops out
    assert np.all(np.abs(pb[10]) <= 1e-9 * np.abs(pb).max(axis=0))


# ---- age-dependent dust (Sec. 3.4.1) ----------------------------------------


def _agedep_pop(n, seed):
    p = synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, n, seed), seed)
    p[3], p[4] = 13.8, 0.0            # still forming stars: the young bins carry the line
    return p


@pytest.mark.parametrize("law,bump", [(0, 0), (1, 1)])
def test_agedep_ew_adjoint_matches_finite_differences(law, bump):
    _, g = _grid(dust_agedep=1, dust_x0=7.2, dust_h=0.4, dust_law=law, dust_bump=bump)
    p = _agedep_pop(3, 15)
    eb = np.array([0.7, -1.2, 1.5])
    ew, pb = oracle.line_ew_vjp(g, p, eb, LC, HW, CW)
    assert pb.shape == (13, 3)
    np.testing.assert_allclose(ew, oracle.line_ew(g, p, LC, HW, CW), rtol=1e-14)
    rows = list(range(11)) + [12, 13]
    scale = np.abs(pb).max()
    for gi, r in enumerate(rows):
        h = 1e-5 * max(1.0, abs(p[r]).max())
        pp, pm = p.copy(), p.copy()
        pp[r] += h
        pm[r] -= h
        fd = eb * (oracle.line_ew(g, pp, LC, HW, CW) - oracle.line_ew(g, pm, LC, HW, CW)) / (2 * h)
        np.testing.assert_allclose(pb[gi], fd, rtol=2e-4, atol=1e-6 * scale, err_msg=f"param row {r}")


def test_agedep_dust_changes_the_width_and_reduces_to_one_curve():
    # Young stars behind more dust than old ones dim the line against the
    # continuum; equal young and old values give the one-curve spectrum and
    # width, and the old-star gradient rows add to the one-curve ones.
    _, g = _grid(dust_agedep=1, dust_x0=7.2, dust_h=0.4)
    _, g0 = _grid()
    p = _agedep_pop(3, 16)
    p[12], p[13] = p[8], p[9]
    q = p[:12]
    np.testing.assert_allclose(oracle.spectra(g, p), oracle.spectra(g0, q), rtol=1e-12)
    eb = np.array([1.0, 2.0, -1.0])
    ew, pb = oracle.line_ew_vjp(g, p, eb, LC, HW, CW)
    ew0, pb0 = oracle.line_ew_vjp(g0, q, eb, LC, HW, CW)
    np.testing.assert_allclose(ew, ew0, rtol=1e-12)
    tol = 1e-9 * np.abs(pb0).max()
    np.testing.assert_allclose(pb[:8], pb0[:8], rtol=1e-9, atol=tol)
    np.testing.assert_allclose(pb[8] + pb[11], pb0[8], rtol=1e-9, atol=tol)
    np.testing.assert_allclose(pb[9] + pb[12], pb0[9], rtol=1e-9, atol=tol)
    dusty = p.copy()
    dusty[8] = p[12] + 1.0            # young stars behind one more magnitude of Av
    assert np.all(oracle.line_ew(g, dusty, LC, HW, CW) < ew)
