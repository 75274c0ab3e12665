"""Pins of the oracle's nebular ionisation axis (Sec. 3.3, Eq. nebsed): the
triweight distribution of log U over bins, the three-factor SSP weights, the
reduction to the two-dimensional grid when the SSPs do not depend on U, and
the adjoint of the two new parameters -- against quadrature, structural
identities and finite differences."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2112_06830_gb300 import synth

LC, HW, CW = synth.EW_LINE
_SPEC = synth.GridSpec(24, 4, 700, 3000.0, 8000.0)


def _grid(ssp, **kw):
    return oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp, t0=ssp.t0, t1=ssp.t1, n_t=ssp.n_t,
                       sfh_model=synth.SFH_DPL_QUENCH, lgu=ssp.lgu, **kw)


def _pop(n, seed):
    return synth.with_nebular(synth.make_population(synth.SFH_DPL_QUENCH, n, seed), seed)


@pytest.fixture(scope="module")
def neb():
    ssp = synth.make_ssp_nebular(_SPEC, 3)
    return ssp, _grid(ssp)


def test_pneb_matches_quadrature_of_the_triweight(neb):
    _, g = neb
    edges = np.r_[-np.inf, 0.5 * (g.lgu[1:] + g.lgu[:-1]), np.inf]
    for us, su in ((-2.0, 0.25), (-3.3, 0.4), (-1.2, 0.1), (-4.5, 0.3)):
        P, dus, dsu = oracle.pneb(g, us, su)
        pdf = lambda x: max(0.0, 1.0 - ((x - us) / (3 * su)) ** 2) ** 3 * 35.0 / (96.0 * su)
        for k in range(g.n_u):
            lo, hi = max(edges[k], us - 3 * su), min(edges[k + 1], us + 3 * su)
            q = integrate.quad(pdf, lo, hi, epsabs=1e-14, epsrel=1e-12)[0] if hi > lo else 0.0
            assert P[k] == pytest.approx(q, abs=1e-12)
        assert P.sum() == pytest.approx(1.0, abs=1e-14)
        h = 1e-6
        np.testing.assert_allclose(dus, (oracle.pneb(g, us + h, su)[0] - oracle.pneb(g, us - h, su)[0]) / (2 * h),
                                   atol=1e-7)
        np.testing.assert_allclose(dsu, (oracle.pneb(g, us, su + h)[0] - oracle.pneb(g, us, su - h)[0]) / (2 * h),
                                   atol=1e-7)


def test_narrow_pneb_is_one_hot(neb):
    _, g = neb
    P, _, _ = oracle.pneb(g, g.lgu[2], 0.05)
    np.testing.assert_array_equal(P, np.eye(g.n_u)[2])


def test_weights_factorise(neb):
    ssp, g = neb
    p = _pop(5, 31)
    w = oracle.weights(g, p)                                 # [G, A, Z, U]
    g2 = oracle.Grid(ssp.log_age_yr, ssp.lgz, ssp.lam, ssp.l_ssp[:, :, 0, :], t0=ssp.t0, t1=ssp.t1,
                     n_t=ssp.n_t, sfh_model=synth.SFH_DPL_QUENCH)
    w2 = oracle.weights(g2, p[:12])                          # pinned 2-D weights
    for k in range(p.shape[1]):
        P, _, _ = oracle.pneb(g, p[12, k], p[13, k])
        np.testing.assert_allclose(w[k], w2[k][:, :, None] * P[None, None, :], rtol=1e-13, atol=0)
    np.testing.assert_allclose(w.sum(axis=(1, 2, 3)), 10.0 ** p[10], rtol=1e-12)


def test_u_independent_grid_reduces_to_two_dimensions():
    ssp2 = synth.make_ssp(_SPEC, 3)
    l4 = np.repeat(ssp2.l_ssp[:, :, None, :], 7, axis=2)
    g4 = oracle.Grid(ssp2.log_age_yr, ssp2.lgz, ssp2.lam, l4, t0=ssp2.t0, t1=ssp2.t1, n_t=ssp2.n_t,
                     sfh_model=synth.SFH_DPL_QUENCH, lgu=synth.LGU_GRID)
    g2 = oracle.Grid(ssp2.log_age_yr, ssp2.lgz, ssp2.lam, ssp2.l_ssp, t0=ssp2.t0, t1=ssp2.t1, n_t=ssp2.n_t,
                     sfh_model=synth.SFH_DPL_QUENCH)
    f = oracle.Filters(synth.make_filters(5, 3500.0, 7000.0))
    p = _pop(6, 32)
    p[11] = np.linspace(0.01, 0.12, 6)    # filters inside the 3000-8000 A grid
    mb = np.random.default_rng(0).standard_normal((6, 5))
    m4, pb4 = oracle.mags_vjp(g4, f, p, mb)
    m2, pb2 = oracle.mags_vjp(g2, f, p[:12], mb)
    np.testing.assert_allclose(m4, m2, rtol=0, atol=1e-11)
    np.testing.assert_allclose(pb4[:11], pb2, rtol=1e-9, atol=1e-12 * np.abs(pb2).max())
    assert np.all(np.abs(pb4[11:]) <= 1e-10 * np.abs(pb2).max(axis=0))


def test_spectrum_is_the_three_factor_sum(neb):
    ssp, g = neb
    p = _pop(4, 33)
    spec = oracle.spectra(g, p)
    w = oracle.weights(g, p)
    ref = np.einsum("gizu,izun->gn", w, ssp.l_ssp.astype(np.float64))
    dust = 10.0 ** (-0.4 * p[8][:, None] * (ssp.lam[None, :] / 5500.0) ** (p[9][:, None] - 0.7))
    np.testing.assert_allclose(spec, ref * dust, rtol=1e-12)


def test_nebular_adjoint_matches_finite_differences(neb):
    _, g = neb
    f = oracle.Filters(synth.make_filters(4, 3500.0, 7500.0))
    p = _pop(3, 34)
    p[11] = [0.02, 0.06, 0.1]
    mb = np.random.default_rng(1).standard_normal((3, 4))
    _, pb = oracle.mags_vjp(g, f, p, mb)
    assert pb.shape == (13, 3)
    rows = list(range(11)) + [12, 13]
    for gi, r in enumerate(rows):
        h = 1e-5 * max(1.0, abs(p[r]).max())
        pp, pm = p.copy(), p.copy()
        pp[r] += h
        pm[r] -= h
        fd = ((oracle.mags(g, f, pp) - oracle.mags(g, f, pm)) * mb).sum(axis=1) / (2 * h)
        np.testing.assert_allclose(pb[gi], fd, rtol=2e-4, atol=1e-6 * np.abs(pb).max(), err_msg=f"param row {r}")


def test_oiii_width_grows_with_ionisation(neb):
    # Sec. 3.3: more highly ionised gas gives stronger [OIII]; the gradient of
    # its width in u_mean is positive for a star-forming galaxy.
    _, g = neb
    p = _pop(1, 35)
    p[3, 0], p[4, 0], p[11, 0] = 13.8, 0.0, 0.1     # still forming stars
    p[12, 0] = -2.0
    ew = [oracle.line_ew(g, q, LC, HW, CW)[0] for q in
          (np.where(np.arange(14)[:, None] == 12, u, p) for u in (-3.0, -2.0, -1.5))]
    assert ew[0] < ew[1] < ew[2]
    _, pb = oracle.line_ew_vjp(g, p, np.ones(1), LC, HW, CW)
    assert pb[11, 0] > 0.0
