"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here compares the oracle with something other than itself: closed
forms, invariants, library routines (scipy quadrature / special functions),
values the paper prints (tests/golden/paper_constants.txt) and brute force on
tiny inputs.  CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from paper_2112_06830_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = float(val)
    return out


# ---------------------------------------------------------------- Appendix B

def test_terf_printed_constraints():
    g = _golden()
    assert oracle.triweight_cdf(-3.0) == pytest.approx(g["terf_at_minus3"], abs=1e-15)
    assert oracle.triweight_cdf(0.0) == pytest.approx(g["terf_at_0"], abs=1e-15)
    assert oracle.triweight_cdf(3.0) == pytest.approx(g["terf_at_plus3"], abs=1e-15)
    # reading: saturates outside [-3, 3]
    assert oracle.triweight_cdf(-7.0) == 0.0 and oracle.triweight_cdf(7.0) == 1.0
    # the polynomial itself reaches the endpoints (not only the clamp)
    assert oracle.triweight_cdf(3.0 - 1e-9) == pytest.approx(1.0, abs=1e-12)
    assert oracle.triweight_cdf(-3.0 + 1e-9) == pytest.approx(0.0, abs=1e-12)


def test_triweight_moments():
    g = _golden()
    norm = integrate.quad(oracle.triweight_pdf, -3, 3, epsabs=1e-14)[0]
    mean = integrate.quad(lambda z: z * oracle.triweight_pdf(z), -3, 3, epsabs=1e-14)[0]
    var = integrate.quad(lambda z: z * z * oracle.triweight_pdf(z), -3, 3, epsabs=1e-14)[0]
    assert norm == pytest.approx(g["triweight_norm"], abs=1e-12)
    assert mean == pytest.approx(0.0, abs=1e-12)
    assert var == pytest.approx(g["triweight_var"], abs=1e-12)
    assert oracle.triweight_pdf(3.5) == 0.0 and oracle.triweight_pdf(-3.5) == 0.0


@pytest.mark.parametrize("z", [-2.9, -1.7, -0.3, 0.0, 0.4, 1.1, 2.5, 2.99])
def test_terf_is_integral_of_triweight(z):
    ref = integrate.quad(oracle.triweight_pdf, -3, z, epsabs=1e-15, epsrel=1e-14)[0]
    assert oracle.triweight_cdf(z) == pytest.approx(ref, abs=1e-13)


@pytest.mark.parametrize("z", [-6.0, -2.0, -0.5, 0.0, 0.7, 3.0, 8.0])
def test_gauss_cdf_matches_library(z):
    assert oracle.gauss_cdf(z) == pytest.approx(stats.norm.cdf(z), rel=1e-13, abs=1e-300)


# ---------------------------------------------------------------- cosmology

H0_GYR = 977.792221 / 70.0


@pytest.mark.parametrize("z", [0.0, 0.1, 0.5, 1.5, 3.0, 8.0])
def test_age_eds_closed_form(z):
    t = oracle.age_gyr(z, om0=1.0, w0=-1.0, h=0.7)
    assert t == pytest.approx(2.0 / 3.0 * H0_GYR * (1 + z) ** -1.5, rel=1e-10)


@pytest.mark.parametrize("z", [0.001, 0.1, 1.0, 3.0])
def test_lum_dist_eds_closed_form(z):
    dl = oracle.lum_dist_mpc(z, om0=1.0, w0=-1.0, h=0.7)
    c_h0 = 299792.458 / 70.0
    ref = 2.0 * c_h0 * (1 + z) * (1 - (1 + z) ** -0.5)
    assert dl == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("z", [0.0, 0.1, 1.5, 3.0])
def test_age_flat_lcdm_closed_form(z):
    om, ol = 0.3, 0.7
    ref = 2.0 / (3.0 * math.sqrt(ol)) * H0_GYR * math.asinh(math.sqrt(ol / om) * (1 + z) ** -1.5)
    assert oracle.age_gyr(z) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("w0", [-1.0, -0.8, -1.2])
def test_lum_dist_wcdm_library_quadrature(w0):
    z = 1.3
    E = lambda x: math.sqrt(0.3 * (1 + x) ** 3 + 0.7 * (1 + x) ** (3 * (1 + w0)))
    ref = (1 + z) * 299792.458 / 70.0 * integrate.quad(lambda x: 1 / E(x), 0, z, epsrel=1e-13)[0]
    assert oracle.lum_dist_mpc(z, w0=w0) == pytest.approx(ref, rel=1e-10)
    assert oracle.dist_mod(z, w0=w0) == pytest.approx(5 * math.log10(ref * 1e5), abs=1e-9)


def test_ab0_is_3631_jansky_at_10pc():
    g = _golden()
    pc = 3.0856775814913673e16
    lsun = 3.828e26
    ab0 = 3631e-26 * 4 * math.pi * (10 * pc) ** 2 / lsun
    assert g["AB0_Lsun_per_Hz"] == pytest.approx(ab0, rel=1e-3)


# ---------------------------------------------------------------- SFH / weights

@pytest.mark.parametrize("model,p", [
    (0, [1.3, 0, 0, 0, 0]),
    (1, [4.0, 2.0, -1.5, 9.0, 1.7]),
    (1, [2.0, 1.2, -2.5, 6.0, 0.4]),
])
@pytest.mark.parametrize("t", [0.3, 5.0, 8.8, 8.95, 12.0])
def test_sfr_gradient_fd(model, p, t):
    _, g = oracle.sfr(model, p, t)
    for k in range(5 if model == 1 else 1):
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = list(p), list(p)
        pp[k] += h
        pm[k] -= h
        fd = (oracle.sfr(model, pp, t)[0] - oracle.sfr(model, pm, t)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_quench_floor_reached_at_tq():
    # Sec. 3.1: q_drop = log10 SFR(t_q) - log10 SFR_ms(t_q) (quench floor at t_q)
    p = [4.0, 2.0, -1.5, 9.0, 1.7]
    ms = lambda t: 1.0 / ((t / 4.0) ** -2.0 + (t / 4.0) ** 1.5)
    for t in (9.0, 9.5, 12.0):
        assert math.log10(oracle.sfr(1, p, t)[0] / ms(t)) == pytest.approx(-1.7, abs=1e-12)
    assert oracle.sfr(1, p, 7.1)[0] == pytest.approx(ms(7.1), rel=1e-14)


def test_cum_mass_exact_for_linear_sfr():
    t0, t1, n = 0.05, 13.8, 200
    t = np.linspace(t0, t1, n)
    a, b = 0.7, 0.31
    s = a + b * t
    for tau in (0.01, 0.05, 0.123, 3.3, 13.47, 13.8):
        v, coef = oracle.cum_mass(s, t0, t1, tau)
        ref = 0.0 if tau <= t0 else a * (tau - t0) + 0.5 * b * (tau ** 2 - t0 ** 2)
        assert v == pytest.approx(ref, rel=1e-12, abs=1e-14)
        assert coef @ s == pytest.approx(v, rel=1e-12, abs=1e-14)


def _tiny_grid(n_age=94, n_t=200, sfh_model=0, kernel=0, n_z=12, lam=None, l_ssp=None):
    log_age = np.linspace(5.5, 10.15, n_age)
    lgz = np.linspace(-2.0, 0.3, n_z)
    if lam is None:
        lam = np.geomspace(1e3, 1e5, 8)
    if l_ssp is None:
        l_ssp = np.ones((n_age, n_z, len(lam)))
    return oracle.Grid(log_age, lgz, lam, l_ssp, n_t=n_t, sfh_model=sfh_model, mdf_kernel=kernel)


def test_age_fracs_constant_sfr_closed_form():
    g = _tiny_grid()
    e = oracle.age_edges_gyr(g)
    t_obs = 9.1
    fr = oracle.age_fracs_from_sfr(g, np.ones(g.n_t), t_obs)
    lo = np.clip(t_obs - e[1:], g.t0, t_obs)
    hi = np.clip(t_obs - e[:-1], g.t0, t_obs)
    ref = (hi - lo) / (t_obs - g.t0)
    np.testing.assert_allclose(fr, ref, rtol=1e-11, atol=1e-15)
    assert fr.sum() == pytest.approx(1.0, abs=1e-13)


def test_age_edges_are_log_midpoints():
    g = _tiny_grid()
    e = oracle.age_edges_gyr(g)
    x = g.log_age_yr
    assert e[0] == 0.0
    np.testing.assert_allclose(np.log10(e[1:-1]) + 9, 0.5 * (x[1:] + x[:-1]), rtol=1e-13)
    assert np.log10(e[-1]) + 9 == pytest.approx(x[-1] + 0.5 * (x[-1] - x[-2]), rel=1e-13)


def test_delayed_tau_converges_to_closed_form():
    """int_{t0}^{t} t' e^{-t'/tau} dt' has a closed form; the piecewise-linear
    reading converges to it at second order as the time grid refines."""
    tau, t_obs = 0.8, 6.0
    errs = []
    for n_t in (100, 200, 400):
        g = _tiny_grid(n_t=n_t)
        tt = np.linspace(g.t0, g.t1, n_t)
        fr = oracle.age_fracs_from_sfr(g, tt * np.exp(-tt / tau), t_obs)
        prim = lambda x: -tau * np.exp(-x / tau) * (x + tau)
        cm = lambda x: np.where(x <= g.t0, 0.0, prim(np.maximum(x, g.t0)) - prim(g.t0))
        e = oracle.age_edges_gyr(g)
        ref = (cm(t_obs - e[:-1]) - cm(t_obs - e[1:])) / cm(t_obs)
        errs.append(np.abs(fr - ref).max())
    assert errs[2] < 1e-4
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.15)


@pytest.mark.parametrize("model", [0, 1])
def test_weights_sum_to_formed_mass(model):
    g, _, _ = synth.workload_inputs("small")
    G = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=model)
    p = synth.make_population(model, 16, 7)
    w = oracle.weights(G, p)
    np.testing.assert_allclose(w.sum(axis=(1, 2)), 10.0 ** p[10], rtol=1e-12)
    assert (w >= 0).all()


# ---------------------------------------------------------------- MDF

@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("mu,sig", [(-0.7, 0.2), (0.25, 0.05), (-1.9, 0.5), (0.0, 1.3)])
def test_mdf_sums_to_one_and_matches_quadrature(kernel, mu, sig):
    g = _tiny_grid(kernel=kernel)
    P, dmu, dsig = oracle.mdf(g, mu, sig)
    assert P.sum() == pytest.approx(1.0, abs=1e-13)
    edges = np.concatenate([[-np.inf], 0.5 * (g.lgz[1:] + g.lgz[:-1]), [np.inf]])
    if kernel == 0:
        cdf = lambda x: 0.0 if x == -np.inf else (1.0 if x == np.inf else integrate.quad(
            oracle.triweight_pdf, -3.0, float(np.clip((x - mu) / sig, -3, 3)), epsabs=1e-15)[0])
    else:
        cdf = lambda x: stats.norm.cdf((x - mu) / sig)
    ref = np.array([cdf(edges[j + 1]) - cdf(edges[j]) for j in range(g.n_z)])
    np.testing.assert_allclose(P, ref, atol=1e-12)
    # derivative columns against central differences
    h = 1e-6
    fd_mu = (oracle.mdf(g, mu + h, sig)[0] - oracle.mdf(g, mu - h, sig)[0]) / (2 * h)
    fd_sig = (oracle.mdf(g, mu, sig + h)[0] - oracle.mdf(g, mu, sig - h)[0]) / (2 * h)
    np.testing.assert_allclose(dmu, fd_mu, atol=1e-6)
    np.testing.assert_allclose(dsig, fd_sig, atol=1e-6)


def test_mdf_mirror_symmetry_and_narrow_limit():
    g = _tiny_grid()
    j0 = 6
    P, _, _ = oracle.mdf(g, g.lgz[j0], 0.15)
    for d in range(1, 5):
        assert P[j0 + d] == pytest.approx(P[j0 - d], abs=1e-14)
    P, _, _ = oracle.mdf(g, g.lgz[j0] + 0.01, 1e-4)
    assert P[j0] == pytest.approx(1.0, abs=1e-14)


# ---------------------------------------------------------------- dust / filters

@pytest.mark.parametrize("delta", [-0.4, 0.0, 0.3])
def test_dust_normalisation(delta):
    assert oracle.dust_trans(1234.0, 0.0, delta) == 1.0
    assert -2.5 * math.log10(oracle.dust_trans(5500.0, 0.63, delta)) == pytest.approx(0.63, rel=1e-14)
    # steeper than lambda_V is more attenuated in the blue for delta < 0.7
    assert oracle.dust_trans(3000.0, 0.5, delta) < oracle.dust_trans(8000.0, 0.5, delta)


def test_filter_interpolation_and_norm():
    lam = np.linspace(4000, 5000, 11)
    tr = 0.2 + 0.5e-3 * (lam - 4000)
    for x in (4000.0, 4123.4, 4999.9, 5000.0):
        assert oracle.filter_trans(lam, tr, x) == pytest.approx(0.2 + 0.5e-3 * (x - 4000), rel=1e-14)
    assert oracle.filter_trans(lam, tr, 3999.0) == 0.0
    assert oracle.filter_trans(lam, tr, 5000.1) == 0.0
    assert oracle.filter_norm(lam, tr) == pytest.approx(np.trapezoid(tr / lam, lam), rel=1e-14)


# ---------------------------------------------------------------- photometry

def _flat_case(n_lam=20000):
    lam = np.geomspace(900.0, 1e5, n_lam)
    return lam


@pytest.mark.parametrize("z", [0.02, 0.7, 1.0])  # filters stay on the rest grid
def test_flat_spectrum_analytic_magnitude(z):
    """Flat L_nu = AB0 10^{-0.4 M}: every filter gives m = M - 2.5 logM + Dmod - 2.5 log10(1+z)."""
    lam = _flat_case()
    Mabs = -1.3
    l_ssp = np.full((2, 2, len(lam)), oracle.AB0 * 10 ** (-0.4 * Mabs))
    g = oracle.Grid([8.0, 9.0], [-0.5, 0.0], lam, l_ssp)
    F = oracle.Filters(synth.make_filters(4))
    omega = np.array([0.1, 0.2, 0.3, 0.4])
    logM, dmod = 10.3, 44.1
    m = oracle.mags_from_weights(g, F, omega, 0.0, 0.0, logM, z, dmod)
    ref = Mabs - 2.5 * logM + dmod - 2.5 * math.log10(1 + z)
    np.testing.assert_allclose(m, ref, atol=2e-6)


@pytest.mark.parametrize("z", [0.1, 1.2])
@pytest.mark.parametrize("beta", [-2.0, 0.5])
def test_narrow_filter_samples_rest_frame_luminosity(z, beta):
    lam = _flat_case(40000)
    L = 1e-14 * (lam / 5000.0) ** beta
    g = oracle.Grid([9.0], [0.0], lam, L.reshape(1, 1, -1))
    lc = 6100.0
    F = oracle.Filters([synth.gaussian_filter(lc, fwhm=10.0, step=0.05)])
    m = oracle.mags_from_weights(g, F, [1.0], 0.0, 0.0, 0.0, z, 0.0)[0]
    ref = -2.5 * math.log10(1e-14 * (lc / (1 + z) / 5000.0) ** beta / oracle.AB0) - 2.5 * math.log10(1 + z)
    assert m == pytest.approx(ref, abs=2e-5)


@pytest.mark.parametrize("delta", [-0.3, 0.2])
def test_dust_at_lambda_v_dims_by_av(delta):
    z = 0.4
    lam = _flat_case(40000)
    L = np.full((1, 1, len(lam)), 1e-14)
    g = oracle.Grid([9.0], [0.0], lam, L)
    F = oracle.Filters([synth.gaussian_filter(5500.0 * (1 + z), fwhm=10.0, step=0.05)])
    m0 = oracle.mags_from_weights(g, F, [1.0], 0.0, delta, 0.0, z, 0.0)[0]
    m1 = oracle.mags_from_weights(g, F, [1.0], 0.8, delta, 0.0, z, 0.0)[0]
    assert m1 - m0 == pytest.approx(0.8, abs=1e-5)


def test_one_hot_weights_reproduce_one_ssp():
    lam = np.geomspace(1e3, 1e5, 300)
    rng = np.random.default_rng(3)
    L = rng.uniform(1e-16, 1e-14, (3, 2, len(lam)))
    g = oracle.Grid([7.0, 8.0, 9.0], [-1.0, 0.0], lam, L)
    F = oracle.Filters(synth.make_filters(3))
    for k in range(6):
        om = np.zeros(6)
        om[k] = 1.0
        g1 = oracle.Grid([9.0], [0.0], lam, L.reshape(6, 1, -1)[k:k + 1])
        a = oracle.mags_from_weights(g, F, om, 0.3, -0.1, 9.5, 0.5, 40.0)
        b = oracle.mags_from_weights(g1, F, [1.0], 0.3, -0.1, 9.5, 0.5, 40.0)
        np.testing.assert_allclose(a, b, atol=1e-12)


def test_logm_shifts_all_bands():
    g, f, p = synth.workload_inputs("small", n_gal=3)
    G = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp)
    F = oracle.Filters(f)
    m0 = oracle.mags(G, F, p)
    p2 = p.copy()
    p2[10] += 0.37
    np.testing.assert_allclose(oracle.mags(G, F, p2) - m0, -2.5 * 0.37, atol=1e-10)


# ---------------------------------------------------------------- brute force

def _brute_force_mags(log_age, lgz, lam, L, filters, par, sfh_model, kernel, om0=0.3, h=0.7, mean=0,
                      x0=9.0, hw=0.5, bump=0, law=0):
    """Independent restatement on a tiny grid: scipy quadrature of the SFR
    function itself for every age bin, quadrature of the MDF density for every
    lgZ bin, scipy quadrature for the cosmology, and an explicit loop for the
    rest-frame trapezoid through np.interp-ed filters."""
    H0 = 977.792221 / (100 * h)
    z = par[11]
    E = lambda x: math.sqrt(om0 * (1 + x) ** 3 + (1 - om0))
    t_obs = H0 * integrate.quad(lambda x: 1.0 / ((1 + x) * E(x)), z, np.inf, epsrel=1e-13, limit=200)[0]
    dl = (1 + z) * 299792.458 / (100 * h) * integrate.quad(lambda x: 1.0 / E(x), 0, z, epsrel=1e-13)[0]
    dmod = 5 * math.log10(dl * 1e5)
    sfr = lambda t: oracle.sfr(sfh_model, par[:5], t)[0]
    t0 = 0.05
    edges = np.concatenate([[0.0], 10 ** (0.5 * (log_age[1:] + log_age[:-1]) - 9),
                            [10 ** (log_age[-1] + 0.5 * (log_age[-1] - log_age[-2]) - 9)]])
    mass = lambda a, b: integrate.quad(sfr, max(a, t0), max(b, t0), epsabs=0, epsrel=1e-12, limit=400)[0] if b > t0 else 0.0
    Mtot = mass(t0, t_obs)
    frac = np.array([mass(t_obs - edges[i + 1], t_obs - edges[i]) / Mtot for i in range(len(log_age))])
    zedges = np.concatenate([[-np.inf], 0.5 * (lgz[1:] + lgz[:-1]), [np.inf]])
    pdf = oracle.triweight_pdf if kernel == 0 else (lambda u: math.exp(-0.5 * u * u) / math.sqrt(2 * math.pi))
    S = np.zeros(len(lam))
    tri = lambda u: 35.0 / 96.0 * (1.0 - u * u / 9.0) ** 3 if abs(u) < 3.0 else 0.0
    for i in range(len(log_age)):
        if mean == 0:
            mu = par[5] + par[7] * (log_age[i] - 9)
        else:   # transition young -> old along the quadrature of the triweight density
            zt = (log_age[i] - x0) / hw
            T = 0.0 if zt <= -3 else (1.0 if zt >= 3 else integrate.quad(tri, -3.0, zt, epsabs=1e-15)[0])
            mu = (1.0 - T) * par[5] + T * par[7]
        sg = par[6]
        for j in range(len(lgz)):
            a = max((zedges[j] - mu) / sg, -8.0)
            b = min((zedges[j + 1] - mu) / sg, 8.0)
            P = integrate.quad(pdf, a, b, epsabs=1e-15, points=[-3.0, 3.0] if a < -3 < b or a < 3 < b else None)[0] if b > a else 0.0
            S += frac[i] * P * L[i, j]
    out = []
    for fl, ft in filters:
        tot = 0.0
        for n in range(len(lam)):
            w = 0.5 * ((lam[min(n + 1, len(lam) - 1)] - lam[max(n - 1, 0)]))
            T = np.interp((1 + z) * lam[n], fl, ft, left=0.0, right=0.0)
            A = (lam[n] / 5500.0) ** (-0.7 + par[9])
            if law:    # Eq. (salim): k0 (lam/lam_V)^delta / 4.05, k0 of Eq. (kzero)
                x = lam[n] * 1e-4
                if x < 0.15:
                    k0 = 5.472 + 0.671 / x - 9.218e-3 / x ** 2 + 2.620e-3 / x ** 3
                elif x < 0.63:
                    k0 = 2.659 * (-2.156 + 1.509 / x - 0.198 / x ** 2 + 0.011 / x ** 3) + 4.05
                else:
                    k0 = 2.659 * (-1.857 + 1.040 / x) + 4.05
                A = max(k0, 0.0) / 4.05 * (lam[n] / 5500.0) ** par[9]
            if bump:   # Drude profile at 2175 A, width 350 A, amplitude 0.85 - 1.9 delta, over 4.05
                x = lam[n] * 350.0
                A += (0.85 - 1.9 * par[9]) * x * x / ((lam[n] ** 2 - 2175.0 ** 2) ** 2 + x * x) / 4.05
            F = 10 ** (-0.4 * par[8] * A)
            tot += w / lam[n] * T * F * S[n]
        D = np.trapezoid(ft / fl, fl)
        out.append(-2.5 * math.log10(10 ** par[10] * tot / (oracle.AB0 * D)) + dmod - 2.5 * math.log10(1 + z))
    return np.array(out)


@pytest.mark.parametrize("sfh_model,kernel,mean,bump,law", [(0, 0, 0, 0, 0), (1, 0, 0, 0, 0), (1, 1, 0, 0, 0),
                                                            (1, 0, 1, 0, 0), (1, 0, 0, 1, 0), (1, 0, 0, 1, 1)])
def test_brute_force_tiny_grid(sfh_model, kernel, mean, bump, law):
    log_age = np.array([6.0, 7.5, 8.7, 9.6])
    lgz = np.array([-1.0, -0.4, 0.1])
    lam = np.geomspace(2000.0, 9000.0, 16)
    rng = np.random.default_rng(11)
    L = rng.uniform(0.5e-15, 2e-15, (4, 3, 16))
    filters = [synth.gaussian_filter(c, fwhm=600.0, step=5.0) for c in (4000.0, 6500.0)]
    n_t = 40001  # fine time grid: the piecewise-linear reading is then within 1e-7 of the quadrature
    if bump:
        lam = np.geomspace(1200.0, 9000.0, 16)      # across the 2175 A bump (and 0.15 um, 0.63 um)
    g = oracle.Grid(log_age, lgz, lam, L, n_t=n_t, sfh_model=sfh_model, mdf_kernel=kernel, mdf_mean=mean,
                    mdf_x0=8.0, mdf_h=0.6, dust_bump=bump, dust_law=law)
    F = oracle.Filters(filters)
    p = synth.make_population(sfh_model, 3, 5)
    p[6] = 0.35
    p[11] = np.minimum(p[11], 0.6)
    if mean == 1:
        p[5], p[7] = [0.2, -0.1, 0.05], [-0.9, -0.6, -1.2]     # mu_young, mu_old
    m = oracle.mags(g, F, p)
    for gi in range(p.shape[1]):
        ref = _brute_force_mags(log_age, lgz, lam, L, filters, p[:, gi], sfh_model, kernel, mean=mean, x0=8.0,
                                hw=0.6, bump=bump, law=law)
        np.testing.assert_allclose(m[gi], ref, atol=2e-6)


# ---------------------------------------------------------------- gradients

@pytest.mark.parametrize("wl,model,kernel,mean,bump,law", [("small", 0, 0, 0, 0, 0), ("small", 1, 0, 0, 0, 0),
                                                            ("small", 1, 1, 0, 0, 0), ("small", 1, 0, 1, 0, 0),
                                                            ("small", 1, 0, 0, 1, 0), ("small", 1, 0, 0, 1, 1)])
def test_adjoint_matches_central_differences(wl, model, kernel, mean, bump, law):
    g, f, _ = synth.workload_inputs(wl, n_gal=1)
    G = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=model, mdf_kernel=kernel, mdf_mean=mean,
                    dust_bump=bump, dust_law=law)
    F = oracle.Filters(f)
    p = synth.make_population(model, 3, 21)
    if mean == 1:
        p[5], p[7] = [0.1, -0.2, 0.25], [-0.8, -1.1, -0.5]     # mu_young, mu_old
    rng = np.random.default_rng(0)
    mbar = rng.standard_normal((p.shape[1], F.n_filt))
    _, pb = oracle.mags_vjp(G, F, p, mbar)
    for gi in range(p.shape[1]):
        for k in range(11):
            if model == 0 and 1 <= k <= 4:
                assert pb[k, gi] == 0.0
                continue
            h = 1e-4 * max(1.0, abs(p[k, gi]))
            pp, pm = p[:, gi:gi + 1].copy(), p[:, gi:gi + 1].copy()
            pp[k] += h
            pm[k] -= h
            fd = ((oracle.mags(G, F, pp) - oracle.mags(G, F, pm)) @ mbar[gi]).item() / (2 * h)
            scale = max(abs(fd), 1e-3 * np.abs(pb[:, gi]).max())
            assert abs(pb[k, gi] - fd) <= 2e-5 * scale + 1e-9, (gi, k, pb[k, gi], fd)


def test_gradient_signs_follow_the_paper():
    """Sec. 3.4: more dust dims every band; Sec. 3.2 (Fig. 4): a higher mean
    metallicity reddens the optical colour (the synthetic grid is cooler at
    higher Z); logM gives -2.5 exactly."""
    g, f, _ = synth.workload_inputs("small", n_gal=1)
    G = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp)
    F = oracle.Filters(f)
    p = synth.make_population(0, 8, 2)
    for q in range(F.n_filt):
        mb = np.zeros((8, F.n_filt))
        mb[:, q] = 1.0
        _, pb = oracle.mags_vjp(G, F, p, mb)
        assert (pb[8] > 0).all()
        np.testing.assert_allclose(pb[10], -2.5, atol=1e-12)
    mb = np.zeros((8, F.n_filt))
    mb[:, 0], mb[:, -1] = 1.0, -1.0          # blue minus red colour
    _, pb = oracle.mags_vjp(G, F, p, mb)
    assert (pb[5] > 0).all()


# ---------------------------------------------------------------- age-dependent MDF, T_erf form

def _terf_grid(x0=8.5, h=0.4):
    xs = np.array([x0 - 3 * h - 0.2, x0 - 3 * h - 0.01, x0 - 0.7 * h, x0, x0 + 1.3 * h, x0 + 3 * h + 0.01,
                   x0 + 3 * h + 0.3])
    lam = np.geomspace(1e3, 1e5, 50)
    L = np.ones((len(xs), 3, len(lam)))
    return oracle.Grid(xs, [-1.0, -0.3, 0.2], lam, L, mdf_mean=1, mdf_x0=x0, mdf_h=h), xs


def test_terf_mean_limits_midpoint_and_weights():
    """Sec. 3.2: the mean is the young value for the youngest populations and
    the old value for the oldest (the triweight CDF saturates at +-3 widths),
    the average of the two at the transition centre, and its derivatives with
    respect to the two values sum to one."""
    g, xs = _terf_grid()
    par = np.zeros(12)
    par[5], par[7] = 0.3, -1.1
    mus = [oracle.mdf_mean(g, par, i) for i in range(len(xs))]
    assert mus[0][0] == 0.3 and mus[1][0] == 0.3
    assert mus[-1][0] == -1.1 and mus[-2][0] == -1.1
    assert mus[3][0] == pytest.approx(0.5 * (0.3 - 1.1), abs=1e-15)
    for mu, d5, d7 in mus:
        assert d5 + d7 == pytest.approx(1.0, abs=1e-15)
        assert 0.0 <= d7 <= 1.0
    # monotone from young to old
    assert all(a[0] >= b[0] for a, b in zip(mus, mus[1:]))


def test_terf_mean_derivatives_match_differences():
    g, xs = _terf_grid()
    par = np.zeros(12)
    par[5], par[7] = 0.2, -0.9
    for i in range(len(xs)):
        _, d5, d7 = oracle.mdf_mean(g, par, i)
        for k, d in ((5, d5), (7, d7)):
            pp, pm = par.copy(), par.copy()
            pp[k] += 1e-6
            pm[k] -= 1e-6
            fd = (oracle.mdf_mean(g, pp, i)[0] - oracle.mdf_mean(g, pm, i)[0]) / 2e-6
            assert fd == pytest.approx(d, abs=1e-9)


def test_terf_mean_with_equal_values_is_the_uncorrelated_mdf():
    """mu_young = mu_old = mu gives the age-independent MDF (Eq. simple_mdf),
    the linear form with zero slope."""
    g, f, p = synth.workload_inputs("small", n_gal=4)
    Gt = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, mdf_mean=1, mdf_x0=8.0, mdf_h=0.7)
    Gl = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, mdf_mean=0)
    pt, pl = p.copy(), p.copy()
    pt[7] = pt[5]
    pl[7] = 0.0
    np.testing.assert_allclose(oracle.weights(Gt, pt), oracle.weights(Gl, pl), rtol=1e-9, atol=0)


# ---------------------------------------------------------------- UV bump (Eq. uvbump)

def test_drude_peak_and_half_maximum():
    """The Drude profile peaks at 1 (unit amplitude) at 2175 A and falls to
    one half where |lam^2 - lam_b^2| = lam dlam, lam = (+-350 + sqrt(350^2 +
    4 2175^2)) / 2."""
    assert oracle.drude(2175.0) == 1.0
    for sgn in (-1.0, 1.0):
        lam = 0.5 * (sgn * 350.0 + math.sqrt(350.0 ** 2 + 4 * 2175.0 ** 2))
        assert oracle.drude(lam) == pytest.approx(0.5, abs=1e-13)
    assert oracle.drude(1.0e5) < 1e-4 and oracle.drude(1000.0) < 0.05


def test_bump_amplitude_vanishes_at_its_zero():
    """E_b = 0.85 - 1.9 delta: at delta = 0.85/1.9 the bump leaves the curve
    unchanged; elsewhere it adds E_b D0 / 4.05 (largest at 2175 A)."""
    lam = np.geomspace(1e3, 1e4, 7)
    g0 = oracle.Grid([9.0], [0.0], lam, np.ones((1, 1, len(lam))))
    g1 = oracle.Grid([9.0], [0.0], lam, np.ones((1, 1, len(lam))), dust_bump=1)
    d0 = 0.85 / 1.9
    for l in list(lam) + [2175.0]:
        assert oracle.dust_curve(g1, l, d0)[0] == pytest.approx(oracle.dust_curve(g0, l, d0)[0], abs=1e-15)
    diff = [oracle.dust_curve(g1, l, -0.2)[0] - oracle.dust_curve(g0, l, -0.2)[0] for l in (1500.0, 2175.0, 3500.0)]
    assert diff[1] > diff[0] > 0 and diff[1] > diff[2] > 0
    assert diff[1] == pytest.approx((0.85 + 0.38) / 4.05, rel=1e-14)


def test_bump_curve_derivative_matches_differences():
    lam = np.geomspace(1e3, 1e4, 5)
    g1 = oracle.Grid([9.0], [0.0], lam, np.ones((1, 1, len(lam))), dust_bump=1)
    for l in (1200.0, 2175.0, 2600.0, 5500.0):
        c, dc = oracle.dust_curve(g1, l, -0.1)
        fd = (oracle.dust_curve(g1, l, -0.1 + 1e-6)[0] - oracle.dust_curve(g1, l, -0.1 - 1e-6)[0]) / 2e-6
        assert dc == pytest.approx(fd, rel=1e-7, abs=1e-10)


# ---------------------------------------------------------------- population statistic (Sec. 5.1)

def test_colour_cut_histogram_counts_a_hand_made_population():
    m = np.array([[20.0, 19.0, 18.5],    # colour 1.0, r 18.5 -> bin 1 of [18, 20) x 4
                  [20.0, 19.9, 19.9],    # colour 0.1: cut
                  [21.0, 20.0, 17.9],    # r below range
                  [22.0, 20.5, 19.99],   # colour 1.5, bin 3
                  [np.nan, 19.0, 18.6],  # NaN colour
                  [23.0, 21.0, 18.0]])   # colour 2.0, r on the lower edge -> bin 0
    h = oracle.colour_cut_histogram(m, 0, 1, 0.5, 2, 18.0, 20.0, 4)
    np.testing.assert_array_equal(h, [1, 1, 0, 1])


# ---------------------------------------------------------------- Eq. (salim) with Eq. (kzero)

def test_k0_is_normalised_at_v_and_continuous_where_the_fits_meet():
    """The starburst curve is built so that k(V) = R_V = 4.05; the Leitherer
    and Calzetti fits meet at 0.15 um to a few tenths of a per cent, and the two
    Calzetti pieces at 0.63 um to about 1 per cent."""
    assert oracle.k0(5500.0) == pytest.approx(4.05, rel=1e-3)
    lo, hi = oracle.k0(1500.0 - 1e-6), oracle.k0(1500.0)
    assert abs(lo - hi) / hi < 3e-3
    lo, hi = oracle.k0(6300.0 - 1e-6), oracle.k0(6300.0)
    assert abs(lo - hi) / hi < 1e-2
    ks = [oracle.k0(l) for l in np.geomspace(912.0, 3.0e4, 400)]
    assert all(a >= b for a, b in zip(ks, ks[1:]))          # decreasing with wavelength
    assert oracle.k0(3.2e4) == 0.0 and oracle.k0(1e5) == 0.0  # clipped where the fit turns negative


def test_salim_curve_at_v_is_av_for_every_delta():
    lam = np.geomspace(1000.0, 1e5, 50)
    g = oracle.Grid([9.0], [0.0], lam, np.ones((1, 1, len(lam))), dust_law=1)
    for d in (-0.6, -0.2, 0.0, 0.3):
        c, dc = oracle.dust_curve(g, 5500.0, d)
        assert c == pytest.approx(oracle.k0(5500.0) / 4.05, rel=1e-14)
        assert dc == pytest.approx(0.0, abs=1e-15)           # the tilt pivots at lambda_V
        for l in (1200.0, 3000.0, 9000.0):
            fd = (oracle.dust_curve(g, l, d + 1e-6)[0] - oracle.dust_curve(g, l, d - 1e-6)[0]) / 2e-6
            assert oracle.dust_curve(g, l, d)[1] == pytest.approx(fd, rel=1e-7)


# ------------------------------------------------------------ domain of the model

def test_out_of_domain_galaxies_give_nan_and_leave_the_rest_alone():
    """Outside the forward model's domain (z <= 0 or not finite, MDF width <= 0;
    the library's own domain) every output of that galaxy is NaN and its
    neighbours are untouched.  z <= -1 puts the cosmology integrals' limits
    outside the reals; the oracle must not evaluate them (it returns at once)."""
    import time
    g = synth.make_ssp(synth.GridSpec(9, 5, 120, 1e3, 1e5), 0)
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=1)
    F = oracle.Filters(synth.make_filters(3))
    p = synth.make_population(1, 9, 2)
    good = p.copy()
    bad_z = [0.0, -0.5, -1.0, -2.0, np.nan, np.inf]
    for k, z in enumerate(bad_z):
        p[11, k] = z
    p[6, 6] = 0.0                                      # zero MDF width
    t0 = time.perf_counter()
    m = oracle.mags(grid, F, p)
    w = oracle.weights(grid, p)
    m2, pb = oracle.mags_vjp(grid, F, p, np.ones((9, 3)))
    ew = oracle.line_ew(grid, p, 5007.0, 40.0, 300.0)
    sp = oracle.spectra(grid, p)
    assert time.perf_counter() - t0 < 30.0
    bad = list(range(7))
    assert np.isnan(m[bad]).all() and np.isnan(w[bad]).all() and np.isnan(pb[:, bad]).all()
    assert np.isnan(ew[bad]).all() and np.isnan(sp[bad]).all() and np.isnan(m2[bad]).all()
    ok = [7, 8]
    np.testing.assert_array_equal(m[ok], oracle.mags(grid, F, good)[ok])
    assert np.isfinite(pb[:, ok]).all()
