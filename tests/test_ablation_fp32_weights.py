"""Ablation of the age-bin masses in FP32 (Sec. 3.1, Eq. cspsum: a bin's mass
is M(t_obs - a_lo) - M(t_obs - a_hi), M the cumulative formed mass).

The plain FP32 form -- the cumulative mass at the time nodes as an FP32
prefix sum of the trapezoid intervals, M(t) interpolated inside an interval,
and each bin's mass the difference of two such values -- loses the young age
bins of quenched galaxies: their masses are ~1e-8 of M(t_obs), below FP32's
relative resolution of M, so the difference is mostly rounding.  The form the
library's weights kernel uses -- each bin integrated directly from the
piecewise-linear SFR (partial intervals at the edges, the whole intervals in
between from a prefix held as an unevaluated FP32 pair, TwoSum at every
addition) -- keeps them at FP32 relative precision.  Both are restated here
in numpy float32 arithmetic (IEEE single, as on the GPU) and compared with the
FP64 oracle; CPU only.  The test prints the error of the youngest bins in both
forms and asserts that the plain one fails the 1e-4 relative bound that the
compensated one meets."""
import numpy as np

import oracle
from paper_2112_06830_gb300 import synth

F = np.float32


def _two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    e = F(F(a - F(s - bb)) + F(b - bb))
    return s, e


def _masses_fp32(sfr, t0, h, t_obs, edges, compensated):
    """Bin masses int_{t_obs - e_{i+1}}^{t_obs - e_i} SFR dt for the piecewise
    linear SFR through the nodes t0 + n h, in float32."""
    n_t = len(sfr)
    sfr = sfr.astype(F)
    h32 = F(h)
    itg = np.array([F(F(0.5) * h32 * F(sfr[j] + sfr[j + 1])) for j in range(n_t - 1)], dtype=F)

    def pos(t):    # interval and position of time t on the node grid (FP64 split, as the prep kernel)
        y = (t - t0) / h
        m = int(np.floor(y))
        return m, F(y - m)

    out = np.zeros(len(edges) - 1)
    if not compensated:
        cum = np.zeros(n_t, dtype=F)
        for j in range(n_t - 1):
            cum[j + 1] = F(cum[j] + itg[j])

        def M(t):
            if t <= t0:
                return F(0.0)
            m, r = pos(t)
            s_at = F(sfr[m] + F(F(sfr[m + 1] - sfr[m]) * r))
            return F(cum[m] + F(F(0.5) * h32 * r * F(sfr[m] + s_at)))
        for i in range(len(edges) - 1):
            out[i] = F(M(t_obs - edges[i]) - M(t_obs - edges[i + 1]))
        return out
    # prefix as an unevaluated pair hi + lo
    ch = np.zeros(n_t, dtype=F)
    cl = np.zeros(n_t, dtype=F)
    for j in range(n_t - 1):
        s, e = _two_sum(ch[j], itg[j])
        ch[j + 1], cl[j + 1] = s, F(cl[j] + e)

    def partial_up(m, r):    # int_{t_m}^{t_m + r h}
        s_at = F(sfr[m] + F(F(sfr[m + 1] - sfr[m]) * r))
        return F(F(0.5) * h32 * r * F(sfr[m] + s_at)), s_at

    for i in range(len(edges) - 1):
        ta, tb = t_obs - edges[i + 1], t_obs - edges[i]     # older, younger edge
        if tb <= t0:
            continue
        mi, ri = pos(tb)
        Pi, si = partial_up(mi, ri)
        if ta <= t0:
            out[i] = F(F(ch[mi] + cl[mi]) + Pi)
            continue
        mo, ro = pos(ta)
        so = F(sfr[mo] + F(F(sfr[mo + 1] - sfr[mo]) * ro))
        w = F(edges[i + 1] - edges[i])
        if mi == mo:
            out[i] = F(F(0.5) * w * F(si + so))
        elif mi == mo + 1:
            yv = F(h32 * ri)
            out[i] = F(F(F(0.5) * F(w - yv) * F(so + sfr[mi])) + F(F(0.5) * yv * F(sfr[mi] + si)))
        else:
            Qo = F(F(0.5) * h32 * F(F(1.0) - ro) * F(so + sfr[mo + 1]))
            mid = F(F(ch[mi] - ch[mo + 1]) + F(cl[mi] - cl[mo + 1]))
            out[i] = F(F(Qo + mid) + Pi)
    return out


def test_fp32_prefix_differencing_loses_the_young_bins():
    g = synth.make_ssp(synth.FULL_GRID, 1)
    grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=synth.SFH_DPL_QUENCH)
    edges = oracle.age_edges_gyr(grid)
    h = (g.t1 - g.t0) / (g.n_t - 1)
    tn = g.t0 + h * np.arange(g.n_t)
    worst = {False: 0.0, True: 0.0}
    rng = np.random.default_rng(3)
    for k in range(12):
        # a galaxy quenched by 3 dex at t_q ~ 5 Gyr, seen at z ~ 0.05-0.4
        p = np.array([rng.uniform(1.5, 4.0), rng.uniform(1.0, 3.0), rng.uniform(-3.0, -0.5), 5.0, 3.0])
        z = rng.uniform(0.05, 0.4)
        t_obs = oracle.age_gyr(z)
        sfr = np.array([oracle.sfr(1, p, t)[0] for t in tn])
        sfr[tn > t_obs + h] = 0.0          # nodes after t_obs bound no bin
        ref = oracle.age_fracs_from_sfr(grid, sfr, t_obs)   # FP64 fractions of the total
        for comp in (False, True):
            mass = _masses_fp32(sfr, g.t0, h, t_obs, edges, comp)
            frac = mass / mass.sum()
            young = (ref > 0) & (np.arange(len(ref)) < 20)  # the youngest populated bins
            rel = np.abs(frac[young] - ref[young]) / ref[young]
            worst[comp] = max(worst[comp], float(rel.max()))
    print(f"youngest 20 age bins, 12 quenched galaxies: worst relative error of the bin masses: "
          f"plain FP32 prefix differencing {worst[False]:.2e}, direct integrals + compensated prefix "
          f"{worst[True]:.2e}")
    assert worst[True] <= 1e-4
    assert worst[False] > 1e-2
