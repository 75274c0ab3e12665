"""Band coverage (include/dsps.h: dsps_band_coverage): the fraction of each
filter's response int T dlam / lam (the denominator of Eq. restmag) that falls
on the SSP grid as the galaxy is seen (Sec. 2.2), against a float64
evaluation from the filter tables, and as the marker of the bands whose
magnitudes carry the far-tail representation error: every band at or above
a coverage floor meets the ordinary tolerance against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _coverage_ref(tables, lam_grid, z, rest):
    """Covered fraction per (galaxy, filter): the trapezoids of T / lam of the
    filter's own table over [lam_0, lam_{N-1}] (times 1+z in the observer
    frame), a partial interval counted in proportion to its length in lam."""
    out = np.zeros((len(z), len(tables)))
    for q, (lam, t) in enumerate(tables):
        seg = 0.5 * np.diff(lam) * (t[1:] / lam[1:] + t[:-1] / lam[:-1])
        D = seg.sum()
        for g, zz in enumerate(z):
            f = 1.0 if rest else 1.0 + float(zz)
            la, lb = lam_grid[0] * f, lam_grid[-1] * f
            t0 = np.clip((la - lam[:-1]) / np.diff(lam), 0.0, 1.0)
            t1 = np.clip((lb - lam[:-1]) / np.diff(lam), 0.0, 1.0)
            out[g, q] = np.sum(seg * (t1 - t0)) / D
    return out


@pytest.mark.parametrize("rest", [False, True])
def test_coverage_matches_the_filter_tables(rest):
    from paper_2112_06830_gb300 import dsps
    g = _util.ssp("full")
    ctx = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH)
    tables = synth.make_filters(16, 3300.0, 11000.0)
    sid = ctx.add_filters(tables, rest_frame=rest)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 40, 5)
    p[11] = np.r_[np.geomspace(1e-3, 9.5, 38), 3.0, 6.0]
    p32, _ = _util.params_f32(p)
    cov = ctx.band_coverage(torch.from_numpy(p32).cuda(), sid).cpu().numpy().astype(np.float64)
    ref = _coverage_ref(tables, np.asarray(g.lam, dtype=np.float64), p32[11].astype(np.float64), rest)
    err = np.abs(cov - ref) / np.maximum(ref, 1e-30)
    print(f"rest={rest}: coverage from {ref.min():.2e} to {ref.max():.3f}, worst relative difference "
          f"{err[ref > 1e-30].max():.2e}")
    assert ((ref <= 1e-30) <= (cov <= 1e-30)).all()
    assert (err[ref > 1e-30] <= 1e-5).all()
    assert ((cov >= 0) & (cov <= 1)).all()
    empty = ctx.band_coverage(torch.from_numpy(np.ascontiguousarray(p32[:, :0])).cuda(), sid)
    assert tuple(empty.shape) == (0, 16)
    p32[11, :3] = [0.0, -1.0, np.nan]
    cov2 = ctx.band_coverage(torch.from_numpy(p32).cuda(), sid).cpu().numpy()
    if rest:
        assert np.isfinite(cov2).all()
    else:
        assert np.isnan(cov2[:3]).all() and np.isfinite(cov2[3:]).all()
    ctx.close()


# Coverage floor of the ordinary tolerance.  The library interpolates the
# filter (tabulated on the grid's ln lam spacing) with four points, the oracle
# linearly in lam between the filter's own table points; the two differ where
# the grid reaches only the last few table points of a filter's far tail.  In
# this sweep every band with coverage >= 1e-9 is within 7e-5 mag in both
# forms, while bands below it reach 0.19 mag; a band with coverage 0 can get
# a finite magnitude (~70 mag) from the stencil's reach one grid step past
# the filter's end.
COV_FLOOR = 1e-8


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_bands_with_coverage_meet_the_oracle_tolerance(prec, tol):
    """Redshifts 2 to 9.9 move the grid's blue end across sixteen filters
    3300-11000 A: a band reached only through a filter's far tail has small
    coverage, and every band at or above the coverage floor is within the
    form's tolerance of the oracle; bands whose finiteness differs from the
    oracle's have coverage below 1e-12."""
    from paper_2112_06830_gb300 import dsps
    g = _util.ssp("full")
    ctx = dsps.Context(g, sfh_model=synth.SFH_DPL_QUENCH)
    tables = synth.make_filters(16, 3300.0, 11000.0)
    sid = ctx.add_filters(tables)
    p = synth.make_population(synth.SFH_DPL_QUENCH, 160, 8)
    p[11] = np.linspace(2.0, 9.9, 160)
    p32, p64 = _util.params_f32(p)
    x = torch.from_numpy(p32).cuda()
    m = ctx.photometry(x, sid, precision=prec).cpu().numpy().astype(np.float64)
    cov = ctx.band_coverage(x, sid).cpu().numpy().astype(np.float64)
    ref = oracle.mags(_util.oracle_grid("full", 1), oracle.Filters(tables), p64)
    fin = np.isfinite(ref)
    bad = np.isfinite(m) != fin
    for g_, q_ in zip(*np.nonzero(bad)):
        print(f"prec={prec} finiteness differs: z={p32[11, g_]:.4f} q={q_} mag {m[g_, q_]} oracle {ref[g_, q_]} "
              f"coverage {cov[g_, q_]:.3e}")
    assert (cov[bad] < 1e-12).all()
    fin &= ~bad
    err = np.where(fin, np.abs(m - np.where(fin, ref, 0.0)), 0.0)
    edges = [0.0, 1e-9, 1e-8, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 0.1, 1.01]
    for a, b in zip(edges[:-1], edges[1:]):
        sel = fin & (cov >= a) & (cov < b)
        if sel.any():
            print(f"prec={prec} coverage [{a:.0e}, {b:.0e}): {sel.sum():4d} bands, max |dm| {err[sel].max():.2e}")
    ok = fin & (cov >= COV_FLOOR)
    assert ok.sum() > 100
    assert (err[ok] <= tol).all(), (err[ok].max(), cov[ok][np.argmax(err[ok])])
    ctx.close()
