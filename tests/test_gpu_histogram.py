"""The benchmark's population statistic (Sec. 5.1: colour cut, then a
histogram of the r-band magnitude of the selected galaxies): the binning
kernel bit-exact against the same FP32 arithmetic in numpy; the fused path
(magnitudes binned where they are formed) against binning the magnitudes the
photometry returns; and the counts against the oracle's, where only galaxies
within the magnitude tolerance of the cut or of a bin edge may move."""
import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_2112_06830_gb300 import dsps
    c = dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH)
    f = synth.make_filters(12)
    return c, c.add_filters(f), oracle.Filters(f)


def _spec(m, n_bins=40, a=2, b=6, r=5):
    from paper_2112_06830_gb300 import dsps
    col = m[:, a] - m[:, b]
    lo, hi = np.percentile(m[:, r], [2, 98])
    return dsps.dsps_hist_spec(a, b, float(np.median(col)), r, float(lo), float(hi), n_bins)


def _numpy_f32(m, s):
    """The library's binning in float32 arithmetic."""
    m = m.astype(np.float32)
    colour = m[:, s.band_a] - m[:, s.band_b]
    r = m[:, s.band_r]
    lo, hi = np.float32(s.lo), np.float32(s.hi)
    scale = np.float32(s.n_bins / (float(np.float32(s.hi)) - float(np.float32(s.lo))))
    with np.errstate(invalid="ignore"):
        sel = (colour > np.float32(s.cut)) & (r >= lo) & (r < hi)
    b = np.minimum(((r[sel] - lo) * scale).astype(np.int64), s.n_bins - 1)
    return np.bincount(b, minlength=s.n_bins)


def test_histogram_kernel_is_exact(full):
    ctx, _, _ = full
    rng = np.random.default_rng(2)
    m = rng.normal(22.0, 1.5, (200_000, 12)).astype(np.float32)
    m[::997, 3] = np.nan
    s = _spec(m)
    got = ctx.histogram(torch.from_numpy(m).cuda(), s).cpu().numpy()
    np.testing.assert_array_equal(got, _numpy_f32(m, s))


@pytest.mark.parametrize("prec", [0, 1])
def test_fused_histogram_equals_binning_the_magnitudes(full, prec):
    ctx, sid, _ = full
    p32, _ = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, 100_000, 1))
    x = torch.from_numpy(p32).cuda()
    m = ctx.photometry(x, sid, precision=prec)
    s = _spec(m.cpu().numpy())
    fused = ctx.photometry_histogram(x, sid, s, precision=prec).cpu().numpy()
    np.testing.assert_array_equal(fused, ctx.histogram(m, s).cpu().numpy())
    assert fused.sum() > 10_000


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_histogram_matches_oracle(full, prec, tol):
    ctx, sid, F = full
    p32, p64 = _util.params_f32(synth.make_population(synth.SFH_DPL_QUENCH, 3000, 1, start=60_000))
    ref_m = oracle.mags(_util.oracle_grid("full", 1), F, p64)
    s = _spec(ref_m, n_bins=25)
    got = ctx.photometry_histogram(torch.from_numpy(p32).cuda(), sid, s, precision=prec).cpu().numpy()
    ref = oracle.colour_cut_histogram(ref_m, s.band_a, s.band_b, s.cut, s.band_r, s.lo, s.hi, s.n_bins)
    edges = np.linspace(s.lo, s.hi, s.n_bins + 1)
    colour = ref_m[:, s.band_a] - ref_m[:, s.band_b]
    r = ref_m[:, s.band_r]
    near = (np.abs(colour - s.cut) <= 2 * tol) | (np.abs(r[:, None] - edges[None, :]).min(axis=1) <= tol)
    l1 = int(np.abs(got - ref).sum())
    print(f"prec={prec}: selected {ref.sum()} of 3000, |gpu - oracle|_1 = {l1}, galaxies near an edge {near.sum()}")
    assert l1 <= 2 * int(near.sum())
