"""Edge cases of the optional model forms through the C ABI: empty calls,
one galaxy and a ragged tile (129 rows) for the nebular axis (Sec. 3.3),
age-dependent dust (Sec. 3.4.1) and tabulated histories (Sec. 3.1), in the
forward, the gradient, spectra and line widths; a single galaxy gets the
magnitudes it gets inside a larger population."""
import functools

import numpy as np
import pytest

from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LC, HW, CW = synth.EW_LINE


@functools.lru_cache(maxsize=None)
def _ssp(kind):
    if kind == "nebular":
        return synth.make_ssp_nebular(synth.FULL_GRID, 1)
    return synth.with_emission_line(_util.ssp("full"))


def _case(kind):
    from paper_2112_06830_gb300 import dsps
    n_t = synth.FULL_GRID.n_t
    if kind == "nebular":
        ctx = dsps.Context(_ssp("nebular"), sfh_model=synth.SFH_DPL_QUENCH)
        make = lambda n, s: synth.with_nebular(synth.make_population(synth.SFH_DPL_QUENCH, n, s), s)
    elif kind == "agedep":
        ctx = dsps.Context(_ssp("line"), sfh_model=synth.SFH_DPL_QUENCH, dust_agedep=True)
        make = lambda n, s: synth.with_agedep_dust(synth.make_population(synth.SFH_DPL_QUENCH, n, s), s)
    else:
        ctx = dsps.Context(_ssp("line"), sfh_model=dsps.DSPS_SFH_TABLE)
        make = lambda n, s: synth.with_sfr_table(synth.make_population(synth.SFH_DPL_QUENCH, n, s), n_t, s)
    return ctx, make


@pytest.mark.parametrize("kind", ["nebular", "agedep", "table"])
def test_empty_single_and_ragged_calls(kind):
    ctx, make = _case(kind)
    sid = ctx.add_filters(synth.make_filters(6))
    lid = ctx.add_line(LC, HW, CW)
    p32 = make(300, 91).astype(np.float32)
    p = torch.from_numpy(p32).cuda()
    empty = torch.zeros((ctx.npar, 0), dtype=torch.float32, device="cuda")
    for prec in (0, 1):
        assert ctx.photometry(empty, sid, precision=prec).shape == (0, 6)
        m0, g0 = ctx.photometry_vjp(empty, sid, torch.zeros((0, 6), device="cuda"), precision=prec)
        assert m0.shape == (0, 6) and g0.shape == (ctx.ngrad, 0)
        full = ctx.photometry(p, sid, precision=prec)
        assert torch.isfinite(full).all()
        for n in (1, 129):
            part = ctx.photometry(p[:, :n].contiguous(), sid, precision=prec)
            assert torch.equal(part, full[:n]), (kind, prec, n)
        mb = torch.ones((129, 6), device="cuda")
        m, g = ctx.photometry_vjp(p[:, :129].contiguous(), sid, mb, precision=prec)
        assert torch.isfinite(m).all() and torch.isfinite(g).all() and g.shape == (ctx.ngrad, 129)
    assert ctx.spectra(empty, 0, 10).shape == (0, 10)
    assert ctx.line_ew(empty, lid).numel() == 0
    e0, g0 = ctx.line_ew_vjp(empty, lid, torch.zeros(0, device="cuda"))
    assert e0.numel() == 0 and g0.shape == (ctx.ngrad, 0)
    ew = ctx.line_ew(p, lid)
    assert torch.isfinite(ew).all()
    assert torch.equal(ctx.line_ew(p[:, :1].contiguous(), lid), ew[:1])
    e1, g1 = ctx.line_ew_vjp(p[:, :129].contiguous(), lid, torch.ones(129, device="cuda"))
    assert torch.isfinite(e1).all() and torch.isfinite(g1).all()
    assert ctx.device_error() == 0
    ctx.close()
