"""Parity of the tabulated star formation history (Sec. 3.1: the SFR given at
the cosmic-time nodes, the last n_t parameter rows) between the CUDA path and
the FP64 oracle: magnitudes in both precision forms over several tiles and a
ragged tail, the gradient (rows 5..10 and the n_t node rows), a table holding a
parametric model's node values against that model, invalid tables, batch
invariance, the request loop and the autograd row mapping.

Gradient tolerance: as for the parametric rows, |g - g_oracle| <= 1e-3
max(|g_oracle|, f max|g_oracle|) with f = 1e-3 (FP32) or 1e-2 (split-bf16),
the maximum taken per galaxy over the block (rows 5..10, or the node rows,
whose units are those of 1/SFR)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2112_06830_gb300 import synth

import _util

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_T = synth.FULL_GRID.n_t


@functools.lru_cache(maxsize=None)
def _ogrid():
    g = _util.ssp("full")
    return oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=oracle.SFH_TABLE)


@pytest.fixture(scope="module")
def table_ctx():
    from paper_2112_06830_gb300 import dsps
    c = dsps.Context(_util.ssp("full"), sfh_model=dsps.DSPS_SFH_TABLE)
    f = synth.make_filters(12)
    yield c, c.add_filters(f), oracle.Filters(f)
    c.close()


def _pop(n, seed, start=0):
    p = synth.make_population(synth.SFH_DPL_QUENCH, n, seed, start)
    return _util.params_f32(synth.with_sfr_table(p, N_T, seed, start))


def _scaled_error(g, ref, rows, floor):
    r, x = ref[rows], g[rows]
    scale = np.maximum(np.abs(r), floor * np.abs(r).max(axis=0, keepdims=True))
    ok = scale > 0
    rel = np.zeros_like(r)
    rel[ok] = np.abs(x - r)[ok] / scale[ok]
    rel[~ok] = np.abs(x[~ok])
    return rel


def test_rows(table_ctx):
    ctx, _, _ = table_ctx
    assert (ctx.npar, ctx.ngrad) == (12 + N_T, 11 + N_T) == (_ogrid().npar, _ogrid().ngrad)


@pytest.mark.parametrize("prec,tol", [(0, _util.TOL_FP32), (1, _util.TOL_BF16X3)])
def test_photometry_matches_oracle(table_ctx, prec, tol):
    ctx, sid, F = table_ctx
    n = 700                      # five full 128-row tiles and a ragged tail
    p32, p64 = _pop(n, 41)
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid, precision=prec).cpu().numpy().astype(np.float64)
    idx = np.r_[0:8, 250:258, 690:700]
    ref = oracle.mags(_ogrid(), F, p64[:, idx])
    err = np.abs(m[idx] - ref)
    print(f"tabulated SFH prec={prec}: max |dm| = {err.max():.3e}")
    assert err.max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_gradients_match_oracle(table_ctx, prec):
    ctx, sid, F = table_ctx
    n = 150
    p32, p64 = _pop(n, 42, 900)
    mbar = np.random.default_rng(13).standard_normal((n, 12))
    _, pb = ctx.photometry_vjp(torch.from_numpy(p32).cuda(), sid, torch.from_numpy(mbar.astype(np.float32)).cuda(),
                               precision=prec)
    pb = pb.cpu().numpy().astype(np.float64)
    assert pb.shape == (11 + N_T, n)
    idx = np.r_[0:6, 128:134, 144:150]
    _, ref = oracle.mags_vjp(_ogrid(), F, p64[:, idx], mbar[idx])
    g = pb[:, idx]
    assert np.all(g[:5] == 0.0)                     # rows 0..4 are unused
    floor = {0: 1e-3, 1: 1e-2}[prec]
    rel_p = _scaled_error(g, ref, slice(5, 11), floor)
    rel_t = _scaled_error(g, ref, slice(11, 11 + N_T), floor)
    print(f"tabulated SFH prec={prec}: max scaled gradient error {rel_p.max():.2e} (rows 5-10), "
          f"{rel_t.max():.2e} (node rows)")
    assert rel_p.max() <= 1e-3 and rel_t.max() <= 1e-3


def test_table_of_a_parametric_model_matches_it(table_ctx):
    from paper_2112_06830_gb300 import dsps
    ctx, sid, _ = table_ctx
    par = dsps.Context(_util.ssp("full"), sfh_model=dsps.DSPS_SFH_DPL_QUENCH)
    sid_p = par.add_filters(synth.make_filters(12))
    p = synth.make_population(synth.SFH_DPL_QUENCH, 200, 43)
    g = _ogrid()
    t = g.t0 + np.arange(g.n_t) * (g.t1 - g.t0) / (g.n_t - 1)
    tab = np.array([[oracle.sfr(synth.SFH_DPL_QUENCH, p[:, k], tn)[0] for tn in t] for k in range(200)])
    q = np.zeros((12 + N_T, 200))
    q[:12] = p
    q[12:] = tab.T
    p32, _ = _util.params_f32(p)
    q32, _ = _util.params_f32(q)
    for prec, tol in ((0, 2e-5), (1, 2e-4)):
        m_t = ctx.photometry(torch.from_numpy(q32).cuda(), sid, precision=prec)
        m_p = par.photometry(torch.from_numpy(p32).cuda(), sid_p, precision=prec)
        assert (m_t - m_p).abs().max().item() <= tol
    par.close()


def test_invalid_tables_and_nodes_after_the_observation(table_ctx):
    from paper_2112_06830_gb300 import dsps
    ctx, sid, _ = table_ctx
    p32, _ = _pop(40, 44)
    p32[11, :] = 1.0                     # t_obs about 5.9 Gyr: node 90 lies after it
    p32[12 + 5, 3] = -1.0                # negative SFR before t_obs
    p32[12 + 2, 7] = np.nan              # NaN before t_obs
    p32[12:, 9] = 0.0                    # no mass formed
    p32[12 + 150, 11] = np.nan           # after t_obs: ignored
    p32[0:5, 12] = np.nan                # rows 0..4: ignored
    m = ctx.photometry(torch.from_numpy(p32).cuda(), sid).cpu().numpy()
    bad = np.zeros(40, bool)
    bad[[3, 7, 9]] = True
    assert np.all(np.isnan(m[bad])) and np.all(np.isfinite(m[~bad]))
    assert ctx.device_error() == dsps.DSPS_ERR_INVALID_ARG
    assert ctx.device_error() == 0
    q = p32.copy()
    q[12 + 150:, :] = 1e3                # any values after t_obs
    q[0:5, :] = 7.0
    m2 = ctx.photometry(torch.from_numpy(q).cuda(), sid).cpu().numpy()
    assert np.array_equal(m2[~bad], m[~bad])


def test_batch_invariance_request_loop_and_autograd():
    from paper_2112_06830_gb300 import autograd, dsps
    big = dsps.Context(_util.ssp("full"), sfh_model=dsps.DSPS_SFH_TABLE)
    small = dsps.Context(_util.ssp("full"), sfh_model=dsps.DSPS_SFH_TABLE, max_chunk=256)
    f = synth.make_filters(8)
    sb, ss = big.add_filters(f), small.add_filters(f)
    p32, _ = _pop(600, 45)
    p = torch.from_numpy(p32).cuda()
    mb = np.random.default_rng(14).standard_normal((600, 8)).astype(np.float32)
    for prec in (0, 1):
        m1, g1 = big.photometry_vjp(p, sb, torch.from_numpy(mb).cuda(), precision=prec)
        m2, g2 = small.photometry_vjp(p, ss, torch.from_numpy(mb).cuda(), precision=prec)
        assert torch.equal(m1, m2) and torch.equal(g1, g2)
    t = big.submit(p32, sb, precision=1, mag_bar=mb)
    while big.poll(t, 100000) in (dsps.DSPS_PENDING, dsps.DSPS_ERR_TIMEOUT):
        pass
    m, g = big.photometry_vjp(p, sb, torch.from_numpy(mb).cuda(), precision=1)
    assert np.array_equal(t.mags, m.cpu().numpy()) and np.array_equal(t.param_bar, g.cpu().numpy())
    x = p.clone().requires_grad_(True)
    out = autograd.photometry(big, x, sb, precision=1)
    out.backward(torch.from_numpy(mb).cuda())
    assert torch.equal(x.grad[:11], g[:11]) and torch.equal(x.grad[12:], g[11:])
    assert torch.all(x.grad[11] == 0)
    big.close()
    small.close()


def test_weights_and_the_static_entry(table_ctx):
    import ctypes
    from paper_2112_06830_gb300 import dsps
    ctx, sid, _ = table_ctx
    p32, p64 = _pop(300, 46)
    d = torch.from_numpy(p32).cuda()
    w = ctx.weights(d).cpu().numpy().astype(np.float64)
    idx = [0, 1, 2, 150, 298, 299]
    ref = oracle.weights(_ogrid(), p64[:, idx])
    mass = 10.0 ** p64[10, idx]
    err = np.abs(w[idx] - ref)
    assert (err <= 2e-5 * np.abs(ref) + 1e-6 * mass[:, None, None]).all(), err.max()
    # the allocation-free FP32 entry on the same table
    lib = dsps.load()
    out = torch.full((300, 12), float("nan"), device="cuda")
    rc = lib.dsps_photometry_fp32_static(ctx.handle, 300, ctypes.c_void_p(d.data_ptr()), sid,
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == dsps.DSPS_OK, lib.dsps_last_error_message()
    want = ctx.photometry(d, sid, precision=dsps.DSPS_PREC_FP32)
    assert (out - want).abs().max().item() <= _util.TOL_FP32
