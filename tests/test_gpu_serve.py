"""The request loop (dsps_submit / dsps_poll): a mixed stream of populations of
different sizes, filter sets and gradient requests, submitted concurrently,
gives each request the same result as a lone call; admission respects the HBM
budget; host-side fault injection fails only the affected batch."""
import os
import threading

import numpy as np
import pytest

import _util
from paper_2112_06830_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(**kw):
    from paper_2112_06830_gb300 import dsps
    return dsps.Context(_util.ssp("full"), sfh_model=synth.SFH_DPL_QUENCH, **kw)


def _requests(n_req, seed, max_gal=30_000):
    rng = np.random.default_rng(seed)
    pool = synth.make_population(synth.SFH_DPL_QUENCH, 120_000, 11).astype(np.float32)
    out = []
    for i in range(n_req):
        g = int(np.clip(np.round(3e3 * np.exp(1.5 * rng.standard_normal())), 100, max_gal))
        s0 = int(rng.integers(0, pool.shape[1] - g))
        q = int(rng.choice([4, 8, 12]))
        grad = bool(rng.uniform() < 0.3)
        prec = 1 if rng.uniform() < 0.8 else 0
        out.append((np.ascontiguousarray(pool[:, s0:s0 + g]), q, grad, prec,
                    rng.standard_normal((g, q)).astype(np.float32)))
    return out


def _direct(ctx, sids, req):
    p, q, grad, prec, mbar = req
    dp = torch.from_numpy(p).cuda()
    if grad:
        m, pb = ctx.photometry_vjp(dp, sids[q], torch.from_numpy(mbar).cuda(), precision=prec)
        torch.cuda.synchronize()
        return m.cpu().numpy(), pb.cpu().numpy()
    m = ctx.photometry(dp, sids[q], precision=prec)
    torch.cuda.synchronize()
    return m.cpu().numpy(), None


def _run_stream(ctx, sids, reqs, n_threads=4):
    from paper_2112_06830_gb300 import dsps
    tickets = [None] * len(reqs)

    def worker(k):
        for i in range(k, len(reqs), n_threads):
            p, q, grad, prec, mbar = reqs[i]
            tickets[i] = ctx.submit(p, sids[q], precision=prec, mag_bar=mbar if grad else None)

    th = [threading.Thread(target=worker, args=(k,)) for k in range(n_threads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    rcs = [ctx.poll(t, timeout_us=60_000_000) for t in tickets]
    assert all(rc in (dsps.DSPS_OK,) for rc in rcs), rcs
    return tickets


def test_mixed_stream_equals_lone_calls():
    ctx = _ctx()
    sids = {q: ctx.add_filters(synth.make_filters(q)) for q in (4, 8, 12)}
    reqs = _requests(36, 0)
    tickets = _run_stream(ctx, sids, reqs)
    for req, t in zip(reqs, tickets):
        m, pb = _direct(ctx, sids, req)
        np.testing.assert_array_equal(t.mags, m)
        if req[2]:
            np.testing.assert_array_equal(t.param_bar, pb)
        assert t.latency_us is not None and t.latency_us > 0
    assert ctx.device_error() == 0


def test_requests_larger_than_one_piece():
    ctx = _ctx()
    sids = {12: ctx.add_filters(synth.make_filters(12))}
    p = synth.make_population(synth.SFH_DPL_QUENCH, 150_000, 5).astype(np.float32)
    mbar = np.random.default_rng(0).standard_normal((150_000, 12)).astype(np.float32)
    (t,) = _run_stream(ctx, sids, [(p, 12, True, 1, mbar)], n_threads=1)
    m, pb = _direct(ctx, sids, (p, 12, True, 1, mbar))
    np.testing.assert_array_equal(t.mags, m)
    np.testing.assert_array_equal(t.param_bar, pb)


def test_admission_under_a_tiny_budget():
    from paper_2112_06830_gb300 import dsps
    # ~1 GB holds one or two batches at a time (a gradient galaxy needs ~45 KB)
    ctx = _ctx(hbm_budget_bytes=1 << 30, n_streams=4)
    sids = {q: ctx.add_filters(synth.make_filters(q)) for q in (4, 8, 12)}
    reqs = _requests(12, 1, max_gal=8_000)
    tickets = _run_stream(ctx, sids, reqs)
    for req, t in zip(reqs, tickets):
        np.testing.assert_array_equal(t.mags, _direct(ctx, sids, req)[0])
    # one piece of 65536 gradient galaxies needs ~3 GB: refused up front
    big = synth.make_population(synth.SFH_DPL_QUENCH, 70_000, 2).astype(np.float32)
    with pytest.raises(dsps.DSPSError) as ei:
        ctx.submit(big, sids[12], mag_bar=np.zeros((70_000, 12), np.float32))
    assert ei.value.code == dsps.DSPS_ERR_OUT_OF_BUDGET


def test_poll_of_unknown_ticket_and_pending():
    from paper_2112_06830_gb300 import dsps
    ctx = _ctx()
    sid = ctx.add_filters(synth.make_filters(12))
    t = ctx.submit(synth.make_population(synth.SFH_DPL_QUENCH, 2000, 3).astype(np.float32), sid)
    assert ctx.poll(t, timeout_us=30_000_000) == dsps.DSPS_OK
    with pytest.raises(dsps.DSPSError) as ei:
        ctx.poll(t)                       # already retired
    assert ei.value.code == dsps.DSPS_ERR_NOT_FOUND


def test_injected_batch_failure_is_contained():
    """A host-side injected failure of one batch (no GPU fault) fails exactly
    that batch's requests; the loop serves the rest."""
    from paper_2112_06830_gb300 import dsps
    os.environ["DSPS_SERVE_FAULT"] = "fail_batch:0"
    try:
        ctx = _ctx(n_streams=1)
        sid = ctx.add_filters(synth.make_filters(12))
        p = synth.make_population(synth.SFH_DPL_QUENCH, 3000, 4).astype(np.float32)
        t0 = ctx.submit(p, sid)
        with pytest.raises(dsps.DSPSError) as ei:
            ctx.poll(t0, timeout_us=30_000_000)
        assert ei.value.code == dsps.DSPS_ERR_CUDA
        t1 = ctx.submit(p, sid)
        assert ctx.poll(t1, timeout_us=30_000_000) == dsps.DSPS_OK
        np.testing.assert_array_equal(t1.mags, _direct(ctx, {12: sid}, (p, 12, False, 1, None))[0])
    finally:
        del os.environ["DSPS_SERVE_FAULT"]
