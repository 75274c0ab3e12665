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


def test_poll_timeout_pending_and_retry():
    """dsps_poll: a zero timeout on an unfinished request returns DSPS_PENDING,
    a positive timeout that elapses returns DSPS_ERR_TIMEOUT and leaves the
    ticket valid, and a later poll collects the result.  The completion is held
    back on the host (DSPS_SERVE_FAULT=delay_us); the GPU work is untouched."""
    from paper_2112_06830_gb300 import dsps
    os.environ["DSPS_SERVE_FAULT"] = "delay_us:1500000"
    try:
        ctx = _ctx(n_streams=1)
        sid = ctx.add_filters(synth.make_filters(12))
        p = synth.make_population(synth.SFH_DPL_QUENCH, 2500, 6).astype(np.float32)
        t = ctx.submit(p, sid)
        assert ctx.poll(t) == dsps.DSPS_PENDING
        assert ctx.poll(t, timeout_us=20_000) == dsps.DSPS_ERR_TIMEOUT
        assert ctx.poll(t, timeout_us=30_000_000) == dsps.DSPS_OK
        np.testing.assert_array_equal(t.mags, _direct(ctx, {12: sid}, (p, 12, False, 1, None))[0])
    finally:
        del os.environ["DSPS_SERVE_FAULT"]


def test_device_buffer_requests_mixed_with_host_requests():
    """Requests whose buffers are device memory (DSPS_BUF_DEVICE) ride in the
    same batches as host requests and give the lone call's results bit for bit;
    a device request holding a host pointer is refused."""
    from paper_2112_06830_gb300 import dsps
    ctx = _ctx()
    sids = {q: ctx.add_filters(synth.make_filters(q)) for q in (4, 8, 12)}
    reqs = _requests(16, 7)
    tickets = []
    for i, (p, q, grad, prec, mbar) in enumerate(reqs):
        if i % 2:
            tickets.append(ctx.submit(torch.from_numpy(p).cuda(), sids[q], precision=prec,
                                      mag_bar=torch.from_numpy(mbar).cuda() if grad else None))
        else:
            tickets.append(ctx.submit(p, sids[q], precision=prec, mag_bar=mbar if grad else None))
    assert all(ctx.poll(t, timeout_us=60_000_000) == dsps.DSPS_OK for t in tickets)
    for i, (req, t) in enumerate(zip(reqs, tickets)):
        m, pb = _direct(ctx, sids, req)
        got = t.mags.cpu().numpy() if i % 2 else t.mags
        np.testing.assert_array_equal(got, m)
        if req[2]:
            gpb = t.param_bar.cpu().numpy() if i % 2 else t.param_bar
            np.testing.assert_array_equal(gpb, pb)
    p = np.ascontiguousarray(reqs[0][0])
    out = torch.empty((p.shape[1], 12), dtype=torch.float32, device="cuda")
    bad = dsps.dsps_request(p.shape[1], p.ctypes.data, sids[12], 1, 0, None, out.data_ptr(), None,
                            dsps.DSPS_BUF_DEVICE)
    with pytest.raises(dsps.DSPSError) as ei:
        dsps.dsps_submit(ctx.handle, bad)
    assert ei.value.code == dsps.DSPS_ERR_INVALID_ARG
    assert ctx.device_error() == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_photometry_host_buffers_equal_device_call(prec):
    """dsps_photometry_host (host parameters in, host magnitudes out, one call)
    equals dsps_photometry on device buffers, with pageable and pinned host
    memory, and over several chunks of a small work space (ragged last chunk)."""
    from paper_2112_06830_gb300 import dsps
    ctx = dsps.Context(_util.ssp("small"), sfh_model=synth.SFH_DELAYED_TAU, max_chunk=256)
    sid = ctx.add_filters(synth.make_filters(6))
    p = synth.make_population(synth.SFH_DELAYED_TAU, 1000, 12).astype(np.float32)
    want = ctx.photometry(torch.from_numpy(p).cuda(), sid, precision=prec)
    torch.cuda.synchronize()
    want = want.cpu().numpy()
    got = ctx.photometry_host(p, sid, precision=prec)
    np.testing.assert_array_equal(got, want)
    pinned = torch.from_numpy(p).pin_memory()
    out = torch.empty((1000, 6), dtype=torch.float32).pin_memory()
    ctx.photometry_host(pinned, sid, precision=prec, out=out)
    np.testing.assert_array_equal(out.numpy(), want)
    assert ctx.device_error() == 0
    ctx.close()
