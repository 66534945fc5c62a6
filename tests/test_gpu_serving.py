"""Request API behaviour under load and failure, with the failures made on the
host: a host mesh step that reports an error, a full queue, a context
destroyed with work in flight.  No GPU fault is involved."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1511_00758_gb300 as S  # noqa: E402

PRM = dict(t_lo=4, t_hi=8, t_grad=8, t_fast=20, kp_per_bin=4, uniq_margin=2)


def _pairs(n, W=320, H=240, iters=3):
    return [scenes.make_pair("polygon", W, H, 900 + i, 48, iters, 16, n_poly=8) for i in range(n)]


def _solo(p):
    with S.Context(mem_budget_bytes=1 << 28, **PRM) as ctx:
        t = ctx.submit(p.left, p.right, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell)
        out = ctx.result_tensors(ctx.poll(t))
        ctx.release(t)
    return out


def test_injected_host_failure_is_reported_and_isolated():
    pairs = _pairs(5)
    with S.Context(mem_budget_bytes=1 << 29, max_slots=5, host_threads=2, inject_mesh_failure=4, **PRM) as ctx:
        ts = [ctx.submit(p.left, p.right, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell) for p in pairs]
        status, outs = [], []
        for t in ts:
            try:
                outs.append(ctx.result_tensors(ctx.poll(t)))
                status.append(0)
            except S.StereoError as e:
                status.append(e.code)
                outs.append(None)
            ctx.release(t)
    assert status.count(-6) == 1 and status.count(0) == 4
    for p, o in zip(pairs, outs):
        if o is not None:
            want = _solo(p)
            for k in ("D_f", "C_f", "mask", "planeidx"):
                assert torch.equal(o[k], want[k])


def test_device_wait_timeout_is_reported_and_context_recovers():
    """A bounded device-side wait that runs out: in the context's first GPU
    round with an iteration stage, the bulk-copy validate's producer issues no
    copy, so its consumers give up after a second and set the error flag.  The
    request fails with STEREO_E_TIMEOUT (-5) in seconds, and the next request
    on the same context equals its solo result."""
    import time
    pairs = _pairs(2)
    with S.Context(mem_budget_bytes=1 << 28, max_slots=1, inject_wait_timeout=1, **PRM) as ctx:
        t0 = time.time()
        tk = ctx.submit(pairs[0].left, pairs[0].right, 320, 240, pairs[0].dmax, pairs[0].iters, pairs[0].cell)
        with pytest.raises(S.StereoError) as e:
            ctx.poll(tk)
        assert e.value.code == -5
        assert time.time() - t0 < 30
        ctx.release(tk)
        tk = ctx.submit(pairs[1].left, pairs[1].right, 320, 240, pairs[1].dmax, pairs[1].iters, pairs[1].cell)
        got = ctx.result_tensors(ctx.poll(tk))
        ctx.release(tk)
    want = _solo(pairs[1])
    for k in ("D_f", "C_f", "mask", "planeidx"):
        assert torch.equal(got[k], want[k])


def test_batch_submit_matches_single_and_takes_a_prefix():
    """stereo_submit_batch: the pairs of a batch give the results they give when
    submitted alone, and one invalid pair rejects the whole batch."""
    pairs = _pairs(4)
    with S.Context(mem_budget_bytes=1 << 29, max_slots=4, host_threads=2, **PRM) as ctx:
        tks = ctx.submit_batch([(p.left, p.right, 320, 240, p.dmax, p.iters, p.cell) for p in pairs])
        assert len(tks) == 4
        outs = [ctx.result_tensors(ctx.poll(t)) for t in tks]
        for t in tks:
            ctx.release(t)
    for p, o in zip(pairs, outs):
        want = _solo(p)
        for k in ("D_f", "C_f", "mask", "planeidx"):
            assert torch.equal(o[k], want[k])
    with S.Context(mem_budget_bytes=1 << 29, max_slots=1, **PRM) as ctx:
        good = (pairs[0].left, pairs[0].right, 320, 240, 48, 2, 16)
        with pytest.raises(S.StereoError) as e:
            ctx.submit_batch([good, (pairs[1].left, pairs[1].right, 320, 240, 300, 2, 16)])
        assert e.value.code == -1
        assert ctx.stats().requests_done == 0


def test_poll_and_release_batch():
    """poll_batch waits for every ticket and reports each request's own result (the same as
    its single poll); release_batch frees them all; unknown tickets are reported."""
    pairs = [scenes.make_pair("polygon", 160, 120, 900 + i, 32, 2, 8, n_poly=6) for i in range(5)]
    with S.Context(mem_budget_bytes=1 << 29, max_slots=5, host_threads=2, **PRM) as ctx:
        tk = ctx.submit_batch([(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda(), 160, 120,
                                p.dmax, p.iters, p.cell) for p in pairs])
        res = ctx.poll_batch(tk)
        assert res is not None and len(res) == 5 and all(r.status == 0 and r.w == 160 for r in res)
        single = [ctx.poll(t) for t in tk]
        for a, b in zip(res, single):
            assert a.disparity == b.disparity and a.latency_ms == b.latency_ms
        with pytest.raises(S.StereoError):
            ctx.poll_batch(tk + [123456789])
        ctx.release_batch(tk)
        with pytest.raises(S.StereoError):
            ctx.poll(tk[0])  # released
        with pytest.raises(S.StereoError):
            ctx.release_batch(tk[:1])


def test_rounds_of_changing_pair_counts():
    """Rounds of 40, 5 and 24 pairs on one context: the device mesh launches of these rounds take
    clusters of 2, 8 and 4 blocks, so each round's graph differs from the last in its launch
    shape.  Every pair gives what it gives in a batch of its own kind on a fresh context."""
    sizes = (40, 5, 24)
    pairs = [scenes.make_pair("polygon", 160, 120, 950 + i, 32, 3, 8, n_poly=6) for i in range(sum(sizes))]
    batch = lambda ps: [(p.left, p.right, 160, 120, p.dmax, p.iters, p.cell) for p in ps]
    got = []
    with S.Context(mem_budget_bytes=1 << 31, max_slots=64, host_threads=2, **PRM) as ctx:
        o = 0
        for n in sizes:
            tk = ctx.submit_batch(batch(pairs[o:o + n]))
            assert len(tk) == n
            got += [ctx.result_tensors(r) for r in ctx.poll_batch(tk)]
            ctx.release_batch(tk)
            o += n
    with S.Context(mem_budget_bytes=1 << 31, max_slots=64, host_threads=2, **PRM) as ctx:
        tk = ctx.submit_batch(batch(pairs[:64]))
        want = [ctx.result_tensors(r) for r in ctx.poll_batch(tk)]
        ctx.release_batch(tk)
        tk = ctx.submit_batch(batch(pairs[64:]))
        want += [ctx.result_tensors(r) for r in ctx.poll_batch(tk)]
        ctx.release_batch(tk)
    for g, w in zip(got, want):
        for k in ("D_f", "C_f", "mask", "planeidx"):
            assert torch.equal(g[k], w[k])


def test_queue_full_returns_busy_then_drains():
    pairs = _pairs(8, 1242, 375)
    got_busy = 0
    with S.Context(mem_budget_bytes=1 << 29, max_slots=1, max_queue=1, **PRM) as ctx:
        ts = []
        for p in pairs:
            try:
                ts.append(ctx.submit(p.left, p.right, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell))
            except S.StereoError as e:
                assert e.code == -3
                got_busy += 1
        for t in ts:
            assert ctx.poll(t).status == 0
            ctx.release(t)
        assert ctx.stats().requests_done == len(ts)
    assert got_busy >= 1 and len(ts) >= 1


def test_destroy_with_work_in_flight():
    pairs = _pairs(6)
    ctx = S.Context(mem_budget_bytes=1 << 29, max_slots=3, host_threads=2, **PRM)
    for p in pairs:
        ctx.submit(p.left, p.right, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell)
    ctx.close()  # queued work is cancelled, in-flight work finishes, nothing leaks or hangs


def test_poll_timeout_and_unknown_ticket():
    p = _pairs(1, 1242, 375)[0]
    with S.Context(mem_budget_bytes=1 << 28, **PRM) as ctx:
        t = ctx.submit(p.left, p.right, 1242, 375, p.dmax, p.iters, p.cell)
        r = ctx.poll(t, timeout_us=0)  # almost surely still running: None, or done
        assert r is None or r.status == 0
        assert ctx.poll(t).status == 0
        with pytest.raises(S.StereoError) as e:
            ctx.release(t + 1000)
        assert e.value.code == -8
        ctx.release(t)
