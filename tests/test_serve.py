"""The request loop: continuous batching gives every request the same result
it gets alone, admission respects the memory budget, and a request larger than
the whole budget is rejected with BF_ERR_BUDGET."""
import threading
import time

import numpy as np
import pytest

from paper_1605_02164_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def bf():
    from paper_1605_02164_gb300 import bf as _bf
    from paper_1605_02164_gb300 import build
    build.build()
    _bf.lib()
    return _bf


def _requests(bf, n, seed):
    from paper_1605_02164_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        H, W = int(rng.integers(40, 300)), int(rng.integers(40, 300))
        # grayscale requests go through the FP32 kernel in the same batch, six-channel
        # ones through the tensor cores' six-channel launch
        d = (1, 3, 6, 3)[i % 4]
        s = float(rng.uniform(1.0, 6.0))
        sr = float(rng.uniform(20, 60))
        f = synth.voronoi_image(H, W, d, 6, 10.0, seed=seed * 100 + i)
        reqs.append(Request(bf.to_pitched(f), np.diag([sr * sr] * d), s, int(rng.choice([16, 32])), 10,
                            seed=seed + i, rid=i))
    return reqs


def _alone(bf, r, variant):
    p = bf.bf_plan(r.x.shape[0], r.C, r.sigma_s, r.N, r.K, r.seed)
    v = variant if r.x.shape[0] in (3, 6) else bf.BF_FP32  # the server's routing
    y = bf.filter_tensor(p, r.x, v)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("variant", ["fp16tc", "fp32"])
def test_results_same_alone_and_in_the_mix(bf, variant):
    from paper_1605_02164_gb300.serve import Server
    v = bf.VARIANTS[variant]
    reqs = _requests(bf, 16, seed=7)
    srv = Server(budget_bytes=64 << 20, streams=2, max_batch=5, variant=v).start()

    def client(rs):
        for r in rs:
            srv.submit(r)
            time.sleep(0.002)  # arrivals interleave with batches already on the GPU

    ts = [threading.Thread(target=client, args=(reqs[k::2],)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for r in reqs:
        assert r.done_evt.wait(120)
    srv.close()
    assert srv.batches >= 2
    assert all(r.status == 0 for r in reqs)
    for r in reqs:
        assert np.array_equal(r.out.cpu().numpy(), _alone(bf, r, v)), r.rid
    assert bf.bf_last_status(0) == bf.BF_OK


def test_budget_admission_and_rejection(bf):
    from paper_1605_02164_gb300.serve import Request, Server, summarize
    reqs = _requests(bf, 6, seed=3)
    one = max(r.x.shape[0] * r.x.shape[1] * r.x.stride(1) * 4 for r in reqs)
    srv = Server(budget_bytes=one, streams=2, max_batch=8).start()  # at most one large request in flight
    big = Request(bf.to_pitched(synth.voronoi_image(400, 400, 3, 4, 10.0, seed=1)), np.diag([900.0] * 3),
                  2.0, 8, 10, seed=1, rid=99)
    t0 = time.perf_counter()
    for r in reqs:
        srv.submit(r)
    if big.x.shape[0] * big.x.shape[1] * big.x.stride(1) * 4 > one:
        srv.submit(big)
        assert big.status == bf.BF_ERR_BUDGET
    for r in reqs:
        assert r.done_evt.wait(120)
    srv.close()
    s = summarize(reqs, t0, time.perf_counter())
    assert s["completed"] == len(reqs) and s["failed"] == 0
    assert srv.used == 0


def test_wide_window_rejected_alone_and_recursive_request_served(bf):
    """A request whose window exceeds the windowed kernels (sigma_s = 12, r = 36)
    is rejected by itself with BF_ERR_UNSUPPORTED; the same request asking for
    the recursive variant is served and equals a lone call; the rest of the
    batch completes."""
    from paper_1605_02164_gb300.serve import Request, Server
    reqs = _requests(bf, 4, seed=11)
    f = synth.voronoi_image(90, 70, 3, 6, 10.0, seed=3)
    C = np.diag([40.0 ** 2] * 3)
    wide = Request(bf.to_pitched(f), C, 12.0, 16, 10, seed=5, rid=50)
    wide_rec = Request(bf.to_pitched(f), C, 12.0, 16, 10, seed=5, rid=51, variant=bf.BF_FP32_RECURSIVE)
    srv = Server(budget_bytes=64 << 20, streams=2, max_batch=8).start()
    for r in reqs + [wide, wide_rec]:
        srv.submit(r)
    assert wide.status == bf.BF_ERR_UNSUPPORTED and wide.done_evt.is_set()
    for r in reqs + [wide_rec]:
        assert r.done_evt.wait(120)
    srv.close()
    assert all(r.status == 0 for r in reqs) and wide_rec.status == 0
    p = bf.bf_plan(3, C, 12.0, 10, 16, 5)
    alone = bf.filter_tensor(p, wide_rec.x, bf.BF_FP32_RECURSIVE)
    torch.cuda.synchronize()
    assert torch.equal(alone, wide_rec.out)
    assert srv.used == 0


def test_cancelled_request_is_not_run(bf):
    """A request withdrawn while still queued completes with CANCELLED, no
    output and no budget held; cancelling an admitted or finished request is
    refused; the other requests are served and equal lone calls."""
    from paper_1605_02164_gb300.serve import CANCELLED, Server, summarize
    reqs = _requests(bf, 5, seed=21)
    srv = Server(budget_bytes=64 << 20, streams=2, max_batch=8)  # not started: everything stays queued
    for r in reqs:
        srv.submit(r)
    victim = reqs[2]
    assert srv.cancel(victim)
    assert victim.status == CANCELLED and victim.done_evt.is_set() and victim.out is None
    assert not srv.cancel(victim)
    t0 = time.perf_counter()
    srv.start()
    rest = [r for r in reqs if r is not victim]
    for r in rest:
        assert r.done_evt.wait(120)
    assert not srv.cancel(rest[0])  # finished
    srv.close()
    s = summarize(reqs, t0, time.perf_counter())
    assert s["completed"] == len(rest) and s["cancelled"] == 1 and s["failed"] == 0
    assert srv.used == 0 and srv.cancelled == [victim]
    for r in rest:
        assert np.array_equal(r.out.cpu().numpy(), _alone(bf, r, bf.BF_FP16TC)), r.rid


def test_input_produced_on_the_submitting_stream(bf):
    """A request whose input is still being written on the caller's stream when
    it is submitted (no synchronisation in between): the batch waits for that
    work, so the result equals filtering the finished input alone."""
    from paper_1605_02164_gb300.serve import Server
    v = bf.BF_FP16TC
    ref = _requests(bf, 6, seed=11)
    srcs = [r.x.clone() for r in ref]
    torch.cuda.synchronize()
    producer = torch.cuda.Stream()
    srv = Server(budget_bytes=64 << 20, streams=2, max_batch=3, variant=v).start()
    busy = torch.empty(4096, 4096, device="cuda")
    reqs = []
    with torch.cuda.stream(producer):
        for r, src in zip(ref, srcs):
            x = bf.pitched_empty(*src.shape)
            x.fill_(float("nan"))
            busy.normal_()
            busy = busy @ busy  # keeps the producer stream busy before the copy lands
            x.copy_(src)
            reqs.append(srv.submit(type(r)(x, r.C, r.sigma_s, r.K, r.N, seed=r.seed, rid=r.rid)))
    for r in reqs:
        assert r.done_evt.wait(120)
    srv.close()
    assert all(r.status == 0 for r in reqs)
    for r, r0 in zip(reqs, ref):
        assert np.array_equal(r.out.cpu().numpy(), _alone(bf, r0, v)), r.rid


def test_loop_with_tuning_cache_gives_untuned_results(bf, tmp_path):
    """A server started with a tuning cache applies it (every class of the
    trace gets 16-row tiles, far from the cost model's choice) and still
    returns each request's untuned, alone result bit for bit."""
    from paper_1605_02164_gb300.serve import Server
    from paper_1605_02164_gb300.tune import TuneCache
    v = bf.BF_FP16TC
    reqs = _requests(bf, 10, seed=11)
    bf.bf_tune_clear()
    expect = [_alone(bf, r, v) for r in reqs]
    cache = TuneCache(str(tmp_path / "tune.json"))
    for r in reqs:
        d, H, W = r.x.shape
        rad = int(np.floor(3.0 * r.sigma_s + 1e-9))
        cls = bf.bf_tune_size_class(H, W)
        for var in (bf.BF_FP16TC, bf.BF_FP32):
            for ctx in (bf.BF_TUNE_ALONE, bf.BF_TUNE_BATCH):
                cache.entries[cache.key(var, d, rad, cls, ctx)] = {"variant": var, "d": d, "r": rad,
                                                                  "size_class": cls, "context": ctx, "rows": 16}
    cache.save()
    try:
        srv = Server(budget_bytes=64 << 20, streams=2, max_batch=4, variant=v, tune_cache=cache.path).start()
        assert srv.tuned_entries == len(cache.entries) == bf.bf_tune_count()
        for r in reqs:
            srv.submit(r)
        for r in reqs:
            assert r.done_evt.wait(120)
        srv.close()
        for r, e in zip(reqs, expect):
            assert r.status == 0 and np.array_equal(r.out.cpu().numpy(), e), r.rid
    finally:
        bf.bf_tune_clear()
