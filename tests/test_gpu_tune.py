"""The tile-height table (bf_tune_*) and its autotuner (tune.py) on the GPU.

The tile height of the windowed kernels only changes how the work is cut into
CTA tiles, never a pixel's arithmetic, so every tuned launch must give exactly
the bytes of the untuned one: for an image alone and in a persistent batch, on
the tensor-core and the FP32 kernels, at every height the tuner may pick.  The
tuner itself must keep the height it measured fastest, and a cache it saved
must restore the same table."""
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
    _bf.bf_tune_clear()
    yield _bf
    _bf.bf_tune_clear()


def _run(bf, items, variant):
    sp = torch.cuda.current_stream().cuda_stream
    outs = []
    calls = []
    for plan, x in items:
        y = bf.pitched_empty(plan.d, x.shape[1], x.shape[2])
        y.fill_(float("nan"))
        outs.append(y)
        calls.append((plan, x.data_ptr(), y.data_ptr(), x.shape[1], x.shape[2], x.stride(1)))
    if len(calls) == 1:
        bf.bf_filter(*calls[0], variant, sp)
    else:
        bf.bf_filter_batch(calls, variant, sp)
    torch.cuda.synchronize()
    assert bf.bf_last_status(sp) == bf.BF_OK
    return [y.cpu().numpy() for y in outs]


def _images(bf, specs, d=3):
    items = []
    for i, (H, W, s, K) in enumerate(specs):
        f = synth.voronoi_image(H, W, d, 9, 10.0, seed=1300 + i)
        plan = bf.bf_plan(d, synth.spd_cond(d, seed=1310 + i), s, 10, K, 1320 + i)
        items.append((plan, bf.to_pitched(f)))
    return items


@pytest.mark.parametrize("variant", ["fp16tc", "bf16tc", "fp32"])
@pytest.mark.parametrize("sigma", [2.0, 8.0, 10.5])
def test_tuned_alone_is_bit_identical(bf, variant, sigma):
    from paper_1605_02164_gb300 import tune
    v = bf.VARIANTS[variant]
    (plan, x), = _images(bf, [(211, 333, sigma, 24)])
    bf.bf_tune_clear()
    ref = _run(bf, [(plan, x)], v)[0]
    assert np.isfinite(ref).all()
    cls = bf.bf_tune_size_class(211, 333)
    try:
        for rows in tune.candidates(v, plan.r, 211):
            bf.bf_tune_set(v, 3, plan.r, cls, bf.BF_TUNE_ALONE, rows)
            got = _run(bf, [(plan, x)], v)[0]
            assert np.array_equal(got, ref), (variant, sigma, rows)
    finally:
        bf.bf_tune_clear()


@pytest.mark.parametrize("variant", ["fp16tc", "fp32"])
def test_tuned_batch_is_bit_identical(bf, variant):
    """Uneven batch (three radius classes, ragged sizes): each image's class
    takes a different height; the batch must equal the untuned batch and the
    per-image calls."""
    v = bf.VARIANTS[variant]
    specs = [(300, 517, 2.0, 32), (129, 64, 5.0, 16), (70, 901, 8.0, 24), (257, 255, 10.0, 16)]
    items = _images(bf, specs)
    bf.bf_tune_clear()
    ref = _run(bf, items, v)
    alone = [_run(bf, [it], v)[0] for it in items]
    for a, b in zip(ref, alone):
        assert np.array_equal(a, b)
    heights = [16, 48, 32, 64]
    try:
        for (plan, x), rows in zip(items, heights):
            cls = bf.bf_tune_size_class(x.shape[1], x.shape[2])
            bf.bf_tune_set(v, 3, plan.r, cls, bf.BF_TUNE_BATCH, rows)
        got = _run(bf, items, v)
        for k, (a, b) in enumerate(zip(got, ref)):
            assert np.array_equal(a, b), (variant, k)
    finally:
        bf.bf_tune_clear()


@pytest.mark.parametrize("variant", ["fp32", "fp16tc"])
def test_tuned_d6_is_bit_identical(bf, variant):
    """Six channels: the FP32 kernel, and the tensor-core kernel whose region
    codes use one affine map per image, so the tiling cannot change them."""
    v = bf.VARIANTS[variant]
    specs = [(150, 190, 4.0, 16), (90, 77, 9.0, 16)]
    items = _images(bf, specs, d=6)
    bf.bf_tune_clear()
    ref = _run(bf, items, v)
    alone = [_run(bf, [it], v)[0] for it in items]
    try:
        for rows in (16, 32, 48):
            for plan, x in items:
                bf.bf_tune_set(v, 6, plan.r, bf.bf_tune_size_class(x.shape[1], x.shape[2]), bf.BF_TUNE_BATCH, rows)
            got = _run(bf, items, v)
            for a, b, c in zip(got, ref, alone):
                assert np.array_equal(a, b) and np.array_equal(a, c), rows
    finally:
        bf.bf_tune_clear()


def test_tuner_keeps_the_fastest_and_cache_restores_it(bf, tmp_path):
    from paper_1605_02164_gb300 import tune
    bf.bf_tune_clear()
    try:
        cache = tune.TuneCache(str(tmp_path / "t.json"))
        keys = [(bf.BF_FP16TC, 3, 9, 700, 1000, bf.BF_TUNE_ALONE), (bf.BF_FP32, 3, 6, 700, 1000, bf.BF_TUNE_BATCH)]
        summary = cache.ensure(keys, K=8, reps=3, copies=2)
        assert summary["tuned"] == 2 and len(cache.entries) == 2
        assert bf.bf_tune_count() == sum(rec["rows"] > 0 for rec in cache.entries.values())
        for rec in cache.entries.values():
            t = {int(k): v for k, v in rec["timings"].items()}
            assert sorted(t) == [0] + tune.candidates(rec["variant"], rec["r"], rec["H"], rec["d"])
            best = min(t, key=t.get)
            if best != 0 and t[best] > 0.99 * t[0]:
                best = 0  # a measured height must beat the cost model (rows 0) by 1 %
            assert rec["rows"] == best
            assert bf.bf_tune_get(rec["variant"], rec["d"], rec["r"], rec["size_class"], rec["context"]) == rec["rows"]
        cache.save()
        assert cache.ensure(keys)["tuned"] == 0        # nothing new to time
        bf.bf_tune_clear()
        again = tune.TuneCache(cache.path)
        assert again.apply() == 2 and bf.bf_tune_count() == sum(r["rows"] > 0 for r in cache.entries.values())
        for rec in cache.entries.values():
            assert bf.bf_tune_get(rec["variant"], rec["d"], rec["r"], rec["size_class"], rec["context"]) == rec["rows"]
    finally:
        bf.bf_tune_clear()
