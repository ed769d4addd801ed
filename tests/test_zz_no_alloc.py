"""bf_filter_batch_noalloc, the entry point for callers that cannot let the
library allocate device memory at call time (their memory belongs to their own
allocator, or a cudaMalloc's synchronisation would stall a latency-critical
loop).  Its scratch is a static device array instead of library-allocated
memory.  Checked through the C ABI against bf_filter_batch, the entry point
that allocates, on two calls in a row: the shared array keeps the previous
call's contents, so the second call shows the counter is reset and the table
rewritten.  Both entry points build the same launch (one shared table
preparation, including the tile height of a lone image), so the results must
be bit-identical.  This file is collected last and builds everything it needs,
so it passes alone in a fresh process as well as after the other tests."""
import ctypes

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


def _batch(bf, n=3):
    specs = [(130, 200, 2.0, 32), (64, 64, 8.0, 64), (97, 150, 5.0, 32)][:n]
    plans, xs, items = [], [], []
    for i, (H, W, s, K) in enumerate(specs):
        f = synth.voronoi_image(H, W, 3, 7, 10.0, seed=900 + i)
        plan = bf.bf_plan(3, synth.spd_cond(3, seed=910 + i), s, 10, K, 920 + i)
        x = bf.to_pitched(f)
        plans.append(plan)
        xs.append(x)
    return specs, plans, xs


def _items(bf, specs, plans, xs, outs):
    arr = (bf.bf_item * len(specs))()
    for k, ((H, W, s, K), plan, x, y) in enumerate(zip(specs, plans, xs, outs)):
        arr[k] = bf.bf_item(plan.handle, x.data_ptr(), y.data_ptr(), H, W, x.stride(1))
    return arr


@pytest.mark.parametrize("variant,n", [("fp16tc", 3), ("bf16tc", 3), ("fp16tc", 1)])
def test_noalloc_matches_allocating_entry_point_twice(bf, variant, n):
    L = bf.lib()
    v = bf.VARIANTS[variant]
    stream = torch.cuda.current_stream().cuda_stream
    specs, plans, xs = _batch(bf, n)
    ref = [bf.pitched_empty(3, H, W) for (H, W, _, _) in specs]
    assert L.bf_filter_batch(_items(bf, specs, plans, xs, ref), len(specs), v, ctypes.c_void_p(stream)) == bf.BF_OK
    torch.cuda.synchronize()
    for call in range(2):
        outs = [bf.pitched_empty(3, H, W) for (H, W, _, _) in specs]
        for y in outs:
            y.fill_(float("nan"))
        rc = L.bf_filter_batch_noalloc(_items(bf, specs, plans, xs, outs), len(specs), v, ctypes.c_void_p(stream))
        assert rc == bf.BF_OK, bf.lib().bf_error_string(rc)
        torch.cuda.synchronize()
        for y, r in zip(outs, ref):
            a, b = y.cpu().numpy(), r.cpu().numpy()
            assert np.isfinite(a).all()
            assert np.array_equal(a, b), f"call {call}"
    assert bf.bf_last_status(stream) == bf.BF_OK


def test_noalloc_rejects_what_it_cannot_hold(bf):
    L = bf.lib()
    specs, plans, xs = _batch(bf)
    outs = [bf.pitched_empty(3, H, W) for (H, W, _, _) in specs]
    arr = _items(bf, specs, plans, xs, outs)
    assert L.bf_filter_batch_noalloc(arr, bf.BF_NOALLOC_MAX_ITEMS + 1, bf.BF_FP16TC, None) == bf.BF_ERR_BUDGET
    assert L.bf_filter_batch_noalloc(arr, len(specs), bf.BF_FP32, None) == bf.BF_ERR_ARG
    assert L.bf_filter_batch_noalloc(arr, 0, bf.BF_FP16TC, None) == bf.BF_OK


def test_noalloc_refuses_stream_capture(bf):
    """The call uploads its table from host memory of the call itself, which a
    captured graph would read again at every replay; under capture it returns
    BF_ERR_ARG and queues nothing."""
    L = bf.lib()
    specs, plans, xs = _batch(bf, 1)
    outs = [bf.pitched_empty(3, H, W) for (H, W, _, _) in specs]
    arr = _items(bf, specs, plans, xs, outs)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    rc = None
    with torch.cuda.graph(g, stream=s):
        rc = L.bf_filter_batch_noalloc(arr, 1, bf.BF_FP16TC, ctypes.c_void_p(s.cuda_stream))
    assert rc == bf.BF_ERR_ARG
