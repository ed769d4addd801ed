"""The checked build (BF_DEVICE_CHECKS): the tensor-core kernel checks its
global, shared- and tensor-memory indices; a failed check records BF_ERR_BOUNDS
in the status word and skips the access, so the build stands in for a memory
checker without faulting the GPU.  Odd shapes through the general and the
specialised step loops, a batch and the allocation-free entry point all report
BF_OK in the checked build and give results bit-identical to the normal build.
Each library runs in a process of its own (chosen with BF_LIBRARY)."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (H, W, sigma_s, K, images, variant, entry[, d])
CASES = [
    (120, 150, 3.0, 8, 1, "fp16tc", "batch"),      # alone: fitted 16-row tile, general loop
    (170, 150, 8.0, 8, 2, "fp16tc", "batch"),      # batch: 80-row tiles, specialised loop (lag 3)
    (512, 512, 1.0, 4, 1, "fp16tc", "batch"),      # alone: 32-row tiles, two-term centre ring
    (70, 90, 10.5, 8, 1, "fp16tc", "batch"),       # r = 31, general loop (lag 4)
    (1, 100, 2.0, 4, 1, "fp16tc", "batch"),        # one row
    (9, 11, 5.0, 4, 1, "bf16tc", "batch"),         # image smaller than the window
    (96, 200, 4.0, 8, 2, "bf16tc", "batch"),       # batch, specialised loop (lag 2)
    (130, 77, 2.5, 8, 3, "fp16tc", "noalloc"),     # allocation-free entry point
    (100, 140, 4.0, 8, 2, "fp16tc", "batch", 6),   # six channels: 16-bit region codes, two passes per term
    (9, 11, 10.9, 4, 1, "bf16tc", "batch", 6),     # six channels, r = 32, image smaller than the window
    (77, 65, 2.0, 4, 2, "fp16tc", "noalloc", 6),   # six channels through the allocation-free entry point
]

SCRIPT = textwrap.dedent("""
    import json, sys
    import numpy as np, torch
    from paper_1605_02164_gb300 import bf, synth
    cases, out = json.loads(sys.argv[1]), sys.argv[2]
    res = {}
    for i, (H, W, s, K, n, variant, entry, *dd) in enumerate(cases):
        d = dd[0] if dd else 3
        C = synth.spd_cond(d, seed=900 + i)
        plans, xs, ys = [], [], []
        for j in range(n):
            f = synth.voronoi_image(H, W, d, 5, 10.0, seed=910 + 10 * i + j)
            plans.append(bf.bf_plan(d, C, s, 10, K, 920 + i))
            xs.append(bf.to_pitched(f))
            ys.append(bf.pitched_empty(d, H, W))
        items = [(p, x.data_ptr(), y.data_ptr(), H, W, x.stride(1)) for p, x, y in zip(plans, xs, ys)]
        call = bf.bf_filter_batch if entry == "batch" else bf.bf_filter_batch_noalloc
        call(items, bf.VARIANTS[variant], torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        res[f"status{i}"] = np.array(bf.bf_last_status(0))
        for j, y in enumerate(ys):
            res[f"out{i}_{j}"] = y.cpu().numpy()
    np.savez(out, **res)
""")


def _run(lib_path, out):
    env = dict(os.environ, BF_LIBRARY=lib_path)
    subprocess.run([sys.executable, "-c", SCRIPT, json.dumps(CASES), out], env=env, cwd=ROOT,
                   check=True, timeout=900)
    return np.load(out)


def test_checked_build_reports_ok_and_matches(tmp_path):
    from paper_1605_02164_gb300 import build
    normal = build.build()
    checked = build.build_checked()
    a = _run(normal, str(tmp_path / "normal.npz"))
    b = _run(checked, str(tmp_path / "checked.npz"))
    assert sorted(a.files) == sorted(b.files)
    for i in range(len(CASES)):
        assert int(a[f"status{i}"]) == 0 and int(b[f"status{i}"]) == 0, CASES[i]
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
