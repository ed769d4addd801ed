"""Autotuner of the windowed kernels' tile height.

The fused kernels (BF_FP32, BF_FP16TC, BF_BF16TC) tile the output into
64- or 32-column tiles of BY rows (a multiple of 16).  BY changes no pixel's
result; it trades halo recompute (a tall tile recomputes the 2r-row halo of
fewer tiles) against how evenly the tiles fill the 152 SMs.  The library's
cost model guesses; this module measures.  For a key (variant, d, r, size
class of H x W, context) it times every candidate BY on a synthetic image of
that shape through the library's own entry points (bf_filter for an image
alone, one bf_filter_batch over several copies for the batch context), keeps
the fastest in the library's tuning table (bf_tune_set) and in a JSON cache
that later processes load.  Radii share an entry per class ceil(r / 8) (the
classes share the tensor-core tile geometry); a key is timed at the radius it
is first asked for.  Timing uses CUDA events on the launching stream, median
of a few launches after warm-ups.  Nothing here computes the filter.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import bf, synth

__all__ = ["candidates", "tune", "TuneCache", "default_cache_path", "tc_max_rows", "radius_class"]


def default_cache_path() -> str:
    return os.environ.get("BF_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "libbf", "tune.json")


def tc_max_rows(r: int) -> int:
    """Tallest tile of the tensor-core kernel for window radius r (its region
    holds 128 rows; at most 5 output chunks of 16)."""
    lag = -(-2 * r // 16)
    return 16 * max(1, min((128 - 2 * r) // 16, 8 - lag, 5))


def candidates(variant: int, r: int, H: int, d: int = 3) -> list[int]:
    top = tc_max_rows(r) if variant in (bf.BF_FP16TC, bf.BF_BF16TC) else 128
    if variant in (bf.BF_FP16TC, bf.BF_BF16TC) and d == 6:
        top = min(top, 64)  # two sets of accumulators: at most 4 output chunks
    top = min(top, 16 * (-(-H // 16)))  # no taller than the image needs
    return list(range(16, top + 1, 16))


def radius_class(r: int) -> int:
    return (r + 7) // 8


def _sigma_for(r: int) -> float:
    return (r + 0.5) / 3.0  # floor(3 sigma) = r


def _time_ms(fn, reps: int) -> float:
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def tune(variant: int, d: int, r: int, H: int, W: int, context: int = bf.BF_TUNE_ALONE, K: int = 16,
         reps: int = 5, copies: int | None = None, batch_pixels: float = 8e6, seed: int = 7,
         margin: float = 0.01) -> dict:
    """Measure every candidate tile height for the key, and the cost model's
    own choice (no entry, timed as rows 0); keep a height in the library's
    table only if it beats the cost model by more than `margin` (else no
    entry: the model stays).  The batch context is timed on one
    bf_filter_batch over `copies` copies of the image (default: enough for
    about `batch_pixels` pixels, 2 to 64 copies), so that the SMs see several
    waves of tiles as in a real batch.  Returns {"rows", "ms", "timings", ...}
    (rows 0: the cost model)."""
    import torch
    cls = bf.bf_tune_size_class(H, W)
    C = np.diag([40.0 ** 2] * d)
    plan = bf.bf_plan(d, C, _sigma_for(r), 10, K, seed)
    if plan.r != r:
        raise ValueError(f"window radius {plan.r} != {r}")
    if context == bf.BF_TUNE_ALONE:
        n = 1
    else:
        n = copies if copies else min(64, max(2, -(-int(batch_pixels) // (H * W))))
    f = synth.voronoi_image(H, W, d, 8, 10.0, seed=seed)
    xs = [bf.to_pitched(f) for _ in range(n)]
    ys = [bf.pitched_empty(d, H, W) for _ in range(n)]
    sp = torch.cuda.current_stream().cuda_stream
    items = [(plan, x.data_ptr(), y.data_ptr(), H, W, x.stride(1)) for x, y in zip(xs, ys)]

    def run():
        if n == 1:
            bf.bf_filter(plan, xs[0].data_ptr(), ys[0].data_ptr(), H, W, xs[0].stride(1), variant, sp)
        else:
            bf.bf_filter_batch(items, variant, sp)

    prev = bf.bf_tune_get(variant, d, r, cls, context)
    timings = {}
    try:
        for rows in [0] + candidates(variant, r, H, d):  # 0: no entry, the cost model
            bf.bf_tune_set(variant, d, r, cls, context, rows)
            timings[rows] = _time_ms(run, reps)
    finally:
        bf.bf_tune_set(variant, d, r, cls, context, prev)
    best = min(timings, key=timings.get)
    if best != 0 and timings[best] > (1.0 - margin) * timings[0]:
        best = 0  # within the margin of the cost model's choice: keep the model
    bf.bf_tune_set(variant, d, r, cls, context, best)
    if bf.bf_last_status(sp) != bf.BF_OK:
        raise RuntimeError("device status after tuning")
    plan.close()
    return {"variant": variant, "d": d, "r": r, "radius_class": radius_class(r), "size_class": cls, "context": context, "rows": best,
            "ms": timings[best], "timings": {str(k): v for k, v in timings.items()}, "H": H, "W": W, "K": K, "images": n}


def identity() -> dict:
    """What a cache's timings belong to: the library's sources (their content
    hashes, as the build computes them) and the device.  A cache written for
    another identity is ignored."""
    import hashlib
    from . import build
    lib_id = hashlib.sha1("".join(build._deps_hash(s) for s in build._sources()).encode()).hexdigest()[:16]
    dev = None
    try:
        import torch
        if torch.cuda.is_available():
            pr = torch.cuda.get_device_properties(torch.cuda.current_device())
            dev = f"{pr.name} ({pr.multi_processor_count} SMs)"
    except Exception:  # no torch: the library identity alone
        dev = None
    return {"library": lib_id, "device": dev}


class TuneCache:
    """JSON file of tuned entries; `apply` loads them into the library's table.
    Entries saved for other library sources or another device are dropped on
    load (their timings no longer hold)."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.identity = identity()
        self.entries: dict[str, dict] = {}
        self.dropped = 0
        if os.path.exists(self.path):
            with open(self.path) as fh:
                data = json.load(fh)
            if data.get("identity") == self.identity:
                self.entries = data.get("entries", {})
            else:
                self.dropped = len(data.get("entries", {}))

    @staticmethod
    def key(variant: int, d: int, r: int, size_class: int, context: int) -> str:
        return f"{variant}:{d}:{radius_class(r)}:{size_class}:{context}"

    def apply(self) -> int:
        for e in self.entries.values():
            bf.bf_tune_set(e["variant"], e["d"], e["r"], e["size_class"], e["context"], e["rows"])
        return len(self.entries)

    def has(self, variant: int, d: int, r: int, H: int, W: int, context: int) -> bool:
        return self.key(variant, d, r, bf.bf_tune_size_class(H, W), context) in self.entries

    def ensure(self, keys, **kw) -> dict:
        """Tune every (variant, d, r, H, W, context) of `keys` that the cache
        lacks (one shape per size class), apply all entries; returns a summary."""
        t0 = time.perf_counter()
        tuned = []
        for variant, d, r, H, W, context in keys:
            if self.has(variant, d, r, H, W, context):
                continue
            rec = tune(variant, d, r, H, W, context, **kw)
            self.entries[self.key(variant, d, r, rec["size_class"], context)] = rec
            tuned.append(rec)
        self.apply()
        return {"tuned": len(tuned), "entries": len(self.entries), "seconds": time.perf_counter() - t0}

    def save(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump({"identity": self.identity, "entries": self.entries}, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

