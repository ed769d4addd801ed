"""CPU-only checks of the C ABI: the library builds, loads, and exports every
function include/bf.h declares; argument checks that return before any CUDA
call behave as documented.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bf.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(bf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_02164_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["bf_plan", "bf_plan_ex", "bf_plan_get_freqs", "bf_plan_info", "bf_plan_destroy", "bf_filter",
              "bf_filter_batch", "bf_filter_host", "bf_last_status", "bf_error_string", "bf_version"]:
        assert n in names, n


def test_every_declared_symbol_is_exported(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), f"{n} declared in bf.h but not exported"


def test_error_strings_and_version(lib):
    lib.bf_error_string.restype = ctypes.c_char_p
    for code in range(0, -10, -1):
        s = lib.bf_error_string(code)
        assert s and s != b"unknown error"
    assert lib.bf_version() >= 10000


def test_host_side_argument_checks(lib):
    """These return before the library touches the GPU."""
    from paper_1605_02164_gb300 import bf
    L = bf.lib()
    h = ctypes.c_void_p()
    C = (ctypes.c_double * 1)(100.0)
    assert L.bf_plan(0, C, 2.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_D_RANGE
    assert L.bf_plan(9, C, 2.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_D_RANGE
    assert L.bf_plan(1, C, -1.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_ARG
    assert L.bf_plan(1, C, 2.0, 10, 0, 1, ctypes.byref(h)) == bf.BF_ERR_ARG
    assert L.bf_plan(1, C, 2.0, 5000, 8, 1, ctypes.byref(h)) == bf.BF_ERR_ARG
    assert L.bf_plan(1, C, 1400.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_UNSUPPORTED
    asym = (ctypes.c_double * 4)(100.0, 1.0, 2.0, 100.0)
    assert L.bf_plan(2, asym, 2.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_ARG
    assert L.bf_plan(1, None, 2.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_ARG
    assert L.bf_filter(None, None, None, 4, 4, 4, 0, None) == bf.BF_ERR_ARG
    assert L.bf_plan_destroy(None) == bf.BF_ERR_ARG
    assert L.bf_filter_batch(None, -1, 0, None) == bf.BF_ERR_ARG
    assert L.bf_filter_batch(None, 0, 0, None) == bf.BF_OK


def test_colour_transform_argument_checks(lib):
    """bf_rgb_to_lab / bf_lab_to_rgb reject bad arguments before any CUDA call."""
    from paper_1605_02164_gb300 import bf
    L = bf.lib()
    vp = ctypes.c_void_p
    for fn in (L.bf_rgb_to_lab, L.bf_lab_to_rgb):
        assert fn(None, None, 0, 5, 8, None) == bf.BF_OK          # empty image: no-op
        assert fn(None, None, 4, 5, 8, None) == bf.BF_ERR_ARG      # null buffers
        assert fn(vp(0x10000), vp(0x20000), 4, 9, 8, None) == bf.BF_ERR_ARG   # pitch < W
        assert fn(vp(0x10000), vp(0x20000), -1, 4, 8, None) == bf.BF_ERR_ARG
        assert fn(vp(0x10004), vp(0x20000), 4, 5, 8, None) == bf.BF_ERR_ALIGN
        assert fn(vp(0x10000), vp(0x20000), 4, 5, 6, None) == bf.BF_ERR_ALIGN  # pitch % 4
        assert fn(vp(0x10000), vp(0x10010), 4, 5, 8, None) == bf.BF_ERR_ARG   # partial overlap


def test_host_entry_points_argument_checks(lib):
    """bf_filter_host / bf_filter_host_async reject bad arguments before any CUDA call."""
    from paper_1605_02164_gb300 import bf
    L = bf.lib()
    vp = ctypes.c_void_p
    buf = (ctypes.c_float * 16)()
    for fn in (L.bf_filter_host, L.bf_filter_host_async):
        assert fn(None, buf, buf, 4, 4, 0, None) == bf.BF_ERR_ARG          # no plan
        assert fn(vp(1), buf, buf, -1, 4, 0, None) == bf.BF_ERR_ARG        # negative size
        assert fn(vp(1), None, buf, 4, 4, 0, None) == bf.BF_ERR_ARG        # null host buffer
        assert fn(vp(1), buf, buf, 0, 4, 0, None) == bf.BF_OK              # empty image: no-op


def test_fault_injection_host_side(lib):
    """bf_debug_inject: unknown bits are rejected; an armed allocation fault is
    consumed by the next plan creation (after its argument checks), which
    fails with BF_ERR_NOMEM before touching the device."""
    from paper_1605_02164_gb300 import bf
    L = bf.lib()
    assert L.bf_debug_inject(4) == bf.BF_ERR_ARG
    assert L.bf_debug_inject(-1) == bf.BF_ERR_ARG
    C = (ctypes.c_double * 1)(900.0)
    h = ctypes.c_void_p()
    try:
        assert L.bf_debug_inject(bf.BF_FAULT_ALLOC) == bf.BF_OK
        assert L.bf_plan(1, C, -1.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_ARG  # checks first, fault kept
        assert L.bf_plan(1, C, 2.0, 10, 8, 1, ctypes.byref(h)) == bf.BF_ERR_NOMEM
        assert not h.value
    finally:
        assert L.bf_debug_inject(0) == bf.BF_OK


def test_tuning_table(lib):
    """bf_tune_*: keys by radius class ceil(r / 8), values 16..128 in steps of
    16, 0 removes; bad keys are refused.  Host-only (no CUDA call)."""
    from paper_1605_02164_gb300 import bf
    bf.bf_tune_clear()
    try:
        cls = bf.bf_tune_size_class(2160, 3840)
        assert cls == 32 * 22 + 23                       # floor(2 log2 2160) = 22, floor(2 log2 3840) = 23
        assert bf.bf_tune_size_class(512, 512) == 32 * 18 + 18
        assert bf.bf_tune_size_class(1, 1) == 0
        assert bf.lib().bf_tune_size_class(0, 5) == bf.BF_ERR_ARG
        bf.bf_tune_set(bf.BF_FP16TC, 3, 24, cls, bf.BF_TUNE_ALONE, 48)
        assert bf.bf_tune_get(bf.BF_FP16TC, 3, 24, cls, bf.BF_TUNE_ALONE) == 48
        assert bf.bf_tune_get(bf.BF_FP16TC, 3, 17, cls, bf.BF_TUNE_ALONE) == 48   # same radius class
        assert bf.bf_tune_get(bf.BF_FP16TC, 3, 25, cls, bf.BF_TUNE_ALONE) == 0    # next class
        assert bf.bf_tune_get(bf.BF_FP16TC, 3, 24, cls, bf.BF_TUNE_BATCH) == 0
        assert bf.bf_tune_get(bf.BF_BF16TC, 3, 24, cls, bf.BF_TUNE_ALONE) == 0
        assert bf.bf_tune_count() == 1
        bf.bf_tune_set(bf.BF_FP32, 6, 3, cls, bf.BF_TUNE_BATCH, 128)
        assert bf.bf_tune_count() == 2
        bf.bf_tune_set(bf.BF_FP16TC, 3, 20, cls, bf.BF_TUNE_ALONE, 0)             # removes the class entry
        assert bf.bf_tune_count() == 1
        L = bf.lib()
        out = ctypes.c_int()
        for bad in [(bf.BF_FP32_RECURSIVE, 3, 4, cls, 0, 32), (7, 3, 4, cls, 0, 32), (0, 0, 4, cls, 0, 32),
                    (0, 9, 4, cls, 0, 32), (0, 3, 33, cls, 0, 32), (0, 3, -1, cls, 0, 32), (0, 3, 4, -1, 0, 32),
                    (0, 3, 4, cls, 2, 32), (0, 3, 4, cls, 0, 24), (0, 3, 4, cls, 0, 144), (0, 3, 4, cls, 0, -16)]:
            assert L.bf_tune_set(*bad) == bf.BF_ERR_ARG, bad
        assert L.bf_tune_get(0, 3, 4, cls, 0, None) == bf.BF_ERR_ARG
        assert L.bf_tune_get(0, 3, 4, cls, 3, ctypes.byref(out)) == bf.BF_ERR_ARG
        assert bf.bf_tune_count() == 1
    finally:
        bf.bf_tune_clear()
    assert bf.bf_tune_count() == 0


def test_tune_cache_round_trip(lib, tmp_path):
    """A saved cache applied in a clean table restores the same entries."""
    from paper_1605_02164_gb300 import bf, tune
    path = str(tmp_path / "tune.json")
    c = tune.TuneCache(path)
    assert c.entries == {}
    cls = bf.bf_tune_size_class(1024, 1024)
    for v, d, r, ctx, rows in [(bf.BF_FP16TC, 3, 9, bf.BF_TUNE_ALONE, 64), (bf.BF_FP32, 6, 30, bf.BF_TUNE_BATCH, 96)]:
        c.entries[c.key(v, d, r, cls, ctx)] = {"variant": v, "d": d, "r": r, "size_class": cls, "context": ctx,
                                               "rows": rows}
    c.save()
    bf.bf_tune_clear()
    try:
        c2 = tune.TuneCache(path)
        assert c2.apply() == 2 and bf.bf_tune_count() == 2
        assert bf.bf_tune_get(bf.BF_FP16TC, 3, 16, cls, bf.BF_TUNE_ALONE) == 64
        assert bf.bf_tune_get(bf.BF_FP32, 6, 25, cls, bf.BF_TUNE_BATCH) == 96
        assert c2.has(bf.BF_FP16TC, 3, 12, 1100, 1050, bf.BF_TUNE_ALONE)   # same half-octave classes
        assert not c2.has(bf.BF_FP16TC, 3, 12, 1100, 1000, bf.BF_TUNE_ALONE)
        assert not c2.has(bf.BF_FP16TC, 3, 17, 1024, 1024, bf.BF_TUNE_ALONE)
        assert tune.candidates(bf.BF_FP16TC, 24, 2160) == [16, 32, 48, 64, 80]
        assert tune.candidates(bf.BF_FP16TC, 32, 2160) == [16, 32, 48, 64]
        assert tune.candidates(bf.BF_FP32, 3, 40) == [16, 32, 48]
        assert tune.candidates(bf.BF_FP16TC, 24, 2160, 6) == [16, 32, 48, 64]
    finally:
        bf.bf_tune_clear()


def test_tune_cache_drops_entries_of_other_sources(tmp_path):
    import json
    from paper_1605_02164_gb300 import tune
    path = str(tmp_path / "old.json")
    with open(path, "w") as fh:
        json.dump({"identity": {"library": "0" * 16, "device": None},
                   "entries": {"1:3:3:600:0": {"variant": 1, "d": 3, "r": 24, "size_class": 600, "context": 0,
                                               "rows": 48}}}, fh)
    c = tune.TuneCache(path)
    assert c.entries == {} and c.dropped == 1
