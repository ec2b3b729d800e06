"""Host-side checks of the autotuner (tune.py; no GPU): every value it sweeps is one the
library accepts for that key, every knob names kernels the library times, the cache key
separates shapes and precisions, and the cache round-trips through its JSON file."""
import ctypes

import workloads as W
from paper_2412_10167_gb300 import mw3, tune


def test_sweep_values_are_accepted_by_the_library():
    lib = mw3.lib
    h = ctypes.c_void_p()
    assert lib.mw3_create(ctypes.byref(h), -1, mw3.MW3_MIXED) == 0
    try:
        for key, values in tune.SWEEP.items():
            for v in values:
                assert lib.mw3_set_tuning(h, key.encode(), v) == 0, (key, v)
                assert lib.mw3_get_tuning(h, key.encode()) == v, (key, v)
    finally:
        lib.mw3_destroy(h)


def test_controls_name_timed_kernels():
    names = set()
    h = ctypes.c_void_p()
    lib = mw3.lib
    assert lib.mw3_create(ctypes.byref(h), -1, mw3.MW3_MIXED) == 0
    try:
        cnt = ctypes.c_int(32)
        arr = (ctypes.c_char_p * 32)()
        ms = (ctypes.c_double * 32)()
        nl = (ctypes.c_long * 32)()
        assert lib.mw3_kernel_times(h, -1, arr, ms, nl, ctypes.byref(cnt)) == 0
        names = {arr[i].decode() for i in range(cnt.value)}
    finally:
        lib.mw3_destroy(h)
    assert set(tune.CONTROLS) == set(tune.SWEEP)
    for knob, kernels in tune.CONTROLS.items():
        assert kernels and set(kernels) <= names, (knob, kernels)


def test_shape_key_and_cache_roundtrip(tmp_path):
    k2m = tune.shape_key(W.C2, "mixed")
    assert k2m != tune.shape_key(W.C2, "fp64")
    assert k2m != tune.shape_key(W.C3, "mixed")
    assert tune.shape_key(W.C2, "mixed") == k2m
    path = str(tmp_path / "sub" / "tune.json")
    assert tune.load_cache(path) == {}
    cache = {k2m: {"best": {"kin_warp": 2, "prod_gather": 1}, "ms_per_step": {}}}
    tune.save_cache(cache, path)
    assert tune.load_cache(path) == cache
