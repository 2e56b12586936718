"""The C-ABI library: it loads, exports every symbol include/distil.h declares,
and its host-side checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2609_37723_b300 import distil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "distil.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(distil_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    from paper_2609_37723_b300 import build
    if not os.path.exists(distil.LIB_PATH):
        build.build()
    return distil.lib()


def test_exports_every_declared_symbol(L):
    syms = header_symbols()
    assert len(syms) >= 8
    for s in syms:
        assert hasattr(L, s), s
    assert set(distil.EXPORTS) <= set(syms)


def test_workspace_queries(L):
    for mode in range(5):
        b = ctypes.c_size_t()
        assert L.distil_correlate_workspace(8, 16, 2, 3, mode, ctypes.byref(b)) == 0
        assert b.value > 0 or mode >= 2
        assert L.distil_elementals_workspace(8, 8, 16, 2, mode, ctypes.byref(b)) == 0
    # FP64 needs twice the FP32 bytes for the same intermediates
    b64, b32 = ctypes.c_size_t(), ctypes.c_size_t()
    L.distil_correlate_workspace(8, 32, 2, 3, 0, ctypes.byref(b64))
    L.distil_correlate_workspace(8, 32, 2, 3, 1, ctypes.byref(b32))
    assert 1.9 < b64.value / b32.value < 2.1


def test_bad_arguments_are_rejected(L):
    b = ctypes.c_size_t()
    assert L.distil_correlate_workspace(8, 16, 2, 17, 0, ctypes.byref(b)) == 1   # nb > 16
    assert L.distil_correlate_workspace(8, 16, 2, 3, 9, ctypes.byref(b)) == 1    # bad mode
    assert b"mode" in L.distil_last_error()
    assert L.distil_elementals_workspace(0, 8, 16, 2, 0, ctypes.byref(b)) == 1   # L = 0
    assert L.distil_correlate_workspace(8, 16, 2, 3, 0, None) == 1
    assert b"null" in L.distil_last_error()
    # null context: EINVAL, no device touched
    assert L.distil_gevp(None, None, 1, 1, 1, 0, None, None) == 1
    assert L.distil_elementals(None, None, 2, 1, 4, None, 1, 0, None, None, 0, None) == 1


def test_create_without_gpu_fails_cleanly(L):
    from conftest import gpu_available
    if gpu_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    st = L.distil_create(0, ctypes.byref(h))
    assert st in (1, 3)
    assert h.value is None
    assert len(L.distil_last_error()) > 0


def test_plan_workspace_host_logic(L):
    """A plan's workspace is the largest configuration's elementals plus the
    largest elementals / correlator workspace: it grows with the largest N_v
    and does not depend on how many smaller configurations come with it."""
    mom = [(0, 0, 0), (1, 0, 0)]
    one = distil.plan_workspace(4, 3, mom, 2, "fp16x6", [16])
    many = distil.plan_workspace(4, 3, mom, 2, "fp16x6", [6, 16, 11, 16])
    small = distil.plan_workspace(4, 3, mom, 2, "fp16x6", [6, 11])
    assert one == many > small > 0
    phi16 = 3 * 2 * distil.n_triples(16) * 16
    assert one >= phi16
    # FP64 plan: elementals in c128, no tensor-core workspace
    assert distil.plan_workspace(4, 3, mom, 2, "fp64", [16]) >= phi16


def test_plan_rejects_bad_ensembles(L):
    mom = [(0, 0, 0)]
    with pytest.raises(distil.DistilError, match="nv < 1"):
        distil.plan_workspace(4, 3, mom, 2, "fp16x6", [8, 0])
    shape, arr, _keep = distil._batch(4, 3, mom, 2, 5, "fp16x6", [{"nv": 8}])   # t0 = 5 >= nt
    b = ctypes.c_size_t()
    assert L.distil_plan_workspace(ctypes.byref(shape), arr, 1, ctypes.byref(b)) == 1
    assert b"t0" in L.distil_last_error()
    assert L.distil_plan_workspace(ctypes.byref(shape), arr, 0, ctypes.byref(b)) == 1
    # a null context or plan is refused without touching a device
    h = ctypes.c_void_p()
    assert L.distil_plan_create(None, ctypes.byref(shape), arr, 1, 0, None, 0, None, ctypes.byref(h)) == 1
    assert L.distil_plan_run(None, None) == 1
    L.distil_plan_destroy(None)


def test_tuning_and_status_argument_checks(L):
    """The tuning table, device-status and plan-info calls refuse null
    handles without touching a device."""
    arr = (ctypes.c_int * 3)(1, 0, 1)
    assert L.distil_set_tuning(None, arr) == 1
    assert L.distil_get_tuning(None, arr) == 1
    code = ctypes.c_uint(7)
    assert L.distil_device_status(None, 0, ctypes.byref(code)) == 1
    assert b"null" in L.distil_last_error()
    assert L.distil_plan_info(None, arr, None) == 1


def test_tuning_cache_round_trip(tmp_path):
    """The plan autotuner's JSON cache: keyed by GPU name and shape (the
    largest N_v of the ensemble), entries replaced in place, unreadable files
    read as empty."""
    path = str(tmp_path / "tune.json")
    assert distil.load_tuning_cache(path) == {}
    k1 = distil.tuning_cache_key("NVIDIA B300 SXM6 AC", 32, 64, 7, 6, "fp16x6", [64, 128, 96])
    k2 = distil.tuning_cache_key("NVIDIA B300 SXM6 AC", 32, 64, 7, 6, "fp16x6", [64, 96])
    assert k1 != k2 and k1.endswith("|nv128") and "|fp16x6|" in k1
    assert distil.tuning_cache_key("X", 32, 64, 7, 6, 5, [8]) == distil.tuning_cache_key("X", 32, 64, 7, 6, "fp16x6", [8])
    distil.store_tuning(path, k1, [1, 0, 0])
    distil.store_tuning(path, k2, [2, 3, 0])
    distil.store_tuning(path, k1, [4, 0, 3])
    d = distil.load_tuning_cache(path)
    assert d == {k1: [4, 0, 3], k2: [2, 3, 0]}
    open(path, "w").write("{not json")
    assert distil.load_tuning_cache(path) == {}


def test_tuning_variant_range(L):
    arr = (ctypes.c_int * 3)(4, 3, 4)
    assert L.distil_set_tuning(None, arr) == 1          # null context first
