"""Host-side checks of the meson entry points (no GPU needed): workspace
queries, the size limits and the modes the build implements."""
import ctypes

import pytest

from paper_2609_37723_b300 import distil


@pytest.fixture(scope="module")
def L():
    return distil.lib()


def _ws(fn, *args):
    b = ctypes.c_size_t()
    st = fn(*args, ctypes.byref(b))
    return st, b.value


def test_meson_workspace_queries(L):
    st, b = _ws(L.distil_meson_elementals_workspace, 24, 48, 200, 1, distil.MODES["fp16x6"])
    assert st == 0 and b > 0
    # the batch of timeslices keeps the elementals workspace within 16 GiB plus one timeslice
    assert b < (17 << 30)
    st1, b1 = _ws(L.distil_meson_elementals_workspace, 24, 1, 200, 1, distil.MODES["fp16x6"])
    assert st1 == 0 and 0 < b1 <= b
    st, c = _ws(L.distil_meson_correlate_workspace, 200, 1, 7, distil.MODES["fp16x6"])
    assert st == 0
    # two [21 * 800][800] double-float products, two split images and the tables
    assert c > 2 * 21 * 800 * 800 * 16


@pytest.mark.parametrize("mode", ["fp64", "fp32", "bf16x6", "bf16x3", "fp16x3"])
def test_meson_other_modes_not_supported(L, mode):
    st, _ = _ws(L.distil_meson_elementals_workspace, 8, 4, 16, 1, distil.MODES[mode])
    assert st == 5
    st, _ = _ws(L.distil_meson_correlate_workspace, 16, 1, 7, distil.MODES[mode])
    assert st == 5


@pytest.mark.parametrize("args", [(0, 4, 16, 1), (129, 4, 16, 1), (8, 0, 16, 1), (8, 4, 0, 1), (8, 4, 1025, 1),
                                  (8, 4, 16, 0), (8, 4, 16, 17)])
def test_meson_elementals_bad_sizes(L, args):
    st, _ = _ws(L.distil_meson_elementals_workspace, *args, distil.MODES["fp16x6"])
    assert st == 1


@pytest.mark.parametrize("args", [(0, 1, 7), (16, 0, 7), (16, 1, 0), (16, 1, 11), (16, 17, 7)])
def test_meson_correlate_bad_sizes(L, args):
    st, _ = _ws(L.distil_meson_correlate_workspace, *args, distil.MODES["fp16x6"])
    assert st == 1


def test_meson_calls_without_context_fail_cleanly(L):
    assert L.distil_meson_prune(None, None, 1, 21, 4, 0, 8, None, None, None, None) == 1
    assert L.distil_meson_correlate(None, None, None, None, 4, 16, 1, None, 7, distil.MODES["fp16x6"], None, None,
                                    0, None) == 1


def test_glueball_workspace_and_sizes(L):
    b = ctypes.c_size_t()
    assert L.distil_glueball_workspace(24, 48, ctypes.byref(b)) == 0
    # 57 complex128 3 x 3 fields per site and timeslice, batched within 4 GiB
    assert 57 * 24 ** 3 * 144 < b.value < (5 << 30)
    for bad in [(1, 4), (129, 4), (8, 0)]:
        assert L.distil_glueball_workspace(*bad, ctypes.byref(b)) == 1
    assert L.distil_glueball_operators(None, None, 8, 4, None, None, 0, None) == 1
