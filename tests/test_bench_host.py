"""bench.py's host-side accounting on CPU: the per-kernel roofline table and
the whole-step flop count follow the per-unit work of each kernel family."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_kernel_rooflines_from_event_times():
    import bench
    from paper_2609_37723_b300 import synth
    p = synth.config(3, 0)
    n, nb, tp = p.nv, p.nb, p.nt * p.np_
    # one step, 1 s per family: achieved = work per step / 1 s
    ks = {"tc_gemm_step_j": (960, 1000.0), "dot": (320, 1000.0), "split_pairs": (1536, 1000.0),
          "normalise": (321, 1000.0)}
    pk = {"bf16_tflops_sustained": 1000.0, "hbm_gbs": 5000.0}
    rows = {r["kernel"]: r for r in bench.kernel_rooflines(ks, p, "fp16x6", pk, 1)}
    assert set(rows) == {"tc_gemm_step_j", "dot", "split_pairs"}   # no model for normalise
    j = rows["tc_gemm_step_j"]
    assert j["bound"] == "tensor" and j["unit"] == "TFLOP/s"
    # step j runs as two passes of three split products each (tc_gemm_step_j, tc_gemm_step_j_2nd)
    assert j["achieved"] == pytest.approx(8 * 3 * 24.0 * nb * n ** 4 * tp / 1e12)
    assert j["frac"] == pytest.approx(j["achieved"] / 1000.0)
    d = rows["dot"]
    P2 = n * (n - 1) // 2
    assert d["bound"] == "hbm" and d["achieved"] == pytest.approx(16.0 * nb * P2 * n * tp / 1e9)
    assert bench.kernel_rooflines(ks, p, "fp32", pk, 1) == []


def test_algorithmic_flops_convention():
    import bench
    from paper_2609_37723_b300 import synth
    p = synth.config(3, 0)
    f = bench.algorithmic_flops(p)
    tp = p.nt * p.np_
    assert f["elementals"] == pytest.approx(8.0 * 3 * p.V3 * p.T3 * tp)
    assert f["correlator"] == pytest.approx(8.0 * 92 * p.nb * p.nv ** 4 * tp)
    assert f["total"] == pytest.approx(f["elementals"] + f["correlator"])


def test_shard_timeslices_cover_each_timeslice_once():
    """Timeslice t goes to rank t mod N; a rank's share repeats when it runs
    more steps than it has timeslices."""
    import bench
    nt, world = 96, 8
    shares = [bench.shard_timeslices(nt, r, world, 12) for r in range(world)]
    flat = sorted(t for s in shares for t in s)
    assert flat == list(range(nt))
    assert bench.shard_timeslices(nt, 3, 8, 14) == [3, 11, 19, 27, 35, 43, 51, 59, 67, 75, 83, 91, 3, 11]
    assert bench.shard_timeslices(96, 0, 1, 25) == list(range(25))
    assert bench.shard_timeslices(2, 5, 8, 3) == [1, 1, 1]          # more ranks than timeslices


def test_elementals_issued_tiles_count_the_triangle_skip():
    """The issued elementals MACs: every 128 x 128 tile whose smallest i is
    below its largest j, over K padded per 4096-wide chunk.  A tiny case by
    hand: N_v = 20, one momentum -> 190 pairs (2 row tiles), 20 (i, p) rows
    (one 32-wide column tile, i_min = 0 < j_max): 2 tiles."""
    import bench
    from paper_2609_37723_b300 import synth
    p = synth.small(4, 1, 20, mom=[(0, 0, 0)])
    K = 3 * 64
    assert bench.elementals_issued_cmacs(p) == 2 * 128 * 32 * 192
    # the full-size workload issues fewer MACs than the dense tile grid and
    # more than the useful i<j<k products
    q = synth.config(5, 0)
    issued = bench.elementals_issued_cmacs(q)
    P2, R = q.nv * (q.nv - 1) // 2, q.nv * q.np_
    dense = -(-P2 // 128) * 128 * -(-R // 128) * 128 * 3 * q.V3
    assert 3 * q.V3 * q.T3 * q.np_ < issued < dense
    assert K == 192


def test_meson_rooflines_follow_the_per_unit_work():
    import bench
    from paper_2609_37723_b300 import synth
    m = synth.meson_config("charm")
    n, V3, nops = m.nv, m.V3, 3 * m.nb
    ks = {"tc_gemm_meson_elem": (33, 1000.0), "tc_gemm_meson_q": (48, 1000.0), "meson_bb": (3, 1000.0),
          "meson_pack": (3, 1000.0)}
    pk = {"bf16_tflops_sustained": 1000.0, "hbm_gbs": 5000.0}
    rows = {r["kernel"]: r for r in bench.meson_rooflines(ks, m, pk, 1)}
    assert set(rows) == {"tc_gemm_meson_elem", "tc_gemm_meson_q", "meson_bb"}
    # elementals: 7 displacements x N_p N_v^2 x 3 V3 complex MACs per timeslice, 8 split products
    assert rows["tc_gemm_meson_elem"]["achieved"] == pytest.approx(8 * 8 * 7.0 * n * m.np_ * n * 3 * V3 * m.nt / 1e12)
    # GEMM 1: 3 N_B (4 N_v)^3 per (t, p), 6 split products
    assert rows["tc_gemm_meson_q"]["achieved"] == pytest.approx(8 * 6 * nops * 64.0 * n ** 3 * m.np_ * m.nt / 1e12)
    assert rows["meson_bb"]["bound"] == "hbm"
    assert rows["meson_bb"]["achieved"] == pytest.approx(96.0 * n * 3 * V3 * m.nt / 1e9)
    # the elementals traffic entry scales a 4-timeslice capture to a 16-timeslice launch
    assert bench.MESON_TRAFFIC[(m.name, "tc_gemm_meson_elem")] == pytest.approx(447.7e6 * 4)


def test_glueball_flop_model():
    import bench
    L, nt = 24, 48
    V3 = L ** 3
    clover = bench.glue_flops("glue_clover", L, nt)[0]
    deriv = bench.glue_flops("glue_deriv", L, nt)[0]
    trace = bench.glue_flops("glue_trace", L, nt)[0]
    # 45360 FP64 flops per site and timeslice in all: 8 x (972 + 4212 + 486) complex multiply-adds
    assert (clover + deriv + trace) / (V3 * nt) == pytest.approx(8 * (972 + 4212 + 486))
    assert bench.glue_flops("glue_final", L, nt) is None
