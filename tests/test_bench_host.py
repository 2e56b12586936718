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
    assert j["achieved"] == pytest.approx(8 * 6 * 24.0 * nb * n ** 4 * tp / 1e12)
    assert j["frac"] == pytest.approx(j["achieved"] / 1000.0)
    d = rows["dot"]
    P2 = n * (n - 1) // 2
    assert d["bound"] == "hbm" and d["achieved"] == pytest.approx((96.0 * nb * n ** 3 + 80.0 * nb * P2 * n) * tp / 1e9)
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
