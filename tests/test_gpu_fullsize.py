"""Parity at the full sizes of the tensor-core workloads, in the launch
configuration bench.py times, against stored FP64 oracle values.

The oracle values (tests/golden/oracle_*.json) were written by
tests/golden/make_oracle_golden.py, which calls only the oracle and the
seeded input generator.  For each workload the test regenerates the inputs
of the sampled timeslices (and checks a few raw values against those the
oracle saw), computes the elementals of every momentum and the correlation
matrix of every sampled (t, p) on the GPU in the FP16X6 mode, and gates
every entry C_ab(t) at 1e-6 relative (an entry below 1e-10 of its matrix's
largest is gated against that largest instead; none is, with these inputs)
and the sampled elementals at 3e-7 of the largest sampled |Phi| of their
(t, p).  The samples cover the first, second, middle and last timeslices
(perambulators decay as exp(-0.4 t): C spans 1e-33 over the workload) and
the first and the last momentum.

  L = 32, N_t = 64, N_v = 128, 5 momenta, 6 profiles     whole-range calls
  L = 32, N_t = 64, N_v = 96 (an ensemble member), 7 mom.  whole-range calls
  L = 48, N_t = 96, N_v = 256, 9 momenta, 8 profiles      one timeslice per call
"""
import json
import os

import numpy as np
import pytest

from paper_2609_37723_b300 import synth
from parity import c_entry_errors, c_scaled_errors

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_C = 1e-6
TOL_PHI = 3e-7


def load(name):
    path = os.path.join(HERE, "golden", f"oracle_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"stored oracle values {os.path.basename(path)} not generated")
    return json.load(open(path))


def cx(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


def inputs(g, ts):
    p = synth.config(g["workload"], g["cfg"])
    v = np.stack([p.eigvecs(t) for t in ts])
    tau = np.stack([p.perambulator(t) for t in ts])
    for s, t in enumerate(ts):
        ref = g["inputs"].get(str(t))
        if ref is None:
            continue
        vf = v[s].reshape(-1)
        tf = tau[s].reshape(-1)
        got_v = vf[:: max(1, vf.size // 8)][:8]
        got_t = tf[:: max(1, tf.size // 8)][:8]
        assert np.allclose(got_v, cx(ref["v_flat"]), rtol=1e-6, atol=0), "regenerated eigenvectors differ"
        assert np.allclose(got_t, cx(ref["tau_flat"]), rtol=1e-6, atol=0), "regenerated perambulators differ"
    return p, v, tau


def check(name, g, p, ts, phi, C_of):
    """phi[s][q] elementals of timeslice ts[s] (device tensor), C_of(t) -> C[np][nb][nb]."""
    worst_c, worst_phi = 0.0, 0.0
    ranks = np.asarray(g["phi_ranks"])
    for smp in g["samples"]:
        t, q = smp["t"], smp["p"]
        ref = cx(smp["C"])
        got = C_of(t)[q]
        e = c_entry_errors(got[None, :, :, None], ref[None, :, :, None])
        sc = c_scaled_errors(got[None, :, :, None], ref[None, :, :, None])
        ph_ref = cx(smp["phi"])
        ph = phi[ts.index(t), q].cpu().numpy()[ranks]
        ephi = np.abs(ph - ph_ref).max() / np.abs(ph_ref).max()
        print(f"{name} t={t} p={q}: C strict per-entry {e.max():.2e} (scaled {sc.max():.2e}), "
              f"|C| {np.abs(ref).max():.1e}; elementals {ephi:.2e}")
        worst_c, worst_phi = max(worst_c, float(e.max())), max(worst_phi, ephi)
    print(f"{name}: worst strict per-entry C error {worst_c:.2e}, worst elementals {worst_phi:.2e}")
    assert worst_c < TOL_C
    assert worst_phi < TOL_PHI


@pytest.mark.parametrize("name", ["L32_Nt64_Nv128", "L32_Nt64_cfg3_Nv96"])
def test_fullsize_whole_range_fp16x6(cuda_lib, name):
    """Workloads run as whole configurations (bench.py --workload 3): the
    elementals and the correlation matrix of a range of timeslices per call."""
    import torch
    from paper_2609_37723_b300 import distil
    g = load(name)
    ts = sorted({0} | {s["t"] for s in g["samples"]})
    p, v, tau = inputs(g, ts)
    vd, taud = torch.from_numpy(v).cuda(), torch.from_numpy(tau).cuda()
    profd = torch.from_numpy(np.ascontiguousarray(p.prof)).cuda()
    phi = distil.elementals(vd, p.L, p.mom, "fp16x6")
    C = distil.correlate(phi, phi[0], taud, profd, "fp16x6").cpu().numpy()
    assert distil.device_status() == 0 and np.isfinite(C).all()
    check(name, g, p, ts, phi, lambda t: C[..., ts.index(t)])


def test_fullsize_timeslice_steps_fp16x6(cuda_lib):
    """The large workload as bench.py runs it: one sink timeslice per call
    (elementals of all 9 momenta, then distil_correlate_slice into column t),
    the source elementals of t0 = 0 computed once."""
    import torch
    from paper_2609_37723_b300 import distil
    name = "L48_Nt96_Nv256"
    g = load(name)
    ts = sorted({0} | {s["t"] for s in g["samples"]})
    p, v, tau = inputs(g, ts)
    profd = torch.from_numpy(np.ascontiguousarray(p.prof)).cuda()
    C = torch.zeros((p.np_, p.nb, p.nb, p.nt), dtype=torch.complex128, device="cuda")
    phis = []
    src = None
    for s, t in enumerate(ts):
        vt = torch.from_numpy(v[s:s + 1]).cuda()
        ph = distil.elementals(vt, p.L, p.mom, "fp16x6")
        if t == 0:
            src = ph
        else:
            distil.correlate_slice(ph[0], src[0], torch.from_numpy(tau[s]).cuda(), profd, profd, C, t, "fp16x6")
        phis.append(ph[0])
        del vt
    Cn = C.cpu().numpy()
    assert distil.device_status() == 0 and np.isfinite(Cn).all()
    check(name, g, p, ts, torch.stack(phis), lambda t: Cn[..., t])
