"""Parity at the full size of the mixed-precision workload (L = 32, N_t = 64,
N_v = 128, 5 momenta, 6 profiles) in the launch configuration bench.py
times: the whole ensemble of timeslices and momenta on the device, then
sampled outputs that the FP64 oracle computes one by one, the column
b = 0 of C(t = 1, p = 0) and its GEVP-independent entries."""
import numpy as np
import pytest

from paper_2609_37723_b300 import synth
from oracle import nucleon as orc

pytestmark = pytest.mark.gpu


def test_fullsize_fp16x6_sampled_slice(cuda_lib):
    import torch
    from paper_2609_37723_b300 import distil
    p = synth.config(3, 0)
    v = p.all_eigvecs().astype(np.complex64)
    tau = p.all_perambulators().astype(np.complex64)
    vd, taud, profd = (torch.from_numpy(x).cuda() for x in (v, tau, np.ascontiguousarray(p.prof)))
    phi = distil.elementals(vd, p.L, p.mom, "fp16x6")
    C = distil.correlate(phi, phi[0], taud, profd, "fp16x6").cpu().numpy()
    assert distil.device_status() == 0
    assert np.isfinite(C).all()
    # oracle on the sampled slice (t = 1, p = 0, b = 0)
    mom0 = p.mom[:1]
    phi0 = orc.elementals_t(v[0].astype(np.complex128), p.L, mom0)[0]
    phi1 = orc.elementals_t(v[1].astype(np.complex128), p.L, mom0)[0]
    ref = orc.correlator_tp(phi1, phi0, tau[1].astype(np.complex128), p.prof, p.prof, bs=[0])[:, 0]
    got = C[0, :, 0, 1]
    scaled = np.abs(got - ref).max() / np.abs(ref).max()
    strict = (np.abs(got - ref) / np.abs(ref)).max()
    print(f"full size fp16x6, t=1 p=0 b=0: scaled {scaled:.2e} strict per-entry {strict:.2e}")
    assert scaled < 1e-6
    # elementals themselves at a sample of triples, t = 1, p = 0
    ph = phi[1, 0].cpu().numpy()
    idx = np.random.default_rng(3).choice(ph.shape[0], 2000, replace=False)
    e = np.abs(ph[idx] - phi1[idx]).max() / np.abs(phi1).max()
    print(f"full size fp16x6 elementals, 2000 sampled triples: {e:.2e}")
    assert e < 3e-7
