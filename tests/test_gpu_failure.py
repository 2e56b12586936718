"""Failure detection on the GPU without a device fault.

The tensor-core pipelines wait on mbarriers with a bounded number of clock
cycles; on expiry a kernel records a code in the context's device word and
returns, and later tensor-core launches of the context return at once until
the word is reset.  These tests make a wait expire on purpose with a tiny
limit (the MMA warp gives up before its first copied stage lands; the copies
and MMAs in flight are still waited for, with the long limit, before the
CTA exits), check that distil_device_status reports it, that a reset clears
it and that the next call with the normal limit is correct.  Input scans and
short workspaces fail on the host with their own codes, nothing launched."""
import ctypes

import numpy as np
import pytest

from paper_2609_37723_b300 import synth
from parity import normwise

pytestmark = pytest.mark.gpu


def T(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _status(L, ctx, reset):
    code = ctypes.c_uint(99)
    st = L.distil_device_status(ctx, int(reset), ctypes.byref(code))
    return st, code.value


def test_expired_wait_is_reported_and_cleared(cuda_lib):
    from paper_2609_37723_b300 import distil
    L = distil.lib()
    ctx = distil.context(0)
    rng = np.random.default_rng(5)
    A = synth.complex_gaussian(rng, (256, 4096)).astype(np.complex64)
    B = synth.complex_gaussian(rng, (192, 4096)).astype(np.complex64)
    ref = A.astype(np.complex128) @ B.astype(np.complex128).T
    assert _status(L, ctx, True) == (0, 0)
    try:
        distil.set_wait_limit(64)          # far shorter than a bulk-copy round trip
        distil.cgemm(T(A), T(B), "fp16x6")
        st, code = _status(L, ctx, False)
        assert st == 4 and code in (1, 2, 3), (st, code)     # DISTIL_ETIMEOUT, a pipeline wait
        assert b"bounded device wait expired" in L.distil_last_error()
        # while the word is set, tensor-core launches return at once: nothing is computed
        import torch
        out = torch.zeros((1, 256, 192), dtype=torch.complex64, device="cuda")
        distil.set_wait_limit(0)
        distil.cgemm(T(A), T(B), "fp16x6", out=out)
        torch.cuda.synchronize()
        assert not out.abs().any()
        st, code2 = _status(L, ctx, True)  # read and clear
        assert st == 4 and code2 == code
        assert _status(L, ctx, False) == (0, 0)
    finally:
        distil.set_wait_limit(0)
        _status(L, ctx, True)
    # the context is usable again: the same product with the default limit
    got = distil.cgemm(T(A), T(B), "fp16x6").cpu().numpy()[0]
    assert normwise(got, ref) < 1e-7
    assert _status(L, ctx, False) == (0, 0)


def test_expired_wait_in_the_correlator_pipeline(cuda_lib):
    """The same through distil_correlate (persistent and one-tile kernels of
    the three contraction sites): the call fails on the device, the status
    says so, and a rerun after the reset matches a clean run bit for bit."""
    from paper_2609_37723_b300 import distil
    from oracle import nucleon as orc
    L = distil.lib()
    ctx = distil.context(0)
    p = synth.small(4, 2, 24, mom=[(0, 0, 0)], sigmas=(0.5, 1.0), seed_cfg=31, dtype=np.complex64)
    v, tau = p.all_eigvecs(), p.all_perambulators()
    phi = T(orc.elementals(v, p.L, p.mom))
    clean = distil.correlate(phi, phi[0], T(tau), T(p.prof), "fp16x6").cpu().numpy()
    try:
        distil.set_wait_limit(64)
        distil.correlate(phi, phi[0], T(tau), T(p.prof), "fp16x6")
        st, code = _status(L, ctx, True)
        assert st == 4 and code in (1, 2, 3)
    finally:
        distil.set_wait_limit(0)
        _status(L, ctx, True)
    again = distil.correlate(phi, phi[0], T(tau), T(p.prof), "fp16x6").cpu().numpy()
    assert np.array_equal(again, clean)


def test_non_finite_inputs_are_found(cuda_lib):
    import torch
    from paper_2609_37723_b300 import distil
    x = torch.randn(1 << 20, dtype=torch.complex64, device="cuda")
    assert distil.scan_finite(x) == -1
    x.view(torch.float32)[777_777] = float("nan")
    x.view(torch.float32)[999_999] = float("inf")
    with pytest.raises(distil.DistilError, match="element 777777"):
        distil.scan_finite(x)
    y = torch.zeros(1000, dtype=torch.float64, device="cuda")
    y[3] = float("-inf")
    with pytest.raises(distil.DistilError, match="element 3"):
        distil.scan_finite(y)
    assert distil.scan_finite(torch.zeros(0, dtype=torch.float64, device="cuda")) == -1


def test_short_workspace_is_refused_before_launch(cuda_lib):
    import torch
    from paper_2609_37723_b300 import distil
    p = synth.small(3, 1, 12, mom=[(0, 0, 0)], sigmas=(0.5,), dtype=np.complex64)
    tau = T(p.all_perambulators())
    phi = torch.zeros((1, 1, p.T3), dtype=torch.complex128, device="cuda")
    need = distil.correlate_workspace(1, p.nv, 1, 1, "fp16x6")
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    C = torch.full((1, 1, 1, 1), complex(2.0, 2.0), dtype=torch.complex128, device="cuda")
    with pytest.raises(distil.DistilError) as e:
        distil.correlate(phi, phi[0], tau, T(p.prof), "fp16x6", out=C, workspace=ws)
    assert e.value.status == 2 and "workspace" in str(e.value)
    assert C.cpu().numpy()[0, 0, 0, 0] == 2 + 2j
    assert distil.device_status() == 0
