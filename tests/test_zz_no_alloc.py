"""The allocation-free correlation entry point (distil_correlate_noalloc).

It serves callers that cannot allocate device memory where they need the
correlation matrix (a fixed, pre-reserved device-memory budget, or a
pipeline that cannot take the device-wide synchronisation of cudaMalloc /
cudaFree): its scratch is a fixed device array inside the library.  The test
calls it through the C ABI twice in a row and compares each result with the
regular entry point (distil_correlate, caller workspace) at the tolerances
of the other plain-path tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import nucleon as orc
from paper_2609_37723_b300 import synth
from parity import max_c_error

pytestmark = pytest.mark.gpu


def _call_noalloc(L, ctx, phi, tau, prof, mode, out):
    import torch
    nt, np_ = int(phi.shape[0]), int(phi.shape[1])
    nv = int(tau.shape[1]) // 4
    nb = int(prof.shape[-2])
    ph0 = phi[0].contiguous()
    st = L.distil_correlate_noalloc(ctx, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(ph0.data_ptr()),
                                    ctypes.c_void_p(tau.data_ptr()), nt, nv, np_,
                                    ctypes.c_void_p(prof.data_ptr()), nb, 0, mode,
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("mode,tol", [(0, 1e-12), (1, 1e-4)])
def test_noalloc_matches_regular_entry(cuda_lib, mode, tol):
    import torch
    from paper_2609_37723_b300 import distil
    L = distil.lib()
    ctx = distil.context(0)
    p = synth.config(1)                                  # N_v = 16, N_B = 3
    cdt = np.complex128 if mode == 0 else np.complex64
    v = p.all_eigvecs().astype(cdt)
    tau = torch.from_numpy(p.all_perambulators().astype(cdt)).cuda()
    prof = torch.from_numpy(p.prof).cuda()
    phi = torch.from_numpy(orc.elementals(v, p.L, p.mom).astype(cdt)).cuda()
    ref = distil.correlate(phi, phi[0].contiguous(), tau, prof, mode).cpu().numpy()
    for call in range(2):
        out = torch.full((p.np_, p.nb, p.nb, p.nt), complex(7.0, 7.0), dtype=torch.complex128, device="cuda")
        assert _call_noalloc(L, ctx, phi, tau, prof, mode, out) == 0, L.distil_last_error()
        got = out.cpu().numpy()
        assert max_c_error(got, ref) < tol, f"call {call}"


def test_noalloc_rejects_oversized_problems(cuda_lib):
    import torch
    from paper_2609_37723_b300 import distil
    L = distil.lib()
    ctx = distil.context(0)
    nv, nb, nt, np_ = 64, 8, 1, 1
    dummy = torch.zeros(16, dtype=torch.complex128, device="cuda")
    st = L.distil_correlate_noalloc(ctx, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                    ctypes.c_void_p(dummy.data_ptr()), nt, nv, np_,
                                    ctypes.c_void_p(dummy.data_ptr()), nb, 0, 0,
                                    ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == 2 and b"scratch" in L.distil_last_error()
    # tensor-core modes are not offered here
    st = L.distil_correlate_noalloc(ctx, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                    ctypes.c_void_p(dummy.data_ptr()), 1, 16, 1,
                                    ctypes.c_void_p(dummy.data_ptr()), 3, 0, 5,
                                    ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == 1


def test_noalloc_size_limit_at_nv16(cuda_lib):
    """N_v = 16 fits the 16 MiB scratch with N_B <= 11 in FP64 (the documented
    limit): N_B = 11 runs and matches the regular entry point, N_B = 12 is
    refused with DISTIL_ENOMEM before anything is launched."""
    import torch
    from paper_2609_37723_b300 import distil
    L = distil.lib()
    ctx = distil.context(0)
    sig = [0.2 + 0.1 * a for a in range(12)]
    for nb, want in ((11, 0), (12, 2)):
        p = synth.small(2, 1, 16, mom=[(0, 0, 0)], sigmas=sig[:nb], seed_cfg=40 + nb)
        v = p.all_eigvecs()
        tau = torch.from_numpy(p.all_perambulators()).cuda()
        prof = torch.from_numpy(p.prof).cuda()
        phi = torch.from_numpy(orc.elementals(v, p.L, p.mom)).cuda()
        out = torch.zeros((p.np_, nb, nb, p.nt), dtype=torch.complex128, device="cuda")
        st = _call_noalloc(L, ctx, phi, tau, prof, 0, out)
        assert st == want, (nb, st, L.distil_last_error())
        if want == 0:
            ref = distil.correlate(phi, phi[0].contiguous(), tau, prof, 0).cpu().numpy()
            assert max_c_error(out.cpu().numpy(), ref) < 1e-12
            assert L.distil_last_error() == b""
        else:
            assert b"scratch" in L.distil_last_error()
            assert not out.abs().any()


def test_noalloc_rejects_misaligned_arrays(cuda_lib):
    """An array pointer off its element alignment is refused with
    DISTIL_EINVAL and nothing is launched (the output stays untouched)."""
    import torch
    from paper_2609_37723_b300 import distil
    L = distil.lib()
    ctx = distil.context(0)
    p = synth.config(1)
    tau = torch.from_numpy(p.all_perambulators()).cuda()
    prof = torch.from_numpy(p.prof).cuda()
    phi = torch.from_numpy(orc.elementals(p.all_eigvecs(), p.L, p.mom)).cuda()
    raw = torch.zeros(p.np_ * p.nb * p.nb * p.nt * 2 + 2, dtype=torch.float64, device="cuda")
    shifted = raw[1:]                     # 8-byte offset: misaligned for complex128 / C
    st = L.distil_correlate_noalloc(ctx, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(phi[0].data_ptr()),
                                    ctypes.c_void_p(tau.data_ptr()), p.nt, p.nv, p.np_,
                                    ctypes.c_void_p(prof.data_ptr()), p.nb, 0, 0,
                                    ctypes.c_void_p(shifted.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == 1 and b"misaligned" in L.distil_last_error()
    assert not raw.any()
    # an 8-byte shifted tau (complex128 in FP64) is refused the same way
    traw = torch.zeros(tau.numel() * 2 + 1, dtype=torch.float64, device="cuda")
    st = L.distil_correlate_noalloc(ctx, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(phi[0].data_ptr()),
                                    ctypes.c_void_p(traw[1:].data_ptr()), p.nt, p.nv, p.np_,
                                    ctypes.c_void_p(prof.data_ptr()), p.nb, 0, 0,
                                    ctypes.c_void_p(raw[:-2].data_ptr()), None)
    assert st == 1
    assert distil.device_status() == 0
