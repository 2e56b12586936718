"""Thin Python binding of libdistil (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the shared library.  PyTorch supplies device memory (tensors are
passed by ``data_ptr``) and the current CUDA stream.  The functions mirror
the C interface in ``include/distil.h`` one to one:

    elementals(v, L, mom, mode)                 -> phi   [nt][np][T3]
    correlate(phi_snk, phi_src, tau, prof, mode) -> C    [np][nb][nb][nt]
    gevp(C, t0)                                 -> lam   [np][nt][nb]

If the library is missing or cannot be loaded these calls raise; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DISTIL_LIBRARY") or os.path.join(HERE, "libdistil.so")  # another build of the library

FP64, FP32, MIXED_BF16X6, MIXED_BF16X3, MIXED_FP16X3, MIXED_FP16X6 = 0, 1, 2, 3, 4, 5
MODE_NAMES = {FP64: "fp64", FP32: "fp32", MIXED_BF16X6: "bf16x6", MIXED_BF16X3: "bf16x3",
              MIXED_FP16X3: "fp16x3", MIXED_FP16X6: "fp16x6"}
MODES = {v: k for k, v in MODE_NAMES.items()}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTSUP"}

# Every symbol include/distil.h declares.
EXPORTS = ["distil_create", "distil_destroy", "distil_last_error",
           "distil_elementals_workspace", "distil_elementals",
           "distil_correlate_workspace", "distil_correlate", "distil_correlate_slice", "distil_gevp",
           "distil_gevp_range", "distil_optimal",
           "distil_cgemm_workspace", "distil_cgemm", "distil_correlate_noalloc",
           "distil_mode_supported", "distil_profile_enable", "distil_profile_read",
           "distil_device_status", "distil_set_tuning", "distil_get_tuning",
           "distil_plan_workspace", "distil_plan_create", "distil_plan_run", "distil_plan_info",
           "distil_plan_destroy", "distil_set_wait_limit", "distil_scan_finite",
           "distil_profiles_eigen", "distil_meson_elementals_workspace", "distil_meson_elementals",
           "distil_meson_correlate_workspace", "distil_meson_correlate", "distil_meson_prune",
           "distil_glueball_workspace", "distil_glueball_operators"]

_lib = None
_ctx = {}


class DistilError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"distil {STATUS.get(status, status)}: {msg}")
        self.status = status


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double)]


class BatchShape(ctypes.Structure):
    """distil_batch_shape: what every configuration of an ensemble shares."""
    _fields_ = [("L", ctypes.c_int), ("nt", ctypes.c_int), ("np", ctypes.c_int), ("nb", ctypes.c_int),
                ("t0", ctypes.c_int), ("mode", ctypes.c_int), ("mom", ctypes.POINTER(ctypes.c_int32))]


class BatchCfg(ctypes.Structure):
    """distil_batch_cfg: one configuration (device pointers)."""
    _fields_ = [("nv", ctypes.c_int), ("v", ctypes.c_void_p), ("tau", ctypes.c_void_p),
                ("prof", ctypes.c_void_p), ("C", ctypes.c_void_p), ("lam", ctypes.c_void_p)]


def _declare(L):
    c_int, c_void_p, c_size_t = ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    L.distil_device_status.argtypes = [c_void_p, c_int, P(ctypes.c_uint)]
    L.distil_device_status.restype = c_int
    L.distil_set_tuning.argtypes = [c_void_p, P(c_int)]
    L.distil_set_tuning.restype = c_int
    L.distil_get_tuning.argtypes = [c_void_p, P(c_int)]
    L.distil_get_tuning.restype = c_int
    L.distil_plan_workspace.argtypes = [P(BatchShape), P(BatchCfg), c_int, P(c_size_t)]
    L.distil_plan_workspace.restype = c_int
    L.distil_plan_create.argtypes = [c_void_p, P(BatchShape), P(BatchCfg), c_int, c_int, c_void_p, c_size_t,
                                     c_void_p, P(c_void_p)]
    L.distil_plan_create.restype = c_int
    L.distil_plan_run.argtypes = [c_void_p, c_void_p]
    L.distil_plan_run.restype = c_int
    L.distil_plan_info.argtypes = [c_void_p, P(c_int), P(c_int)]
    L.distil_plan_info.restype = c_int
    L.distil_plan_destroy.argtypes = [c_void_p]
    L.distil_plan_destroy.restype = None
    L.distil_create.argtypes = [c_int, P(c_void_p)]
    L.distil_create.restype = c_int
    L.distil_destroy.argtypes = [c_void_p]
    L.distil_destroy.restype = None
    L.distil_last_error.argtypes = []
    L.distil_last_error.restype = ctypes.c_char_p
    L.distil_elementals_workspace.argtypes = [c_int, c_int, c_int, c_int, c_int, P(c_size_t)]
    L.distil_elementals_workspace.restype = c_int
    L.distil_elementals.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, P(ctypes.c_int32), c_int, c_int,
                                    c_void_p, c_void_p, c_size_t, c_void_p]
    L.distil_elementals.restype = c_int
    L.distil_correlate_workspace.argtypes = [c_int, c_int, c_int, c_int, c_int, P(c_size_t)]
    L.distil_correlate_workspace.restype = c_int
    L.distil_correlate.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_int,
                                   c_int, c_int, c_void_p, c_void_p, c_size_t, c_void_p]
    L.distil_correlate.restype = c_int
    L.distil_gevp.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]
    L.distil_gevp.restype = c_int
    L.distil_gevp_range.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p,
                                    c_void_p, c_void_p]
    L.distil_gevp_range.restype = c_int
    L.distil_correlate_slice.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p,
                                         c_int, c_int, c_void_p, c_int, c_int, c_void_p, c_size_t, c_void_p]
    L.distil_correlate_slice.restype = c_int
    L.distil_optimal.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_void_p,
                                 c_void_p]
    L.distil_optimal.restype = c_int
    L.distil_profiles_eigen.argtypes = [c_void_p, c_void_p, c_int, c_int, P(ctypes.c_double), c_int, c_void_p,
                                        c_void_p]
    L.distil_profiles_eigen.restype = c_int
    L.distil_set_wait_limit.argtypes = [c_void_p, ctypes.c_longlong]
    L.distil_set_wait_limit.restype = c_int
    L.distil_scan_finite.argtypes = [c_void_p, c_void_p, ctypes.c_longlong, c_int, P(ctypes.c_longlong), c_void_p]
    L.distil_scan_finite.restype = c_int
    L.distil_cgemm_workspace.argtypes = [c_int, c_int, c_int, c_int, c_int, P(c_size_t)]
    L.distil_cgemm_workspace.restype = c_int
    L.distil_cgemm.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int,
                               c_void_p, c_size_t, c_void_p]
    L.distil_cgemm.restype = c_int
    L.distil_correlate_noalloc.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                           c_int, c_int, c_int, c_void_p, c_void_p]
    L.distil_correlate_noalloc.restype = c_int
    L.distil_mode_supported.argtypes = [c_int]
    L.distil_mode_supported.restype = c_int
    L.distil_profile_enable.argtypes = [c_void_p, c_int]
    L.distil_profile_enable.restype = c_int
    L.distil_meson_elementals_workspace.argtypes = [c_int, c_int, c_int, c_int, c_int, P(c_size_t)]
    L.distil_meson_elementals_workspace.restype = c_int
    L.distil_meson_elementals.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, P(ctypes.c_int32),
                                          c_int, c_int, c_void_p, c_void_p, c_size_t, c_void_p]
    L.distil_meson_elementals.restype = c_int
    L.distil_meson_correlate_workspace.argtypes = [c_int, c_int, c_int, c_int, P(c_size_t)]
    L.distil_meson_correlate_workspace.restype = c_int
    L.distil_meson_correlate.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                         c_int, c_int, c_void_p, c_void_p, c_size_t, c_void_p]
    L.distil_meson_correlate.restype = c_int
    L.distil_meson_prune.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                     c_void_p, c_void_p]
    L.distil_meson_prune.restype = c_int
    L.distil_glueball_workspace.argtypes = [c_int, c_int, P(c_size_t)]
    L.distil_glueball_workspace.restype = c_int
    L.distil_glueball_operators.argtypes = [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_size_t,
                                            c_void_p]
    L.distil_glueball_operators.restype = c_int
    L.distil_profile_read.argtypes = [c_void_p, P(KernelStat), c_int, P(c_int)]
    L.distil_profile_read.restype = c_int


def lib(path: str = LIB_PATH):
    """Load the shared library (once).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise DistilError(5, f"{path} not built (python -m paper_2609_37723_b300.build)")
        L = ctypes.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        msg = lib().distil_last_error()
        raise DistilError(status, msg.decode() if msg else "")


def context(device: int = 0):
    if device not in _ctx:
        h = ctypes.c_void_p()
        _check(lib().distil_create(device, ctypes.byref(h)))
        _ctx[device] = h
    return _ctx[device]


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _mode(mode) -> int:
    return MODES[mode] if isinstance(mode, str) else int(mode)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def n_triples(nv: int) -> int:
    return nv * (nv - 1) * (nv - 2) // 6


def elementals_workspace(L: int, nt: int, nv: int, np_: int, mode) -> int:
    b = ctypes.c_size_t()
    _check(lib().distil_elementals_workspace(L, nt, nv, np_, _mode(mode), ctypes.byref(b)))
    return b.value


def correlate_workspace(nt: int, nv: int, np_: int, nb: int, mode) -> int:
    b = ctypes.c_size_t()
    _check(lib().distil_correlate_workspace(nt, nv, np_, nb, _mode(mode), ctypes.byref(b)))
    return b.value


def _workspace(nbytes: int, device):
    import torch
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _nbytes(workspace) -> int:
    """Size of a caller's workspace tensor (the library checks it is enough)."""
    return 0 if workspace is None else int(workspace.numel()) * int(workspace.element_size())


def elementals(v, L: int, mom, mode="fp64", out=None, workspace=None, stream=None):
    """v: [nt][nv][L^3][3] complex tensor on the GPU; mom: [np][3] ints (host)."""
    import torch
    mode = _mode(mode)
    nt, nv = int(v.shape[0]), int(v.shape[1])
    assert v.is_cuda and v.is_contiguous() and v.shape[2] == L ** 3 and v.shape[3] == 3
    mom_np = np.ascontiguousarray(np.asarray(mom, dtype=np.int32).reshape(-1, 3))
    np_ = mom_np.shape[0]
    cdt = torch.complex128 if mode == FP64 else torch.complex64
    assert v.dtype == cdt, f"v must be {cdt} for mode {MODE_NAMES[mode]}"
    odt = torch.complex64 if mode == FP32 else torch.complex128   # tensor-core modes keep c128 elementals
    if out is None:
        out = torch.empty((nt, np_, n_triples(nv)), dtype=odt, device=v.device)
    ws_bytes = elementals_workspace(L, nt, nv, np_, mode)
    if workspace is None:
        workspace = _workspace(ws_bytes, v.device)
    ctx = context(v.device.index or 0)
    _check(lib().distil_elementals(ctx, _ptr(v), L, nt, nv,
                                   mom_np.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), np_, mode,
                                   _ptr(out), _ptr(workspace) if workspace is not None else None,
                                   _nbytes(workspace), _stream(stream)))
    return out


def correlate(phi_snk, phi_src, tau, prof, mode="fp64", prof_per_t: bool = False, out=None,
              workspace=None, stream=None):
    """phi_snk [nt][np][T3], phi_src [np][T3], tau [nt][4nv][4nv], prof [nb][nv] (f64, GPU)."""
    import torch
    mode = _mode(mode)
    nt, np_ = int(phi_snk.shape[0]), int(phi_snk.shape[1])
    nv = int(tau.shape[1]) // 4
    nb = int(prof.shape[-2])
    assert prof.dtype == torch.float64 and prof.is_cuda and prof.is_contiguous()
    for x in (phi_snk, phi_src, tau):
        assert x.is_cuda and x.is_contiguous()
    if out is None:
        out = torch.empty((np_, nb, nb, nt), dtype=torch.complex128, device=tau.device)
    ws_bytes = correlate_workspace(nt, nv, np_, nb, mode)
    if workspace is None:
        workspace = _workspace(ws_bytes, tau.device)
    ctx = context(tau.device.index or 0)
    _check(lib().distil_correlate(ctx, _ptr(phi_snk), _ptr(phi_src), _ptr(tau), nt, nv, np_, _ptr(prof), nb,
                                  int(prof_per_t), mode, _ptr(out),
                                  _ptr(workspace) if workspace is not None else None, _nbytes(workspace),
                                  _stream(stream)))
    return out


def correlate_slice(phi_snk_t, phi_src, tau_t, prof_snk, prof_src, C, t: int, mode="fp64", workspace=None,
                    stream=None):
    """Column t of C[np][nb][nb][nt] from one sink timeslice: phi_snk_t [np][T3],
    phi_src [np][T3], tau_t [4nv][4nv], prof_snk / prof_src [nb][nv] (f64)."""
    mode = _mode(mode)
    np_ = int(phi_snk_t.shape[0])
    nv = int(tau_t.shape[-1]) // 4
    nb = int(prof_snk.shape[-2])
    nt = int(C.shape[-1])
    for x in (phi_snk_t, phi_src, tau_t, prof_snk, prof_src, C):
        assert x.is_cuda and x.is_contiguous()
    ws_bytes = correlate_workspace(1, nv, np_, nb, mode)
    if workspace is None:
        workspace = _workspace(ws_bytes, tau_t.device)
    ctx = context(tau_t.device.index or 0)
    _check(lib().distil_correlate_slice(ctx, _ptr(phi_snk_t), _ptr(phi_src), _ptr(tau_t), nv, np_, _ptr(prof_snk),
                                        _ptr(prof_src), nb, mode, _ptr(C), nt, int(t),
                                        _ptr(workspace) if workspace is not None else None, _nbytes(workspace),
                                        _stream(stream)))
    return C


def cgemm(A, B, mode="fp16x3", out=None, workspace=None, stream=None):
    """C[b] = A[b] @ B[b]^T (complex64, tensor cores, split pieces)."""
    import torch
    mode = _mode(mode)
    if A.dim() == 2:
        A, B = A[None], B[None]
    batch, M, K = (int(s) for s in A.shape)
    N = int(B.shape[1])
    assert A.dtype == torch.complex64 and B.dtype == torch.complex64 and A.is_contiguous() and B.is_contiguous()
    if out is None:
        out = torch.empty((batch, M, N), dtype=torch.complex64, device=A.device)
    b = ctypes.c_size_t()
    _check(lib().distil_cgemm_workspace(M, N, K, batch, mode, ctypes.byref(b)))
    if workspace is None:
        workspace = _workspace(b.value, A.device)
    _check(lib().distil_cgemm(context(A.device.index or 0), _ptr(A), _ptr(B), _ptr(out), M, N, K, batch, mode,
                              _ptr(workspace), _nbytes(workspace), _stream(stream)))
    return out


def gevp(C, t0: int, out=None, stream=None):
    import torch
    np_, nb, _, nt = (int(s) for s in C.shape)
    assert C.dtype == torch.complex128 and C.is_cuda and C.is_contiguous()
    if out is None:
        out = torch.empty((np_, nt, nb), dtype=torch.complex128, device=C.device)
    ctx = context(C.device.index or 0)
    _check(lib().distil_gevp(ctx, _ptr(C), np_, nb, nt, t0, _ptr(out), _stream(stream)))
    return out


def gevp_range(C, t0: int, t_begin: int = 0, t_count: Optional[int] = None, lam=None, vecs=None,
               want_vectors: bool = False, stream=None):
    """Eigenvalues lam[np][nt][nb] (and eigenvectors vecs[np][nt][nb][nb] when
    want_vectors or vecs is given) for timeslices [t_begin, t_begin + t_count)."""
    import torch
    np_, nb, _, nt = (int(s) for s in C.shape)
    t_count = nt - t_begin if t_count is None else int(t_count)
    assert C.dtype == torch.complex128 and C.is_cuda and C.is_contiguous()
    if lam is None:
        lam = torch.full((np_, nt, nb), complex("nan"), dtype=torch.complex128, device=C.device)
    if vecs is None and want_vectors:
        vecs = torch.full((np_, nt, nb, nb), complex("nan"), dtype=torch.complex128, device=C.device)
    ctx = context(C.device.index or 0)
    _check(lib().distil_gevp_range(ctx, _ptr(C), np_, nb, nt, int(t0), int(t_begin), t_count, _ptr(lam),
                                   _ptr(vecs) if vecs is not None else None, _stream(stream)))
    return (lam, vecs) if vecs is not None else lam


def optimal(C, vecs, td: int, stream=None):
    """Optimal-operator correlators copt[np][nb][nt] = u^H C(t) u for the GEVP
    eigenvectors vecs[np][nt][nb][nb] at timeslice td, and their effective
    masses meff[np][nb][nt] (NaN at the last timeslice)."""
    import torch
    np_, nb, _, nt = (int(s) for s in C.shape)
    assert C.is_contiguous() and vecs.is_contiguous() and vecs.shape == (np_, nt, nb, nb)
    copt = torch.empty((np_, nb, nt), dtype=torch.complex128, device=C.device)
    meff = torch.empty((np_, nb, nt), dtype=torch.float64, device=C.device)
    _check(lib().distil_optimal(context(C.device.index or 0), _ptr(C), np_, nb, nt, _ptr(vecs), int(td), _ptr(copt),
                                _ptr(meff), _stream(stream)))
    return copt, meff


def mode_available(mode) -> bool:
    return bool(lib().distil_mode_supported(_mode(mode)))


def device_status(reset: bool = False, device: int = 0) -> int:
    """Code of the first expired bounded device wait since the last reset
    (0 = none); synchronises.  Raises DistilError when it is nonzero."""
    code = ctypes.c_uint()
    _check(lib().distil_device_status(context(device), int(reset), ctypes.byref(code)))
    return int(code.value)


def profiles_eigen(lam, sigmas, stream=None):
    """Profiles exp(-(lam_i / sigma_b)^2) from Laplacian eigenvalues lam
    ([nt][nv] or [nv], f64 on the GPU): [nt][nb][nv] (or [nb][nv])."""
    import torch
    squeeze = lam.dim() == 1
    lam2 = lam[None] if squeeze else lam
    assert lam2.dtype == torch.float64 and lam2.is_cuda and lam2.is_contiguous()
    nt, nv = int(lam2.shape[0]), int(lam2.shape[1])
    sig = (ctypes.c_double * len(sigmas))(*[float(x) for x in sigmas])
    out = torch.empty((nt, len(sigmas), nv), dtype=torch.float64, device=lam.device)
    _check(lib().distil_profiles_eigen(context(lam.device.index or 0), _ptr(lam2), nt, nv, sig, len(sigmas),
                                       _ptr(out), _stream(stream)))
    return out[0] if squeeze else out


def set_wait_limit(cycles: int, device: int = 0):
    """Limit of the tensor-core pipeline waits in clock cycles (<= 0: default)."""
    _check(lib().distil_set_wait_limit(context(device), int(cycles)))


def scan_finite(x, stream=None) -> int:
    """Index of the first NaN/Inf among the real values of tensor x (complex
    tensors are scanned as interleaved reals), or -1; raises DistilError
    (EINVAL) when there is one."""
    import torch
    assert x.is_cuda and x.is_contiguous()
    f32 = x.dtype in (torch.float32, torch.complex64)
    assert f32 or x.dtype in (torch.float64, torch.complex128)
    count = x.numel() * (2 if x.is_complex() else 1)
    bad = ctypes.c_longlong()
    st = lib().distil_scan_finite(context(x.device.index or 0), _ptr(x), count, int(f32), ctypes.byref(bad),
                                  _stream(stream))
    if st != 0 and bad.value < 0:
        _check(st)
    if st != 0:
        raise DistilError(st, lib().distil_last_error().decode())
    return int(bad.value)


def profile_enable(timing: bool = False, device: int = 0):
    """Reset the library's per-kernel launch counters (and event timing)."""
    _check(lib().distil_profile_enable(context(device), int(timing)))


def profile_read(device: int = 0) -> dict:
    """{kernel family: (launches, summed ms)} since profile_enable()."""
    n = ctypes.c_int()
    _check(lib().distil_profile_read(context(device), None, 0, ctypes.byref(n)))
    arr = (KernelStat * max(1, n.value))()
    _check(lib().distil_profile_read(context(device), arr, n.value, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(n.value)}


# ------------------------------------------------------------------ tuning and batched plans

def set_tuning(variants, device: int = 0):
    """Kernel variant of each mode-contraction site {step i, step j, T contraction}:
    0 = one 128 x 128 tile per CTA, 1 = persistent, overlapped epilogue,
    2 (step i only) = persistent with the A tile resident in shared memory."""
    arr = (ctypes.c_int * 3)(*[int(x) for x in variants])
    _check(lib().distil_set_tuning(context(device), arr))


def get_tuning(device: int = 0):
    arr = (ctypes.c_int * 3)()
    _check(lib().distil_get_tuning(context(device), arr))
    return list(arr)


def _batch(L, nt, mom, nb, t0, mode, cfgs):
    mom_np = np.ascontiguousarray(np.asarray(mom, dtype=np.int32).reshape(-1, 3))
    shape = BatchShape(int(L), int(nt), int(mom_np.shape[0]), int(nb), int(t0), _mode(mode),
                       mom_np.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    arr = (BatchCfg * len(cfgs))()
    for i, c in enumerate(cfgs):
        arr[i] = BatchCfg(int(c["nv"]), c["v"].data_ptr() if "v" in c else None,
                          c["tau"].data_ptr() if "tau" in c else None,
                          c["prof"].data_ptr() if "prof" in c else None,
                          c["C"].data_ptr() if "C" in c else None,
                          c["lam"].data_ptr() if c.get("lam") is not None else None)
    return shape, arr, mom_np


def plan_workspace(L, nt, mom, nb, mode, nvs) -> int:
    """Workspace bytes of a plan over configurations with these N_v (no device needed)."""
    shape, arr, _keep = _batch(L, nt, mom, nb, 0, mode, [{"nv": nv} for nv in nvs])
    b = ctypes.c_size_t()
    _check(lib().distil_plan_workspace(ctypes.byref(shape), arr, len(nvs), ctypes.byref(b)))
    return b.value


def tuning_cache_key(gpu_name: str, L: int, nt: int, np_: int, nb: int, mode, nvs) -> str:
    """Key of a tuned plan in the tuning cache: the GPU and the shape the
    variants were timed on (the autotuner times the first configuration; the
    largest N_v of the ensemble is part of the key)."""
    return f"{gpu_name}|L{int(L)}|nt{int(nt)}|np{int(np_)}|nb{int(nb)}|{MODE_NAMES[_mode(mode)]}|nv{max(nvs)}"


def load_tuning_cache(path: str) -> dict:
    """{key: [variants]} from a JSON tuning cache ({} if absent or unreadable)."""
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        return {k: [int(x) for x in v] for k, v in d.items() if isinstance(v, list) and len(v) == 3}
    except (OSError, ValueError):
        return {}


def store_tuning(path: str, key: str, variants) -> None:
    """Add or replace one entry of the JSON tuning cache (written to a
    temporary file, then renamed over the old one)."""
    import json
    d = load_tuning_cache(path)
    d[key] = [int(x) for x in variants]
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Plan:
    """An ensemble of configurations (shared L, nt, momenta, nb, mode; each
    with its own N_v) captured into one CUDA graph.  cfgs: list of dicts
    with device tensors v, tau, prof (f64 [nb][nv]) and outputs C
    ([np][nb][nb][nt] c128) and optionally lam ([np][nt][nb] c128).
    tuning_cache: path of a JSON file of autotuned kernel variants keyed by
    GPU name and shape; a hit skips the autotuner, a miss stores its choice."""

    def __init__(self, L, nt, mom, nb, t0, mode, cfgs, autotune=True, stream=None, tuning_cache=None):
        import torch
        self.cfgs = cfgs
        dev = cfgs[0]["v"].device
        self.device = dev.index or 0
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.cache_hit = False
        key = None
        if tuning_cache is not None and autotune:
            key = tuning_cache_key(torch.cuda.get_device_name(dev), L, nt, len(np.asarray(mom).reshape(-1, 3)), nb,
                                   mode, [int(c["nv"]) for c in cfgs])
            hit = load_tuning_cache(tuning_cache).get(key)
            if hit is not None:
                set_tuning(hit, device=self.device)
                autotune, self.cache_hit = False, True
        shape, arr, self._mom = _batch(L, nt, mom, nb, t0, mode, cfgs)
        b = ctypes.c_size_t()
        _check(lib().distil_plan_workspace(ctypes.byref(shape), arr, len(cfgs), ctypes.byref(b)))
        self.workspace = torch.empty(b.value, dtype=torch.uint8, device=dev)
        torch.cuda.current_stream(dev).synchronize()   # inputs written on other streams are visible
        h = ctypes.c_void_p()
        _check(lib().distil_plan_create(context(self.device), ctypes.byref(shape), arr, len(cfgs), int(autotune),
                                        _ptr(self.workspace), b.value, ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h)))
        self.handle = h
        if key is not None and not self.cache_hit:
            store_tuning(tuning_cache, key, self.info()[0])

    def run(self, stream=None):
        s = self.stream if stream is None else stream
        _check(lib().distil_plan_run(self.handle, ctypes.c_void_p(s.cuda_stream)))

    def info(self):
        v = (ctypes.c_int * 3)()
        k = ctypes.c_int()
        _check(lib().distil_plan_info(self.handle, v, ctypes.byref(k)))
        return list(v), int(k.value)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.distil_plan_destroy(h)
            self.handle = None


# ------------------------------------------------------------------ mesons


def meson_elementals_workspace(L: int, nt: int, nv: int, np_: int, mode="fp16x6") -> int:
    b = ctypes.c_size_t()
    _check(lib().distil_meson_elementals_workspace(L, nt, nv, np_, _mode(mode), ctypes.byref(b)))
    return b.value


def meson_elementals(v, U, L: int, mom, mode="fp16x6", out=None, workspace=None, stream=None):
    """v [nt][nv][L^3][3] c64, U [nt][3][L^3][3][3] c64 (GPU); mom [np][3]
    ints (host) -> phi [nt][np][7][nv][nv] c128."""
    import torch
    mode = _mode(mode)
    nt, nv = int(v.shape[0]), int(v.shape[1])
    V3 = L ** 3
    assert v.is_cuda and v.is_contiguous() and v.dtype == torch.complex64 and tuple(v.shape[2:]) == (V3, 3)
    assert U.is_cuda and U.is_contiguous() and U.dtype == torch.complex64 and tuple(U.shape) == (nt, 3, V3, 3, 3)
    mom_np = np.ascontiguousarray(np.asarray(mom, dtype=np.int32).reshape(-1, 3))
    np_ = mom_np.shape[0]
    if out is None:
        out = torch.empty((nt, np_, 7, nv, nv), dtype=torch.complex128, device=v.device)
    if workspace is None:
        workspace = _workspace(meson_elementals_workspace(L, nt, nv, np_, mode), v.device)
    _check(lib().distil_meson_elementals(context(v.device.index or 0), _ptr(v), _ptr(U), L, nt, nv,
                                         mom_np.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), np_, mode,
                                         _ptr(out), _ptr(workspace), _nbytes(workspace), _stream(stream)))
    return out


def meson_correlate_workspace(nv: int, np_: int, nb: int, mode="fp16x6") -> int:
    b = ctypes.c_size_t()
    _check(lib().distil_meson_correlate_workspace(nv, np_, nb, _mode(mode), ctypes.byref(b)))
    return b.value


def meson_correlate(phi_snk, phi_src, tau, prof, mode="fp16x6", out=None, workspace=None, stream=None):
    """phi_snk [nt][np][7][nv][nv], phi_src [np][7][nv][nv] (c128), tau
    [nt][4nv][4nv] (c64), prof [nb][nv] (f64) -> C [np][3nb][3nb][nt] c128."""
    import torch
    mode = _mode(mode)
    nt, np_, _, nv, _ = (int(x) for x in phi_snk.shape)
    nb = int(prof.shape[0])
    for x in (phi_snk, phi_src, tau, prof):
        assert x.is_cuda and x.is_contiguous()
    assert phi_snk.dtype == torch.complex128 and phi_src.dtype == torch.complex128
    assert tau.dtype == torch.complex64 and prof.dtype == torch.float64
    if out is None:
        out = torch.empty((np_, 3 * nb, 3 * nb, nt), dtype=torch.complex128, device=tau.device)
    if workspace is None:
        workspace = _workspace(meson_correlate_workspace(nv, np_, nb, mode), tau.device)
    _check(lib().distil_meson_correlate(context(tau.device.index or 0), _ptr(phi_snk), _ptr(phi_src), _ptr(tau),
                                        nt, nv, np_, _ptr(prof), nb, mode, _ptr(out), _ptr(workspace),
                                        _nbytes(workspace), _stream(stream)))
    return out


def meson_prune(C, t_prune: int, nkeep: int, stream=None):
    """C [np][nops][nops][nt] c128 -> (Ct [np][nkeep][nkeep][nt], Un
    [np][nops][nkeep], singular values [np][nops])."""
    import torch
    np_, nops, _, nt = (int(x) for x in C.shape)
    assert C.is_cuda and C.is_contiguous() and C.dtype == torch.complex128
    Ct = torch.empty((np_, nkeep, nkeep, nt), dtype=torch.complex128, device=C.device)
    Un = torch.empty((np_, nops, nkeep), dtype=torch.complex128, device=C.device)
    sv = torch.empty((np_, nops), dtype=torch.float64, device=C.device)
    _check(lib().distil_meson_prune(context(C.device.index or 0), _ptr(C), np_, nops, nt, int(t_prune), int(nkeep),
                                    _ptr(Ct), _ptr(Un), _ptr(sv), _stream(stream)))
    return Ct, Un, sv


# ---------------------------------------------------------------- glueballs


def glueball_workspace(L: int, nt: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().distil_glueball_workspace(L, nt, ctypes.byref(b)))
    return b.value


def glueball_operators(U, L: int, out=None, workspace=None, stream=None):
    """U [nt][3][L^3][3][3] c64 (GPU) -> O [nt][5] c128, the five A1-+
    glueball operators of every timeslice."""
    import torch
    nt = int(U.shape[0])
    assert U.is_cuda and U.is_contiguous() and U.dtype == torch.complex64 and tuple(U.shape[1:]) == (3, L ** 3, 3, 3)
    if out is None:
        out = torch.empty((nt, 5), dtype=torch.complex128, device=U.device)
    if workspace is None:
        workspace = _workspace(glueball_workspace(L, nt), U.device)
    _check(lib().distil_glueball_operators(context(U.device.index or 0), _ptr(U), L, nt, _ptr(out), _ptr(workspace),
                                           _nbytes(workspace), _stream(stream)))
    return out
