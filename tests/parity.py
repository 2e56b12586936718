"""Error measures used by the parity tests.

Correlator entries are gated per entry, e_ab(t) = |C_gpu - C_ref| / |C_ref|;
an entry whose reference is below 1e-10 of the largest |C(t)| at that
(p, t) is gated normwise instead (relative to that largest entry).
"""
import numpy as np


def c_entry_errors(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """got, ref: [np][nb][nb][nt] -> per-entry relative errors (same shape)."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    denom = np.abs(ref)
    tiny = denom < 1e-10 * scale
    denom = np.where(tiny, np.maximum(scale, 1e-300), denom)
    return np.abs(got - ref) / denom


def max_c_error(got, ref) -> float:
    return float(c_entry_errors(got, ref).max())


def normwise(got, ref, axis=None) -> float:
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def phi_error(got, ref) -> float:
    """Elementals: max over (t, p) of max_r |dPhi| / max_r |Phi| (entries of
    a random elemental vary over orders of magnitude; a per-(t,p) scale keeps
    near-zero entries from dominating)."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    scale = np.maximum(np.abs(ref).max(axis=-1, keepdims=True), 1e-300)
    return float((np.abs(got - ref) / scale).max())


def c_scaled_errors(got, ref) -> np.ndarray:
    """Per-entry error relative to the scale of its matrix C(p, t):
    |dC_ab(t)| / max_a'b' |C_a'b'(t)|  ->  [np][nb][nb][nt]."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    scale = np.maximum(np.abs(ref).max(axis=(1, 2), keepdims=True), 1e-300)
    return np.abs(got - ref) / scale


def max_c_scaled_error(got, ref) -> float:
    return float(c_scaled_errors(got, ref).max())


def c_operator_scaled_errors(got, ref) -> np.ndarray:
    """Per-entry error relative to the magnitude of the two operators the
    entry couples: |dC_ab(t)| / sqrt(R_a(t) R_b(t)), R_a = the largest
    |C| in row a or column a at (p, t).  For matrices whose operators differ
    in magnitude by orders (derivative and profile operators of very
    different widths), where single entries can be 1e-5 of the largest one."""
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    A = np.abs(ref)
    R = np.maximum(A.max(axis=2), A.max(axis=1))
    scale = np.sqrt(R[:, :, None, :] * R[:, None, :, :])
    return np.abs(got - ref) / np.maximum(scale, 1e-300)


def max_c_operator_scaled_error(got, ref) -> float:
    return float(c_operator_scaled_errors(got, ref).max())
