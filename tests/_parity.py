"""Parity criteria shared by the GPU tests.

Forward (per level i of each signal, against the FP64 oracle):
    ||Y_gpu - Y_ref||_2 / ||Y_ref||_2 <= 2e-6 * i
    max |Y_gpu - Y_ref|              <= 1e-5 * ||x||_2
Adjoint (per signal): ||gx_gpu - gx_ref||_2 / ||gx_ref||_2 <= 1e-5 and
    max |gx_gpu - gx_ref| <= 1e-5 * ||gy||_2.
"""
import numpy as np

REL_PER_LEVEL = 2e-6
ABS_FRAC = 1e-5
ADJ_REL = 1e-5


def check_forward_levels(y_gpu, y_ref, x, what=""):
    """y_gpu [m, N] complex64, y_ref [m, N] complex128, x [N]."""
    xn = float(np.linalg.norm(np.asarray(x, dtype=np.complex128)))
    worst = 0.0
    for i in range(y_ref.shape[0]):
        d = y_gpu[i].astype(np.complex128) - y_ref[i]
        ref_n = float(np.linalg.norm(y_ref[i]))
        rel = float(np.linalg.norm(d)) / ref_n if ref_n > 0 else float(np.linalg.norm(d))
        mx = float(np.abs(d).max())
        assert rel <= REL_PER_LEVEL * (i + 1), f"{what} level {i + 1}: rel L2 {rel:.3e}"
        assert mx <= ABS_FRAC * xn + 1e-30, f"{what} level {i + 1}: max abs {mx:.3e} (||x|| {xn:.3e})"
        worst = max(worst, rel / (REL_PER_LEVEL * (i + 1)))
    return worst


def check_adjoint(gx_gpu, gx_ref, gy, what=""):
    d = gx_gpu.astype(np.complex128) - gx_ref
    rel = float(np.linalg.norm(d) / np.linalg.norm(gx_ref))
    mx = float(np.abs(d).max())
    gn = float(np.linalg.norm(np.asarray(gy, dtype=np.complex128)))
    assert rel <= ADJ_REL, f"{what} adjoint rel L2 {rel:.3e}"
    assert mx <= ABS_FRAC * gn, f"{what} adjoint max abs {mx:.3e}"
    return rel
