"""FP64 CPU oracle for the multiresolution DFT (MrDFT) -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs may import this module.  The
product path (the CUDA library and its binding) never touches it, and it never
touches the product path: the two share no code, tables or helpers.

Paper: Andreatto & Cariow, "An algorithm for fast computation of the
multiresolution discrete Fourier transform" (arXiv:1507.02525).

What is computed (Sec. 2, Eq. 1): for x of length N = 2^m and each level
i = 1..m, the spectra of the N/2^i non-overlapping rectangular windows of
length 2^i, unnormalised, sign exp(-j 2 pi n k / 2^i), bins in natural order,
levels stacked as ``y[i-1, w*2^i + k]``.

The C part (``mrdft_oracle.c``) holds the definition evaluated directly, a
separate per-window radix-2 FFT, the adjoint both ways, and the paper's
rationalised procedure (Eq. 4) with operation counting (Eqs. 6-7).  The dense
matrices of Sec. 3 / Sec. 4 are built in :mod:`oracle.matrices`.

Every function takes and returns numpy arrays (complex128 in, complex128 out).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrdft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmrdft_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in place (gcc, FP64, OpenMP, portable flags)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            for name in ("mro_forward_direct", "mro_forward_fft",
                         "mro_adjoint_direct", "mro_adjoint_fft"):
                f = getattr(lib, name)
                f.argtypes = [dp, ctypes.c_int, dp]
                f.restype = ctypes.c_int
            lib.mro_forward_level_fft.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.mro_forward_level_fft.restype = ctypes.c_int
            lib.mro_bin.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp]
            lib.mro_bin.restype = ctypes.c_int
            lib.mro_rationalized.argtypes = [dp, ctypes.c_int, dp, i64p, ctypes.c_int]
            lib.mro_rationalized.restype = ctypes.c_int
            lib.mro_set_num_threads.argtypes = [ctypes.c_int]
            lib.mro_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _log2_len(n: int) -> int:
    m = int(n).bit_length() - 1
    if n < 2 or (1 << m) != n:
        raise ValueError(f"signal length must be a power of two >= 2, got {n}")
    return m


def set_num_threads(n: int) -> None:
    _load().mro_set_num_threads(int(n))


def num_threads() -> int:
    return int(_load().mro_num_threads())


def forward(x, method: str = "auto") -> np.ndarray:
    """MrDFT of one signal (Eq. 1).  Returns complex128 array of shape [m, N].

    method: "direct" (Eq. 1 term by term), "fft" (per-window radix-2 FFT) or
    "auto" (direct for N <= 2^12, else fft).
    """
    x = _as_c128(x).reshape(-1)
    m = _log2_len(x.size)
    if method == "auto":
        method = "direct" if m <= 12 else "fft"
    y = np.empty((m, x.size), dtype=np.complex128)
    fn = {"direct": _load().mro_forward_direct, "fft": _load().mro_forward_fft}[method]
    rc = fn(_dptr(x), m, _dptr(y))
    if rc:
        raise RuntimeError(f"oracle forward failed ({rc})")
    return y


def forward_level(x, level: int) -> np.ndarray:
    """Level ``level`` (1-based) of Eq. 1 only, via the per-window FFT: [N]."""
    x = _as_c128(x).reshape(-1)
    m = _log2_len(x.size)
    y = np.empty(x.size, dtype=np.complex128)
    rc = _load().mro_forward_level_fft(_dptr(x), m, int(level), _dptr(y))
    if rc:
        raise RuntimeError(f"oracle forward_level failed ({rc})")
    return y


def bin_value(x, level: int, pos: int) -> complex:
    """One output bin Y^(level)[pos] by the direct sum of Eq. 1."""
    x = _as_c128(x).reshape(-1)
    m = _log2_len(x.size)
    out = np.zeros(2, dtype=np.float64)
    rc = _load().mro_bin(_dptr(x), m, int(level), int(pos), _dptr(out))
    if rc:
        raise RuntimeError(f"oracle bin failed ({rc})")
    return complex(out[0], out[1])


def adjoint(gy, method: str = "auto") -> np.ndarray:
    """Conjugate transpose of Eq. 1: gy [m, N] -> x_bar [N] (complex128)."""
    gy = _as_c128(gy)
    if gy.ndim != 2:
        raise ValueError("gy must have shape [m, N]")
    m = _log2_len(gy.shape[1])
    if gy.shape[0] != m:
        raise ValueError("gy must have m = log2(N) levels")
    if method == "auto":
        method = "direct" if m <= 12 else "fft"
    gx = np.empty(gy.shape[1], dtype=np.complex128)
    fn = {"direct": _load().mro_adjoint_direct, "fft": _load().mro_adjoint_fft}[method]
    rc = fn(_dptr(gy), m, _dptr(gx))
    if rc:
        raise RuntimeError(f"oracle adjoint failed ({rc})")
    return gx


def rationalized(x=None, m: int | None = None, compute: bool = True):
    """The paper's procedure, Eq. 4, with operation counts (Eqs. 6, 7).

    Returns (y, counts) where y is [m, N] complex128 in natural bin order (None
    when ``compute`` is False) and counts is an int64 array [m, 3]:
    (complex multiplications incl. trivial twiddles, non-trivial
    multiplications, complex additions) per iteration i = 1..m.
    """
    lib = _load()
    counts = np.zeros((m if x is None else _log2_len(np.asarray(x).size), 3),
                      dtype=np.int64)
    i64p = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if compute:
        x = _as_c128(x).reshape(-1)
        m = _log2_len(x.size)
        y = np.empty((m, x.size), dtype=np.complex128)
        rc = lib.mro_rationalized(_dptr(x), m, _dptr(y), i64p, 1)
    else:
        if m is None:
            m = _log2_len(np.asarray(x).size)
        y = None
        rc = lib.mro_rationalized(None, int(m), None, i64p, 0)
    if rc:
        raise RuntimeError(f"oracle rationalized failed ({rc})")
    return y, counts


# ------------------------------------------------------------------ batches

def forward_batch(xs, method: str = "auto"):
    """Forward for a list of signals (uneven lengths allowed): list of [m_s, N_s]."""
    return [forward(x, method) for x in xs]


def adjoint_batch(gys, method: str = "auto"):
    return [adjoint(g, method) for g in gys]
