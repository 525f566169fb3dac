"""The allocation-free entry point, mrdft_forward_noalloc, against the FP64
oracle and against mrdft_forward.

mrdft_forward_noalloc serves callers that must not call cudaMalloc (an
external memory manager owns all device memory, or a hot loop cannot afford
an allocation's implicit synchronisation): it keeps the two-pass levels'
intermediate in a fixed device array instead of plan-owned scratch.  Every
level of its output must match the oracle within the parity tolerance, and
the planned forward too; two calls in a row must both be right (the shared
array keeps the previous call's contents); and its device status word, read
with mrdft_status_poll(NULL), must report no skipped work item.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1507_02525_gb300 import _lib, inputs  # noqa: E402

from tests._parity import ABS_FRAC, REL_PER_LEVEL  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _planned(x):
    n = x.size
    plan = _lib.Plan([n], 1)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(plan.out_elems, dtype=torch.complex64, device="cuda")
    plan.forward(xt.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _noalloc(x):
    n = x.size
    m = n.bit_length() - 1
    xt = torch.from_numpy(x).cuda()
    y = torch.empty(m * n, dtype=torch.complex64, device="cuda")
    lib = _lib.load()
    st = lib.mrdft_forward_noalloc(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(y.data_ptr()), n,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.MRDFT_OK, lib.mrdft_last_error(None).decode()
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _poll_noalloc():
    lib = _lib.load()
    st = lib.mrdft_status_poll(None)
    assert st == _lib.MRDFT_OK, lib.mrdft_last_error(None).decode()


def _close(y_new, y_ref, x):
    m = x.size.bit_length() - 1
    xn = float(np.linalg.norm(x.astype(np.complex128)))
    a = y_new.reshape(m, -1).astype(np.complex128)
    b = y_ref.reshape(m, -1).astype(np.complex128)
    for i in range(m):
        d = a[i] - b[i]
        assert np.linalg.norm(d) <= REL_PER_LEVEL * (i + 1) * np.linalg.norm(b[i]), f"level {i + 1}"
        assert np.abs(d).max() <= ABS_FRAC * xn, f"level {i + 1}"


@pytest.mark.parametrize("m", [16, 15, 14, 13, 12, 10, 5, 4, 3, 1])
def test_noalloc_matches_oracle_and_forward_twice(oracle, m):
    n = 1 << m
    xa = inputs.complex_signals(1, n, seed=900 + m)[0]
    xb = inputs.complex_signals(1, n, seed=950 + m)[0]
    ya1 = _noalloc(xa)
    yb = _noalloc(xb)  # second call in a row, other data, same shared scratch
    ya2 = _noalloc(xa)
    _poll_noalloc()
    for y, x in ((ya1, xa), (yb, xb)):
        _close(y, oracle.forward(x.astype(np.complex128)).reshape(-1), x)
        _close(y, _planned(x), x)
    np.testing.assert_array_equal(ya1, ya2)


def test_noalloc_rejects_oversize_and_bad_arguments():
    lib = _lib.load()
    buf = torch.empty(16, dtype=torch.complex64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.mrdft_forward_noalloc(p, p, 1 << 17, None) == _lib.MRDFT_EINVAL
    assert "exceeds" in lib.mrdft_last_error(None).decode()
    assert lib.mrdft_forward_noalloc(p, p, 12, None) == _lib.MRDFT_EINVAL
    assert lib.mrdft_forward_noalloc(None, p, 16, None) == _lib.MRDFT_EINVAL
