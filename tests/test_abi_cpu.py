"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point include/mrdft.h declares, and argument validation
rejects bad requests before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrdft.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1507_02525_gb300 import _lib
    return _lib.load()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(mrdft_[a-z_]+)\s*\(", text)))


def test_header_declares_abi():
    names = _declared()
    for required in ("mrdft_plan", "mrdft_forward", "mrdft_adjoint", "mrdft_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1507_02525_gb300 import _lib
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_lib.EXPORTS) == set(_declared())


def test_built_for_sm103a():
    from paper_1507_02525_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def _plan(lib, lengths, batch, dtype=0, flags=0):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * len(lengths))(*lengths)
    st = lib.mrdft_plan(ctypes.byref(h), arr, len(lengths), batch, dtype, flags)
    return st, h


@pytest.mark.parametrize("lengths,batch", [([0], 1), ([1], 1), ([3], 1), ([6], 2), ([1 << 27], 1),
                                          ([8, 12], 2), ([8], 0), ([8, 8, 8], 2), ([-4], 1)])
def test_plan_rejects_bad_lengths(lib, lengths, batch):
    st, h = _plan(lib, lengths, batch)
    assert st == 1  # MRDFT_EINVAL
    assert h.value is None
    msg = lib.mrdft_last_error(None).decode()
    assert msg and msg != "no error"


def test_plan_rejects_bad_dtype_and_flags(lib):
    assert _plan(lib, [16], 1, dtype=7)[0] == 1
    assert _plan(lib, [16], 1, flags=0x80)[0] == 1


def test_plan_opts_rejects_bad_shapes(lib):
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 1)(1 << 16)
    for seg, streams in ((11, 0), (27, 0), (-1, 0), (0, 17), (0, -2)):
        st = lib.mrdft_plan_opts(ctypes.byref(h), arr, 1, 1, 0, 0, seg, streams)
        assert st == 1, (seg, streams)  # MRDFT_EINVAL, before any device work
        assert h.value is None


def test_null_arguments(lib):
    assert lib.mrdft_plan(None, None, 1, 1, 0, 0) == 1
    assert lib.mrdft_forward(None, None, None, None) == 1
    assert lib.mrdft_adjoint(None, None, None, None) == 1
    assert lib.mrdft_forward_host(None, None, None, None) == 1
    assert lib.mrdft_loss_grad(None, None, None, None, None, None, None) == 1
    # NULL polls the allocation-free entry point's status word: OK where it
    # never ran, ECUDA where there is no device to ask
    assert lib.mrdft_status_poll(None) in (0, 3)
    assert lib.mrdft_plan_graph_stats(None, None, None, None) == 1
    assert lib.mrdft_debug_item(None, 1, 0, None, None) == 1
    n = ctypes.c_int64()
    assert lib.mrdft_output_elems(None, ctypes.byref(n)) == 1
    assert lib.mrdft_plan_info(None, None, None, None) == 1
    lib.mrdft_destroy(None)  # no-op
    assert lib.mrdft_last_error(None)


def test_python_plan_raises(lib):
    from paper_1507_02525_gb300 import _lib
    with pytest.raises(_lib.MrdftError) as e:
        _lib.Plan([12])
    assert e.value.status == _lib.MRDFT_EINVAL


def test_api_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_1507_02525_gb300 import api
    with pytest.raises(ValueError):
        api.mrdft(torch.zeros(16, dtype=torch.complex64))


@pytest.mark.parametrize("field,value", [("seg_log", 11), ("seg_log", 27), ("streams", 17), ("fwd_cb", 8),
                                         ("fwd_cb", 12), ("adj_cb", 11), ("fwd_rows_prefetch", 3),
                                         ("dual_cols", -1), ("fwd_tree", 7), ("adj_rows13", 5),
                                         ("tile_lean", 4), ("top_cols_early", 9), ("top_overlap", 3),
                                         ("tile_split", 65), ("levels_parallel", 4)])
def test_plan_ex_rejects_bad_options(lib, field, value):
    """Every execution option is range-checked before any device work."""
    from paper_1507_02525_gb300 import _lib
    h = ctypes.c_void_p()
    arr = (ctypes.c_int64 * 1)(1 << 16)
    o = _lib.ExecOpts()
    setattr(o, field, value)
    assert lib.mrdft_plan_ex(ctypes.byref(h), arr, 1, 1, 0, 0, ctypes.byref(o)) == 1
    assert h.value is None
    assert "mrdft_plan_ex" in lib.mrdft_last_error(None).decode()


def test_exec_opts_layout_matches_header():
    """The ctypes mirror of mrdft_exec_opts has the header's fields, in order."""
    from paper_1507_02525_gb300 import _lib
    hdr = open(HEADER).read()
    body = re.search(r"typedef struct \{([^}]*)\} mrdft_exec_opts;", hdr).group(1)
    fields = re.findall(r"int32_t (\w+);", body)
    assert fields == [n for n, _ in _lib.ExecOpts._fields_]
    assert ctypes.sizeof(_lib.ExecOpts) == 4 * len(fields)


def test_exec_opts_from_dict():
    from paper_1507_02525_gb300 import _lib
    o = _lib.ExecOpts.from_dict({"seg_log": 21, "dual_cols": False, "fwd_tree": True, "fwd_cb": 10})
    assert (o.seg_log, o.dual_cols, o.fwd_tree, o.fwd_cb, o.streams) == (21, _lib.OPT_OFF, _lib.OPT_ON, 10, 0)
    assert o.to_dict()["fwd_rows_prefetch"] is None
    with pytest.raises(ValueError):
        _lib.ExecOpts.from_dict({"tile_log": 13})
