"""ctypes binding of the C ABI in ``include/mrdft.h`` (argument marshalling only).

Every step of the transform runs in the CUDA library; this module only
passes device pointers, sizes and stream handles.  Loading fails loudly when
``libmrdft.so`` is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrdft.so")

MRDFT_OK = 0
MRDFT_EINVAL = 1
MRDFT_ENOMEM = 2
MRDFT_ECUDA = 3
MRDFT_EUNSUPPORTED = 4
MRDFT_ETIMEOUT = 5
MRDFT_EDEVICE = 6
MRDFT_C64 = 0
MRDFT_R32 = 1
MRDFT_FLAG_GRAPH = 1
MRDFT_FLAG_BITREV = 2

STATUS_NAMES = {0: "MRDFT_OK", 1: "MRDFT_EINVAL", 2: "MRDFT_ENOMEM", 3: "MRDFT_ECUDA",
                4: "MRDFT_EUNSUPPORTED", 5: "MRDFT_ETIMEOUT", 6: "MRDFT_EDEVICE"}

# every entry point declared in include/mrdft.h
EXPORTS = ("mrdft_plan", "mrdft_plan_opts", "mrdft_plan_ex", "mrdft_plan_get_opts", "mrdft_output_elems", "mrdft_input_elems", "mrdft_forward",
           "mrdft_adjoint", "mrdft_forward_host", "mrdft_status_poll", "mrdft_last_error",
           "mrdft_plan_info", "mrdft_timing_enable", "mrdft_timing_read", "mrdft_loss_grad",
           "mrdft_forward_noalloc", "mrdft_plan_graph_stats", "mrdft_debug_item", "mrdft_destroy")
NOALLOC_MAX_LOG = 16

KINDS = ("fwd_tile", "fwd_tiny", "fwd_window", "fwd_cols", "fwd_rows",
         "adj_tile", "adj_tiny", "adj_window", "adj_rows", "adj_cols")


OPT_DEFAULT, OPT_OFF, OPT_ON = 0, 1, 2


class ExecOpts(ctypes.Structure):
    """mrdft_exec_opts (include/mrdft.h): 0 = library default; switches 1 = off, 2 = on."""
    _fields_ = [(n, ctypes.c_int32) for n in ("seg_log", "streams", "fwd_cb", "adj_cb", "fwd_rows_prefetch",
                                               "fwd_rows14", "adj_rows13", "dual_cols", "fwd_tree", "tile_first",
                                               "tile_lean", "fwd_rows12", "tile_split", "top_cols_early",
                                               "top_overlap", "levels_parallel")]
    SWITCHES = ("fwd_rows_prefetch", "fwd_rows14", "adj_rows13", "dual_cols", "fwd_tree", "tile_first", "tile_lean",
                "fwd_rows12", "top_cols_early", "top_overlap", "levels_parallel")

    @classmethod
    def from_dict(cls, d):
        """Fields by name; switches may be given as bools."""
        o = cls()
        for k, v in (d or {}).items():
            if k not in dict(cls._fields_):
                raise ValueError(f"unknown execution option {k!r}")
            if k in cls.SWITCHES and isinstance(v, bool):
                v = OPT_ON if v else OPT_OFF
            setattr(o, k, int(v or 0))
        return o

    def to_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_}
        for k in self.SWITCHES:
            d[k] = {OPT_ON: True, OPT_OFF: False}.get(d[k], None)
        return d


class MrdftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libmrdft.so (building it from source first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            if _build.is_stale():
                _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"MrDFT CUDA library not found at {LIB_PATH}; "
                               "run paper_1507_02525_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
        lib.mrdft_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i64, i32, u32]
        lib.mrdft_plan_opts.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i64, i32, u32, i32, i32]
        lib.mrdft_plan_ex.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), i64, i64, i32, u32,
                                      ctypes.POINTER(ExecOpts)]
        lib.mrdft_plan_get_opts.argtypes = [vp, ctypes.POINTER(ExecOpts)]
        lib.mrdft_output_elems.argtypes = [vp, ctypes.POINTER(i64)]
        lib.mrdft_input_elems.argtypes = [vp, ctypes.POINTER(i64)]
        lib.mrdft_forward.argtypes = [vp, vp, vp, vp]
        lib.mrdft_adjoint.argtypes = [vp, vp, vp, vp]
        lib.mrdft_forward_host.argtypes = [vp, vp, vp, vp]
        lib.mrdft_status_poll.argtypes = [vp]
        lib.mrdft_last_error.argtypes = [vp]
        lib.mrdft_last_error.restype = ctypes.c_char_p
        lib.mrdft_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib.mrdft_timing_enable.argtypes = [vp, i32]
        lib.mrdft_timing_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.mrdft_loss_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.mrdft_forward_noalloc.argtypes = [vp, vp, i64, vp]
        lib.mrdft_forward_noalloc.restype = ctypes.c_int
        lib.mrdft_plan_graph_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i64),
                                               ctypes.POINTER(i64)]
        lib.mrdft_debug_item.argtypes = [vp, i32, i64, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32)]
        lib.mrdft_destroy.argtypes = [vp]
        lib.mrdft_destroy.restype = None
        for name in ("mrdft_plan", "mrdft_plan_opts", "mrdft_plan_ex", "mrdft_plan_get_opts", "mrdft_output_elems", "mrdft_input_elems", "mrdft_forward",
                     "mrdft_adjoint", "mrdft_forward_host", "mrdft_status_poll", "mrdft_plan_info",
                     "mrdft_timing_enable", "mrdft_timing_read", "mrdft_loss_grad", "mrdft_plan_graph_stats",
                     "mrdft_debug_item"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def forward_noalloc(x_ptr: int, y_ptr: int, n: int, stream: int = 0) -> None:
    """mrdft_forward_noalloc: one complex64 signal, no plan, no allocation."""
    lib = load()
    check(lib.mrdft_forward_noalloc(ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(n),
                                    ctypes.c_void_p(stream)), None)


def check(status: int, plan=None) -> None:
    if status != MRDFT_OK:
        msg = load().mrdft_last_error(plan).decode(errors="replace")
        raise MrdftError(status, msg)


class Plan:
    """Owner of an ``mrdft_plan_t`` (see ``mrdft_plan`` in include/mrdft.h)."""

    def __init__(self, lengths, batch: int | None = None, real_input: bool = False,
                 graph: bool = False, seg_log: int | None = None, streams: int | None = None,
                 opts: dict | None = None, bitrev: bool = False):
        """``opts``: execution options by name (mrdft_exec_opts); ``seg_log`` and
        ``streams`` are shorthands for two of them."""
        lib = load()
        lengths = [int(v) for v in (lengths if hasattr(lengths, "__len__") else [lengths])]
        if batch is None:
            batch = len(lengths)
        arr = (ctypes.c_int64 * len(lengths))(*lengths)
        h = ctypes.c_void_p()
        o = dict(opts or {})
        if seg_log:
            o["seg_log"] = seg_log
        if streams:
            o["streams"] = streams
        eo = ExecOpts.from_dict(o)
        st = lib.mrdft_plan_ex(ctypes.byref(h), arr, len(lengths), int(batch),
                               MRDFT_R32 if real_input else MRDFT_C64,
                               (MRDFT_FLAG_GRAPH if graph else 0) | (MRDFT_FLAG_BITREV if bitrev else 0),
                               ctypes.byref(eo))
        check(st, None)
        self._h = h
        self._lib = lib
        self.batch = int(batch)
        self.lengths = lengths if len(lengths) == batch else lengths * batch
        self.real_input = real_input
        self.graph = graph
        self.seg_log = seg_log
        self.streams = streams
        n = ctypes.c_int64()
        check(lib.mrdft_output_elems(h, ctypes.byref(n)), h)
        self.out_elems = n.value
        check(lib.mrdft_input_elems(h, ctypes.byref(n)), h)
        self.in_elems = n.value

    @property
    def handle(self):
        return self._h

    def opts(self) -> dict:
        """The execution options the plan runs with."""
        eo = ExecOpts()
        check(self._lib.mrdft_plan_get_opts(self._h, ctypes.byref(eo)), self._h)
        return eo.to_dict()

    def info(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.mrdft_plan_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), self._h)
        return {"tile_log": a.value, "fwd_launches": b.value, "adj_launches": c.value}

    def forward(self, x_ptr: int, y_ptr: int, stream: int = 0) -> None:
        check(self._lib.mrdft_forward(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                      ctypes.c_void_p(stream)), self._h)

    def adjoint(self, gy_ptr: int, gx_ptr: int, stream: int = 0) -> None:
        check(self._lib.mrdft_adjoint(self._h, ctypes.c_void_p(gy_ptr), ctypes.c_void_p(gx_ptr),
                                      ctypes.c_void_p(stream)), self._h)

    def loss_grad(self, x_ptr: int, t_ptr: int, y_ptr: int, gx_ptr: int, loss_ptr: int, stream: int = 0) -> None:
        """mrdft_loss_grad: Y = MrDFT(x), L = sum_i 2^-i |Y_i - T_i|^2 into the
        device double at loss_ptr (0: not computed), gx = dL/dx*."""
        check(self._lib.mrdft_loss_grad(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr),
                                        ctypes.c_void_p(y_ptr), ctypes.c_void_p(gx_ptr),
                                        ctypes.c_void_p(loss_ptr or None), ctypes.c_void_p(stream)), self._h)

    def forward_host(self, x_host_ptr: int, y_host_ptr: int, stream: int = 0) -> None:
        check(self._lib.mrdft_forward_host(self._h, ctypes.c_void_p(x_host_ptr),
                                           ctypes.c_void_p(y_host_ptr), ctypes.c_void_p(stream)), self._h)

    def timing_enable(self, on: bool = True, serial: bool = False) -> None:
        """Bracket every launch with CUDA events; ``serial`` also runs the
        launches one after another on the caller's stream."""
        mode = (2 if serial else 1) if on else 0
        check(self._lib.mrdft_timing_enable(self._h, mode), self._h)

    def timing_read(self) -> dict:
        """{kind: (ms, launches, algorithmic_bytes)} since timing_enable."""
        out = {}
        for k, name in enumerate(KINDS):
            ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
            check(self._lib.mrdft_timing_read(self._h, k, ctypes.byref(ms), ctypes.byref(n),
                                              ctypes.byref(b)), self._h)
            if n.value:
                out[name] = (ms.value, n.value, b.value)
        return out

    def status_poll(self) -> None:
        check(self._lib.mrdft_status_poll(self._h), self._h)

    def graph_stats(self) -> dict:
        """Executable graphs held, captures made, captures that re-targeted a held graph."""
        c, n, u = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.mrdft_plan_graph_stats(self._h, ctypes.byref(c), ctypes.byref(n), ctypes.byref(u)), self._h)
        return {"cached": c.value, "captures": n.value, "updates": u.value}

    def debug_item(self, lst: int, index: int, new=None):
        """Read (and with ``new`` overwrite) work item ``index`` of list 0 (tiles)
        or 1 (levels) as four int32 words; None past the end of the list."""
        old = (ctypes.c_int32 * 4)()
        nw = (ctypes.c_int32 * 4)(*new) if new is not None else None
        st = self._lib.mrdft_debug_item(self._h, int(lst), int(index), nw, old)
        if st == MRDFT_EINVAL:
            return None
        check(st, self._h)
        return list(old)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.mrdft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
