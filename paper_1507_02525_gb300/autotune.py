"""Autotuner of a plan's execution shape, with a JSON cache.

The transform's result does not depend on how a plan cuts its signals into
segments (at most 2^seg_log samples each, whose level chains run concurrently
on `streams` worker streams; see mrdft_plan_opts in include/mrdft.h), but its
speed does: segments small enough for their levels to stay in L2 but large
enough to fill the GPU.  `tune` times the forward, the adjoint or both (the
objective) of every candidate shape on scratch buffers of the plan's own
size, with CUDA events after warm-up, and keeps the fastest; results are
cached per (device, dtype, batch, length list, objective) in a JSON file so
that a process plans tuned shapes without timing again.

The cache lives at $MRDFT_AUTOTUNE_CACHE, else
~/.cache/paper_1507_02525_gb300/autotune.json.  Cache handling is host-only
(tested on CPU); timing needs a GPU.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (20, 4), (21, 2), (21, 4), (22, 2), (22, 4), (23, 2), (23, 4), (24, 2), (26, 1))
OBJECTIVES = ("both", "forward", "adjoint")

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("MRDFT_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1507_02525_gb300", "autotune.json")


def cache_key(device_name: str, real_input: bool, batch: int, lengths: Sequence[int]) -> str:
    """Key of a plan configuration: the device, the input type, the batch and
    the multiset of signal lengths (a digest of the sorted list)."""
    ls = sorted(int(v) for v in lengths)
    digest = hashlib.sha1(",".join(map(str, ls)).encode()).hexdigest()[:16]
    return f"{device_name}|{'r32' if real_input else 'c64'}|b{int(batch)}|n{len(ls)}|{digest}"


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: Optional[str] = None) -> None:
    """Add one entry to the cache file (read-modify-write, atomic replace)."""
    path = path or cache_path()
    with _lock:
        data = load_cache(path)
        data[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def pick(timings: Dict[Tuple[int, int], float]) -> Tuple[int, int]:
    """Fastest candidate; ties go to the larger segment (fewer launches)."""
    if not timings:
        raise ValueError("no timings")
    return min(timings, key=lambda c: (timings[c], -c[0], c[1]))


def tune(lengths: Sequence[int], batch: Optional[int] = None, real_input: bool = False,
         candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES, adjoint: bool = True,
         reps: int = 5, use_cache: bool = True, timer: Optional[Callable] = None,
         objective: Optional[str] = None) -> Tuple[int, int]:
    """Best (seg_log, streams) for this plan configuration on the current GPU.

    `objective` is what is timed: "both" (forward + adjoint, the default),
    "forward" or "adjoint" (a plan used in one direction only); `adjoint=False`
    is the same as "forward".  `timer(seg_log, streams) -> ms` may replace the
    GPU timing (tests)."""
    objective = objective or ("both" if adjoint else "forward")
    if objective not in OBJECTIVES:
        raise ValueError(f"objective must be one of {OBJECTIVES}")
    lengths = [int(v) for v in lengths]
    batch = len(lengths) if batch is None else int(batch)
    import torch
    dev_name = torch.cuda.get_device_name() if timer is None else "test-device"
    key = cache_key(dev_name, real_input, batch, lengths if len(lengths) == batch else lengths * batch)
    if objective != "both":
        key += f"|{objective}"
    if use_cache:
        hit = load_cache().get(key)
        if hit and "seg_log" in hit and "streams" in hit:
            return int(hit["seg_log"]), int(hit["streams"])
    if timer is None:
        timer = _gpu_timer(lengths, batch, real_input, objective, reps)
    total = sum(lengths) if len(lengths) == batch else sum(lengths) * batch
    cands: List[Tuple[int, int]] = []
    for s, k in candidates:
        s = min(max(int(s), 12), 26)
        if (1 << s) >= total and any((1 << c[0]) >= total for c in cands):
            continue  # once one segment holds every signal, larger segments give the same plan
        if (s, k) not in cands:
            cands.append((s, int(k)))
    timings = {c: float(timer(*c)) for c in cands}
    best = pick(timings)
    if use_cache:
        store(key, {"seg_log": best[0], "streams": best[1],
                    "ms": {f"{s},{k}": round(v, 5) for (s, k), v in timings.items()}})
    return best


def _gpu_timer(lengths, batch, real_input, objective, reps):
    import torch
    from . import _lib

    first = _lib.Plan(lengths, batch, real_input=real_input)
    x = torch.randn(first.in_elems, dtype=torch.float32 if real_input else torch.complex64, device="cuda")
    y = torch.empty(first.out_elems, dtype=torch.complex64, device="cuda")
    gx = torch.empty(first.in_elems, dtype=torch.complex64, device="cuda")
    first.close()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def timer(seg_log: int, streams: int) -> float:
        plan = _lib.Plan(lengths, batch, real_input=real_input, graph=True, seg_log=seg_log, streams=streams)
        try:
            def step():
                if objective != "adjoint":
                    plan.forward(x.data_ptr(), y.data_ptr(), sp)
                if objective != "forward":
                    plan.adjoint(y.data_ptr(), gx.data_ptr(), sp)
            plan.forward(x.data_ptr(), y.data_ptr(), sp)  # the adjoint's input: a real spectrum
            for _ in range(2):
                step()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            plan.status_poll()
            return e0.elapsed_time(e1) / reps
        finally:
            plan.close()

    return timer
