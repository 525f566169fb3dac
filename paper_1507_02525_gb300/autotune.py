"""Autotuner of a plan's execution options, with a JSON cache.

The transform's result does not depend on how a plan cuts its signals into
segments (at most 2^seg_log samples each, whose level chains run concurrently
on `streams` worker streams), nor on the kernel variants it launches (the
two-pass split C of the large levels, the rows CTA shape, the pairing of two
levels in one cols pass, the tree schedule of the levels above a segment; see
mrdft_exec_opts in include/mrdft.h), but its speed does.  `tune_plan` times
the forward, the adjoint or both (the objective) on scratch buffers of the
plan's own size, with CUDA events after warm-up: first every candidate shape
with the default kernel variants, then each kernel variant in turn on the
best shape (coordinate descent: a variant is kept only when it is faster by
more than 1%), and returns the options of the fastest plan.  Results are
cached per (device, dtype, batch, length list, objective) in a JSON file so
that a process plans tuned options without timing again.  `tune` is the
shape-only search.

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

# kernel variants searched after the shape, per objective: (option, values);
# the first value of each is the library default
FWD_KNOBS = (("fwd_cb", (9, 10, 11)), ("fwd_rows_prefetch", (False, True)), ("fwd_rows12", (False, True)),
             ("dual_cols", (True, False)), ("fwd_tree", (False, True)))
ADJ_KNOBS = (("adj_cb", (10, 9)), ("adj_rows13", (True, False)), ("dual_cols", (True, False)))
# searched together with the shape (they change how the segments overlap):
# whether the in-tile levels run as one launch, and then into how many groups
SHAPE_SWITCHES = ("tile_first", (True, False))
TILE_SPLITS = (1,)  # more groups measured slower: a tile launch beside the segment chains evicts their L2 data
KEEP_MARGIN = 0.99  # a variant replaces the current choice only when at least 1% faster


def knobs_for(objective: str, lengths: Sequence[int], seg_log: int):
    """The kernel variants that can change this workload's plan: the two-pass
    ones only when some signal has two-pass levels (N > 2^14), the tree only
    when some signal is longer than a segment."""
    mx = max(int(v) for v in lengths)
    if mx <= (1 << 14):
        return ()
    knobs = {"forward": FWD_KNOBS, "adjoint": ADJ_KNOBS}.get(objective)
    if knobs is None:  # both: the union, in order
        knobs = FWD_KNOBS + tuple(k for k in ADJ_KNOBS if k[0] not in dict(FWD_KNOBS))
    return tuple(k for k in knobs if k[0] != "fwd_tree" or mx > (1 << seg_log))

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


def tune_plan(lengths: Sequence[int], batch: Optional[int] = None, real_input: bool = False,
              objective: str = "both", candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES,
              reps: int = 5, use_cache: bool = True, timer: Optional[Callable] = None) -> dict:
    """Execution options (a dict for ``_lib.Plan(opts=...)``) of the fastest plan
    found for this configuration on the current GPU.  `timer(opts) -> ms` may
    replace the GPU timing (tests)."""
    if objective not in OBJECTIVES:
        raise ValueError(f"objective must be one of {OBJECTIVES}")
    lengths = [int(v) for v in lengths]
    batch = len(lengths) if batch is None else int(batch)
    full = lengths if len(lengths) == batch else lengths * batch
    import torch
    dev_name = torch.cuda.get_device_name() if timer is None else "test-device"
    key = cache_key(dev_name, real_input, batch, full) + f"|{objective}|opts"
    if use_cache:
        hit = load_cache().get(key)
        if hit and isinstance(hit.get("opts"), dict):
            return dict(hit["opts"])
    if timer is None:
        gpu = _gpu_timer(lengths, batch, real_input, objective, reps)
        timer = lambda o: gpu(o.get("seg_log"), o.get("streams"), o)  # noqa: E731
    log = {}

    def t(o):
        k = json.dumps(o, sort_keys=True)
        if k not in log:
            log[k] = float(timer(dict(o)))
        return log[k]

    best, best_ms = None, float("inf")
    name0, values0 = SHAPE_SWITCHES
    for v0 in values0:
        shape = tune(lengths, batch, real_input, candidates=candidates, use_cache=False, objective=objective,
                     timer=lambda s_, k_: t({"seg_log": s_, "streams": k_, name0: v0}))
        trial = {"seg_log": shape[0], "streams": shape[1], name0: v0}
        ms = t(trial)
        if best is None or ms < KEEP_MARGIN * best_ms:
            best, best_ms = trial, ms
    if best.get("tile_first") and sum(full) > (1 << best["seg_log"]):  # several segments: split the tiles
        for k in TILE_SPLITS[1:]:
            trial = dict(best, tile_split=k)
            ms = t(trial)
            if ms < KEEP_MARGIN * best_ms:
                best, best_ms = trial, ms
    for name, values in knobs_for(objective, full, best["seg_log"]):
        for v in values[1:]:
            trial = dict(best, **{name: v})
            ms = t(trial)
            if ms < KEEP_MARGIN * best_ms:
                best, best_ms = trial, ms
    if use_cache:
        store(key, {"opts": best, "ms": round(best_ms, 5), "timed": {k: round(v, 5) for k, v in log.items()}})
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

    def timer(seg_log: int, streams: int, opts: Optional[dict] = None) -> float:
        plan = _lib.Plan(lengths, batch, real_input=real_input, graph=True, seg_log=seg_log, streams=streams,
                         opts={k: v for k, v in (opts or {}).items() if k not in ("seg_log", "streams")})
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
