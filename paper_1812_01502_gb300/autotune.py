"""Autotuner for the launch configuration of a filter or a batch of filters.

For one problem (model kind, state dimension, N, radices) it times a few
candidate configurations - the tile size of the shared-memory tile kernel
(digits that are not power-of-two radices <= 32) and the number of persistent
thread blocks - over whole cycles of the radix schedule, and keeps the
fastest.  Results are cached per device in a JSON file (``BFPF_TUNE_CACHE``,
default ``~/.cache/bfpf/tune.json``), keyed by device name, SM count and the
problem, so later filters of the same shape start with the tuned options.

For a batch (``tune_batch``) it times the tile size and the work of one
thread block (``unit_work``: how finely each filter's step is split over
blocks), keyed by the batch's shape signature (the multiset of model kind,
state dimension, N and radices).

Tuning changes only how the work is split: states and ancestors do not depend
on it, and the likelihood, mean and ESS only through the summation order of
their FP32 partial sums.
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "bfpf", "tune.json")


def cache_path() -> str:
    return os.environ.get("BFPF_TUNE_CACHE", DEFAULT_CACHE)


def problem_key(device_name: str, sm_count: int, kind: str, d: int, N: int, radices: Sequence[int]) -> str:
    return f"{device_name}|{sm_count}|{kind}|d{d}|N{N}|r{'x'.join(str(int(a)) for a in radices)}"


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    data = load_cache(path)
    data[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(sm_count: int, d: int) -> Iterable[Tuple[int, int]]:
    """(tile, grid) pairs: tile 0 / grid 0 mean the library's own choice."""
    tiles = [0, 1024, 2048, 4096] if d <= 2 else [0, 512, 1024, 2048]
    grids = [0, sm_count, 2 * sm_count]
    for t in tiles:
        for g in grids:
            yield t, g


def pick_best(timings: Dict[Tuple[int, int], float]) -> Tuple[Tuple[int, int], float]:
    best = min(timings.items(), key=lambda kv: kv[1])
    return best[0], best[1]


def tune(model, N: int, radices: Sequence[int], *, cycles: int = 2, device=None, use_cache: bool = True,
         timer: Optional[Callable] = None) -> dict:
    """Tuned pf_options {tile, grid} for this problem (cached per device)."""
    import torch
    from . import ButterflyFilter
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    d = 1 if model.kind == "sv" else int(model.A.shape[0])
    key = problem_key(props.name, props.multi_processor_count, model.kind, d, N, radices)
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            return hit
    m = len(radices)
    steps = max(4, cycles * m)
    dy = 1 if model.kind == "sv" else int(model.H.shape[0])
    y = torch.zeros((steps + m, dy), dtype=torch.float32, device=dev)

    def default_timer(tile, grid):
        f = ButterflyFilter(model, N, radices, 12345, tile=tile, grid=grid, device=dev)
        f.push(y[:m])
        f.advance(m)                                  # warm-up: one cycle
        f.push(y[m:m + steps])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(f.stream)
        f.advance(steps)
        e1.record(f.stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        f.close()
        return ms

    run = timer or default_timer
    timings = {}
    for tile, grid in candidates(props.multi_processor_count, d):
        try:
            timings[(tile, grid)] = run(tile, grid)
        except Exception:          # a candidate that does not fit (shared memory) is skipped
            continue
    (tile, grid), ms = pick_best(timings)
    entry = {"tile": tile, "grid": grid, "ms_per_step": ms, "default_ms_per_step": timings.get((0, 0)),
             "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        store(key, entry)
    return entry


def batch_signature(specs) -> str:
    """Shape signature of a batch: sorted (kind, d, N, radices) counts."""
    import hashlib
    shapes = {}
    for model, N, radices, _seed in specs:
        d = 1 if model.kind == "sv" else int(model.A.shape[0])
        k = f"{model.kind}:{d}:{int(N)}:{'x'.join(str(int(a)) for a in radices)}"
        shapes[k] = shapes.get(k, 0) + 1
    text = ";".join(f"{k}*{v}" for k, v in sorted(shapes.items()))
    return hashlib.sha1(text.encode()).hexdigest()[:16]


def batch_candidates() -> Iterable[Tuple[int, int]]:
    """(tile, unit_work) pairs: 0 means the library's own choice."""
    for t in (0, 1024, 2048):
        for u in (0, 8192, 16384, 65536, 131072):
            yield t, u


def tune_batch(specs, *, steps: int = 8, device=None, use_cache: bool = True,
               timer: Optional[Callable] = None) -> dict:
    """Tuned {tile, unit_work} for a batch of filters (cached per device and batch signature)."""
    import torch
    from . import FilterBatch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    key = f"{props.name}|{props.multi_processor_count}|batch|{batch_signature(specs)}"
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            return hit
    dy_max = max(1 if m.kind == "sv" else int(m.H.shape[0]) for m, _, _, _ in specs)
    y = torch.zeros((len(specs), 2 * steps, dy_max), dtype=torch.float32, device=dev)

    def default_timer(tile, unit_work):
        b = FilterBatch(specs, tile=tile, unit_work=unit_work, chunk_len=steps, device=dev)
        b.run(y[:, :steps], outputs=False)            # warm-up: graph capture
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.run(y[:, steps:], outputs=False)
        e1.record(b.stream)
        torch.cuda.synchronize(dev)
        b.close()
        return e0.elapsed_time(e1) / steps

    run = timer or default_timer
    timings = {}
    for tile, uw in batch_candidates():
        try:
            timings[(tile, uw)] = run(tile, uw)
        except Exception:          # a candidate that does not fit (shared memory) is skipped
            continue
    (tile, uw), ms = pick_best(timings)
    entry = {"tile": tile, "unit_work": uw, "ms_per_step": ms, "default_ms_per_step": timings.get((0, 0)),
             "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        store(key, entry)
    return entry
