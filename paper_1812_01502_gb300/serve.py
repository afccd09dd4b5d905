"""Serving loop: filtering requests admitted by device memory, continuously batched.

A request is one filtering job - a model, N, radices, seed and an observation
series that arrives in chunks (50 observations by default), chunk c at
arrival + (c + 1) * chunk_interval (all at once when the interval is 0).  The
server keeps at most ``slots`` requests on the GPU, each with its own filter
handle, workspace and CUDA stream; particle state stays resident on the device
between chunks.  Requests that arrive while others run are admitted as soon as
a slot and enough device memory are free: the handle's workspace size checked
against ``memory_budget`` when one is given, else against the device's free
memory (cudaMemGetInfo, plus what the PyTorch allocator holds unused) less
``reserve``.  Every scheduling pass copies each arrived chunk from pinned host
memory and enqueues its steps, so the chunks of different requests overlap on
the device; completions are detected with CUDA events.

Latency of a request = completion of its last chunk - its arrival; latency
of a chunk = its completion - the later of its arrival and its admission.  A request
whose filter reports non-finite weights (a NaN observation, say) is finished
with ``error`` set; the other requests are not affected.  The
server reports p50 / p99 request latency, chunk latency and throughput in
particle-steps/s.  The filtering itself runs in the library's kernels; this
module only schedules.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import ButterflyFilter, PFOptions, _check, load_library, make_model


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the server's start
    model: object
    N: int
    radices: Sequence[int]
    seed: int
    y: np.ndarray                  # (T, dy) observations
    chunk: int = 50
    chunk_interval: float = 0.0    # seconds between the arrivals of consecutive chunks
    # filled in by the server
    admitted: Optional[float] = None
    finished: Optional[float] = None
    chunk_latencies: List[float] = field(default_factory=list)
    means: Optional[np.ndarray] = None
    incs: Optional[np.ndarray] = None
    loglik: Optional[float] = None
    status: int = 0                # sticky device status bits of the request's filter
    error: Optional[str] = None    # set when the filter reported a failure (others keep running)


def workspace_bytes(model, N: int, radices: Sequence[int]) -> int:
    """Device bytes one request needs (pf_workspace_size)."""
    lib = load_library()
    pm, keep = make_model(model)
    rad = (ctypes.c_int32 * len(radices))(*radices)
    nbytes = ctypes.c_size_t(0)
    opts = PFOptions(tile=0, chunk_len=0, flags=0, grid=0, stream=None)
    _check(lib.pf_workspace_size(ctypes.byref(pm), int(N), rad, len(radices), ctypes.byref(opts),
                                 ctypes.byref(nbytes)))
    return int(nbytes.value)


class _Active:
    def __init__(self, req: Request, filt: ButterflyFilter, stream, nbytes: int, device):
        import torch
        self.req = req
        self.filt = filt
        self.stream = stream
        self.nbytes = nbytes
        T = len(req.y)
        self.T = T
        # observations wait in pinned host memory; each chunk is copied when it arrives
        self.y_host = torch.tensor(np.asarray(req.y, dtype=np.float32).reshape(T, -1)).pin_memory()
        self.means = torch.empty((T, filt.d), dtype=torch.float32, device=device)
        self.incs = torch.empty(T, dtype=torch.float64, device=device)
        self.next = 0                      # first observation not yet enqueued
        self.inflight = collections.deque()  # (event, t_enqueue, end)


class Server:
    """Continuous-batching server on one GPU."""

    def __init__(self, memory_budget: Optional[int] = None, slots: int = 16, device=None, chunk_len: int = 50,
                 reserve: int = 2 << 30):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.memory_budget = None if memory_budget is None else int(memory_budget)
        self.reserve = int(reserve)
        self.slots = int(slots)
        self.chunk_len = int(chunk_len)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.slots)]
        self.free_streams = list(range(self.slots))
        self.in_use = 0
        self.active: Dict[int, _Active] = {}
        self.done: List[Request] = []

    def available(self) -> int:
        """Device bytes a new request may take now."""
        if self.memory_budget is not None:
            return self.memory_budget - self.in_use
        torch = self.torch
        free, _total = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return free + cached - self.reserve

    def _admit(self, req: Request, now: float) -> bool:
        need = workspace_bytes(req.model, req.N, req.radices)
        if not self.free_streams or need > self.available():
            return False
        si = self.free_streams.pop()
        stream = self.streams[si]
        with self.torch.cuda.stream(stream):
            filt = ButterflyFilter(req.model, req.N, req.radices, req.seed, chunk_len=self.chunk_len,
                                   device=self.device, stream=stream)
        act = _Active(req, filt, stream, need, self.device)
        act.slot = si
        self.in_use += need
        req.admitted = now
        self.active[req.rid] = act
        return True

    def _enqueue(self, act: _Active, now: float):
        torch = self.torch
        if act.next >= act.T or len(act.inflight) >= 2:
            return
        s = act.next
        e = min(act.T, s + act.req.chunk)
        ready = act.req.arrival + (s // act.req.chunk + 1) * act.req.chunk_interval
        if now < ready:                     # this chunk's observations have not arrived yet
            return
        lib = load_library()
        h = act.filt._h
        with torch.cuda.stream(act.stream):
            _check(lib.pf_push_observations(h, ctypes.c_void_p(act.y_host[s:e].data_ptr()), e - s), h)
            _check(lib.pf_advance(h, e - s, ctypes.c_void_p(act.means[s:e].data_ptr()),
                                  ctypes.c_void_p(act.incs[s:e].data_ptr()), None), h)
            ev = torch.cuda.Event()
            ev.record(act.stream)
        act.filt.steps += e - s
        act.inflight.append((ev, max(ready, act.req.admitted), e))
        act.next = e

    def _retire(self, act: _Active, now: float) -> bool:
        while act.inflight and act.inflight[0][0].query():
            ev, t0, end = act.inflight.popleft()
            act.req.chunk_latencies.append(now - t0)
            if end == act.T:
                req = act.req
                req.finished = now
                req.means = act.means.cpu().numpy()
                req.incs = act.incs.cpu().numpy()
                req.status = act.filt.status()
                try:
                    req.loglik = act.filt.loglik()
                except Exception as ex:      # a failure of this request only
                    req.loglik = None
                    req.error = str(ex)
                if req.status & 1 and req.error is None:
                    req.error = "non-finite log-weights (e.g. a NaN observation)"
                act.filt.close()
                self.in_use -= act.nbytes
                self.free_streams.append(act.slot)
                del self.active[req.rid]
                self.done.append(req)
                return True
        return False

    def run(self, requests: Sequence[Request], poll_sleep: float = 0.0002, timeout_s: float = 600.0):
        """Serve requests (sorted by arrival) in real time; returns the finished requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        t_start = time.perf_counter()
        while pending or waiting or self.active:
            now = time.perf_counter() - t_start
            if now > timeout_s:
                raise TimeoutError("serving did not finish in time")
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting and self._admit(waiting[0], now):
                waiting.popleft()
            if waiting and not self.active:
                req = waiting[0]
                if workspace_bytes(req.model, req.N, req.radices) > self.available():
                    raise MemoryError(f"request {req.rid} needs more than the whole memory budget")
            self.max_active = max(getattr(self, "max_active", 0), len(self.active))
            self.max_in_use = max(getattr(self, "max_in_use", 0), self.in_use)
            for act in list(self.active.values()):
                self._enqueue(act, now)
            now = time.perf_counter() - t_start
            for act in list(self.active.values()):
                self._retire(act, now)
            if poll_sleep:
                time.sleep(poll_sleep)
        self.wall = time.perf_counter() - t_start
        return self.done


def summarize(done: Sequence[Request], wall: float) -> dict:
    failed = sum(1 for r in done if r.error)
    lat = np.array([r.finished - r.arrival for r in done])
    clat = np.array([c for r in done for c in r.chunk_latencies])
    # the server's own delay: completion after the last chunk's arrival
    extra = np.array([r.finished - (r.arrival + -(-len(r.y) // r.chunk) * r.chunk_interval) for r in done])
    ps = sum(r.N * len(r.y) for r in done)
    return {"requests": len(done), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "p50_chunk_latency_s": float(np.percentile(clat, 50)),
            "p99_chunk_latency_s": float(np.percentile(clat, 99)),
            "p50_after_last_chunk_s": float(np.percentile(extra, 50)),
            "p99_after_last_chunk_s": float(np.percentile(extra, 99)), "wall_s": wall,
            "particle_steps_per_s": ps / wall, "failed_requests": failed}


def requests_from_stream(stream, chunk: int = 50, chunk_interval: float = 0.0) -> List[Request]:
    """Requests from (arrival, workload) pairs (synthetic.serving_stream)."""
    out = []
    for rid, (t, w) in enumerate(stream):
        out.append(Request(rid=rid, arrival=float(t), model=w.model, N=w.N, radices=w.radices, seed=w.filter_seed,
                           y=w.observations(), chunk=chunk, chunk_interval=chunk_interval))
    return out
