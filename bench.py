#!/usr/bin/env python
"""Throughput of the butterfly-interaction bootstrap particle filter on GB300.

One bench step = one filter time step (weight, one butterfly resampling stage,
mutate: the whole hot path) over all N particles of the workload, run through
the library's C ABI (``paper_1812_01502_gb300``).  Default workload: the stochastic-volatility
model with N = 2^24 particles, radix 16 (m = 6 digits).

Timing (device, CUDA events on the filter's stream): observations are pushed
to the device before the timed region; before every timed step a 512 MB
buffer is written to flush the 129 MB L2, so each step streams its particles
from HBM; only the step kernel sits between the events.  ``value`` =
particle-steps/s over all ranks (max time over ranks).  ``e2e`` runs the same
steps through the public ``run`` call with host observations in and host
per-step outputs (mean, log-likelihood increment, ESS) out.

``--impl reference`` times the FP64 CPU oracle (the reference of this build)
on a bounded sample of the same workload.

Multi-GPU: independent filter replicas, one per rank (weak scaling; the
method needs no exchange between replicas).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
FLUSH_BYTES = 512 << 20


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="sv_n16m")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-rate", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--oracle-n", type=int, default=0, help=argparse.SUPPRESS)
    p.add_argument("--oracle-seconds", type=float, default=12.0, help=argparse.SUPPRESS)
    p.add_argument("--oracle-steps", type=int, default=0, help=argparse.SUPPRESS)
    return p.parse_args()


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def algorithmic_bytes(w, n: int) -> int:
    """Bytes one time step n must move: read + write the states (4 d N each),
    read the carried weights (one per group of the previous digit) and write
    the new ones (one per group of digit k)."""
    m = len(w.radices)
    a = w.radices[n % m]
    ap = w.radices[(n - 1) % m]
    return 8 * w.model.d * w.N + 4 * (w.N // ap) + 4 * (w.N // a)


KERNEL_SOURCES = ("bfpf_device.cuh", "bfpf_epilogue.cuh", "bfpf_model.cuh", "step_group.cuh",
                  "step_butterfly.cu")


def _kernel_source_hash() -> str:
    """Hash of the step kernels' sources: a committed ncu figure is used only while it matches."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1812_01502_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"step_group_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    mb = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not mh or not mb or mh.group(1) != _kernel_source_hash():
        return None
    return float(mb.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference of this build)
# ---------------------------------------------------------------------------
def oracle_rate_main(a):
    """Run in a fresh single-threaded process: FP64 oracle particle-steps/s."""
    try:   # one core: the timed baseline is the oracle as it stands, single-threaded
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    import numpy as np
    import synthetic as S
    from oracle import bpf
    w = S.workload(a.workload)
    N = a.oracle_n or w.N
    radices = list(w.radices)
    while int(np.prod(radices)) > N:        # shrink the top digits for a smaller sample
        radices[-1] //= 2
        if radices[-1] == 1:
            radices.pop()
    N = int(np.prod(radices))
    y = w.observations(max(8, a.oracle_steps or 8))
    st = bpf.init_state(w.model, N, w.filter_seed)
    t0 = time.perf_counter()
    steps = 0
    while True:
        st, _ = bpf.step(w.model, radices, w.filter_seed, st, y[steps])
        steps += 1
        el = time.perf_counter() - t0
        if a.oracle_steps and steps >= a.oracle_steps:
            break
        if not a.oracle_steps and (el >= a.oracle_seconds or steps >= len(y)):
            break
    print(json.dumps({"value": N * steps / el, "N": N, "radices": radices, "steps": steps, "seconds": el}))


def oracle_rate(workload: str, n: int = 0, seconds: float = 12.0, steps: int = 0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-rate", "--workload", workload,
           "--oracle-n", str(n), "--oracle-seconds", str(seconds), "--oracle-steps", str(steps)]
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1200)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_main(a):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import synthetic as S
    w = S.workload(a.workload)
    n_sample = 1 << 20 if w.N > (1 << 20) else w.N
    # warm-up steps are included in the sample run's start-up; time K steps
    r = oracle_rate(a.workload, n=n_sample, steps=max(1, a.steps))
    sample = (f"first {r['steps']} time steps of {a.workload} with N={r['N']} particles "
              f"(radices {r['radices']}) on the FP64 numpy oracle, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": METRIC,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1000.0 * r["seconds"] / r["steps"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload, "N": r["N"], "radices": r["radices"]},
            "cpu_baseline": {"value": r["value"], "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": r["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def ours_main(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    import synthetic as S
    import paper_1812_01502_gb300 as bf

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = S.workload(a.workload)
    K, W = a.steps, a.warmup
    T_need = W + K + min(K, 1000) + 8
    y = S.simulate(w.model, max(w.T, T_need), w.data_seed)[1].astype(np.float32)
    filt = bf.ButterflyFilter(w.model, w.N, w.radices, w.filter_seed + rank, device=dev)
    stream = filt.stream
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # --- device-timed steps, L2 flushed before each -------------------------
    # Observations are pushed (device to device) in chunks of <= 1000 between
    # timed steps; only the step kernel sits between each pair of events.
    y_dev = torch.tensor(y[:W + K], device=dev).contiguous()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(local)
    with torch.cuda.stream(stream):
        filt.push(y_dev[:W])
        for _ in range(W):
            flush.zero_()
            filt.advance(1)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks.start()
        time.sleep(0.3)                  # let the sampler attach before the timed region
        n0 = filt.steps
        for j in range(K):
            if j % 1000 == 0:
                filt.push(y_dev[W + j:W + min(K, j + 1000)])
            flush.zero_()
            starts[j].record(stream)
            filt.advance(1)
            ends[j].record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
    # --- L2-resident chunk (consecutive steps, CUDA graph), for reference ----
    KR = min(K, 1000)
    y_dev2 = torch.tensor(y[W + K:W + K + KR], device=dev).contiguous()
    with torch.cuda.stream(stream):
        filt.push(y_dev2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        filt.advance(KR)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    resident_ms = e0.elapsed_time(e1) * K / KR

    # --- end to end through the public call, host buffers -------------------
    y_host = np.ascontiguousarray(y[:K])
    efilt = bf.ButterflyFilter(w.model, w.N, w.radices, w.filter_seed + rank, device=dev)
    efilt.run(y_host[:min(W, K)])          # warm-up (graph capture, first touch)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    out = efilt.run(y_host)                # H2D observations, D2H per-step outputs; synchronises
    e2e_s = time.perf_counter() - t0
    ll_e2e = float(np.sum(out["inc"]))
    efilt.close()

    if world > 1:
        t = torch.tensor([total_ms, e2e_s, resident_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, e2e_s, resident_ms = (float(v) for v in t.tolist())
    value = world * w.N * K / (total_ms * 1e-3)
    e2e_value = world * w.N * K / e2e_s
    if rank != 0:
        if world > 1:
            dist.barrier()
        return

    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    traffic = _profiled_traffic(a.workload)
    cpu = None
    if not a.no_cpu_baseline:
        try:
            r = oracle_rate(a.workload, seconds=12.0)
            cpu = {"value": r["value"], "unit": METRIC, "cores": 1, "kind": "oracle",
                   "sample": f"first {r['steps']} time steps of {a.workload} at full size "
                             f"(N={r['N']}) on the FP64 numpy oracle, 1 thread"}
        except Exception as ex:  # report, never hide
            cpu = {"value": None, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": a.workload, "N": w.N, "radices": list(w.radices), "d": w.model.d,
                   "model": w.model.kind, "l2": "flushed before every timed step (512 MB write)",
                   "parallelism": f"replicas{world}",
                   "resident_particle_steps_per_s": world * w.N * K / (resident_ms * 1e-3),
                   "resident_ms_per_step": resident_ms / K},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak, "unit": "GB/s",
                     "frac": achieved_gbs / peak, "traffic": traffic,
                     "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                     "algorithmic_bytes_per_launch": sum(bytes_steps) / K},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": 4 * w.model.dy,
                "d2h_bytes_per_step": 4 * w.model.d + 8 + 4, "loglik": ll_e2e},
        "gpu_launches": K,
        "clocks": clk,
    }
    print(json.dumps(line))
    filt.close()
    if world > 1:
        dist.barrier()


def main():
    a = _args()
    if a.oracle_rate:
        return oracle_rate_main(a)
    if a.impl == "reference":
        return reference_main(a)
    return ours_main(a)


if __name__ == "__main__":
    main()
