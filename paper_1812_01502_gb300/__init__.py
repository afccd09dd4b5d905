"""Butterfly-interaction bootstrap particle filter on GB300 (sm_103a).

Python binding of the C ABI in ``include/bfpf.h`` (library ``libbfpf.so``,
built in-tree by ``paper_1812_01502_gb300._build``).  This module only marshals
arguments: every step of the filter runs in the CUDA kernels of the library.
PyTorch supplies device memory (the filter's workspace) and the CUDA stream.

There is no CPU fallback: importing works without a GPU (so the ABI can be
inspected), but creating a filter needs the compiled library and a CUDA
device, and fails loudly otherwise.

The method: Heine, Whiteley & Cemgil, "Parallelising particle filters with
butterfly interactions" (arXiv 1812.01502) - Algorithm 1 whose resampling is
one stage of Algorithm 3 per time step on digit k = n mod m of the mixed-radix
particle index (N = a_0 ... a_{m-1}).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfpf.so")

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ETIMEOUT, PF_ESTATE = range(6)
PF_MODEL_LINEAR_GAUSSIAN = 1
PF_MODEL_STOCH_VOL = 2
PF_RECORD_ANCESTORS = 1
PF_ALL_STAGES = 2
PF_ADAPTIVE = 4
PF_ROTATE = 8
PF_ISLANDS = 16
PF_ISLANDS_PLAIN = 32
PF_TEST_SMALL_BUCKETS = 0x40000000
PF_TEST_STAGE_PER_LAUNCH = 0x20000000
PF_DIGIT_SETS = 64
PF_RECORD_DRAWS = 128
STATUS_NAMES = {PF_EINVAL: "PF_EINVAL", PF_ENOMEM: "PF_ENOMEM", PF_ECUDA: "PF_ECUDA",
                PF_ETIMEOUT: "PF_ETIMEOUT", PF_ESTATE: "PF_ESTATE"}

_dp = ctypes.POINTER(ctypes.c_double)


class PFModel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("dy", ctypes.c_int32),
                ("A", _dp), ("Lq", _dp), ("H", _dp), ("Lr", _dp), ("m0", _dp), ("L0", _dp),
                ("phi", ctypes.c_double), ("sigma", ctypes.c_double), ("beta", ctypes.c_double)]


class PFOptions(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("chunk_len", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("grid", ctypes.c_int32), ("stream", ctypes.c_void_p), ("ess_threshold", ctypes.c_float)]


class PFError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbfpf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    c = ctypes
    vp, i32, i64, u32, u64 = c.c_void_p, c.c_int32, c.c_int64, c.c_uint32, c.c_uint64
    sig = {
        "pf_workspace_size": (i32, [c.POINTER(PFModel), i64, c.POINTER(i32), i32, c.POINTER(PFOptions),
                                    c.POINTER(c.c_size_t)]),
        "pf_create": (i32, [c.POINTER(PFModel), i64, c.POINTER(i32), i32, u64, c.POINTER(PFOptions), vp,
                            c.c_size_t, c.POINTER(vp)]),
        "pf_step": (i32, [vp, vp, vp, vp, vp]),
        "pf_run": (i32, [vp, vp, i32, vp, vp, vp]),
        "pf_push_observations": (i32, [vp, vp, i32]),
        "pf_advance": (i32, [vp, i32, vp, vp, vp]),
        "pf_loglik": (i32, [vp, c.POINTER(c.c_double)]),
        "pf_get_state": (i32, [vp, vp, vp, vp]),
        "pf_get_ancestors": (i32, [vp, vp]),
        "pf_get_status": (i32, [vp, c.POINTER(u32)]),
        "pf_get_draw_prefix": (i32, [vp, vp]),
        "pf_stage_count": (i32, [vp, c.POINTER(c.c_uint64)]),
        "pf_checkpoint_size": (i32, [vp, c.POINTER(c.c_size_t)]),
        "pf_save": (i32, [vp, vp, c.c_size_t]),
        "pf_load": (i32, [vp, vp, c.c_size_t]),
        "pf_destroy": (i32, [vp]),
        "pf_describe": (i32, [vp, c.c_char_p, c.c_size_t]),
        "pf_last_error": (c.c_char_p, [vp]),
        "pf_philox_blocks": (i32, [u64, u32, u32, u32, u32, i64, vp, vp]),
        "pf_batch_workspace_size": (i32, [i32, c.POINTER(PFModel), c.POINTER(i64), c.POINTER(i32), c.POINTER(i32),
                                          c.POINTER(PFOptions), c.POINTER(c.c_size_t)]),
        "pf_batch_create": (i32, [i32, c.POINTER(PFModel), c.POINTER(i64), c.POINTER(i32), c.POINTER(i32),
                                  c.POINTER(u64), c.POINTER(PFOptions), vp, c.c_size_t, c.POINTER(vp)]),
        "pf_batch_run": (i32, [vp, vp, i32, vp, vp, vp]),
        "pf_batch_loglik": (i32, [vp, vp]),
        "pf_batch_get_state": (i32, [vp, i32, vp, vp, vp]),
        "pf_batch_destroy": (i32, [vp]),
        "pf_batch_last_error": (c.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, handle=None):
    if status != PF_OK:
        msg = _lib.pf_last_error(handle).decode(errors="replace")
        raise PFError(status, msg)


def _dbl(arr):
    if arr is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
    return a, a.ctypes.data_as(_dp)


def make_model(model):
    """pf_model from a model description with the attributes of ``synthetic``'s
    LinearGaussian (kind 'lg': A, Lq, H, Lr, m0, L0) or StochVol (kind 'sv': phi, sigma, beta)."""
    keep = []
    m = PFModel()
    if model.kind == "sv":
        m.kind, m.d, m.dy = PF_MODEL_STOCH_VOL, 1, 1
        m.phi, m.sigma, m.beta = float(model.phi), float(model.sigma), float(model.beta)
        return m, keep
    m.kind = PF_MODEL_LINEAR_GAUSSIAN
    m.d = int(np.asarray(model.A).shape[0])
    m.dy = int(np.asarray(model.H).shape[0])
    for name in ("A", "Lq", "H", "Lr", "m0", "L0"):
        arr, ptr = _dbl(getattr(model, name))
        keep.append(arr)
        setattr(m, name, ptr)
    return m, keep


def _torch():
    import torch
    return torch


def _cuda_ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class ButterflyFilter:
    """A filter handle: N = prod(radices) particles, digit k = n mod m interacts at step n.

    all_stages=True runs every stage of Algorithm 3 in each step instead
    (digits 0..m-1 in turn; consecutive digits of one radix share a launch
    where their particles fit one shared-memory tile, else m launches per
    step; describe() lists them).  adaptive=True is fully
    adapted augmented resampling: stages run while the ESS is below
    ``ess_threshold`` (optionally from a rotated start, ``rotate``).
    islands="modified" (or "plain") is AIRPF with radices (M, m): m islands of
    M particles, island resampling by Algorithm 7 (or 6).  digit_sets=True runs
    Algorithm 3 with the paper's stage matrices: stage s on digits {0, s}.
    radices = (N,) is the global-resampling bootstrap filter (Algorithm 1 + 2).
    The workspace is a torch uint8 tensor on ``device``; work runs on the
    current torch stream of that device unless ``stream`` is given.
    """

    def __init__(self, model, N: int, radices: Sequence[int], seed: int, *, tile: int = 0,
                 chunk_len: int = 0, record_ancestors: bool = False, grid: int = 0,
                 device=None, stream=None, tune: bool = False, all_stages: bool = False,
                 adaptive: bool = False, ess_threshold: float = 0.5, rotate: bool = False,
                 islands: Optional[str] = None, digit_sets: bool = False, extra_flags: int = 0):
        torch = _torch()
        lib = load_library()
        if not torch.cuda.is_available():
            raise PFError(PF_ECUDA, "no CUDA device: the butterfly filter runs only on the GPU")
        if tune:    # launch configuration from the autotuner (cached per device and problem)
            from . import autotune
            best = autotune.tune(model, int(N), tuple(radices), device=device)
            tile, grid = int(best["tile"]), int(best["grid"])
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.model = model
        self.N = int(N)
        self.radices = tuple(int(a) for a in radices)
        self.m = len(self.radices)
        self.seed = int(seed)
        self._pm, self._keep = make_model(model)
        self.d, self.dy = self._pm.d, self._pm.dy
        self._rad = (ctypes.c_int32 * self.m)(*self.radices)
        self._opts = PFOptions(tile=int(tile), chunk_len=int(chunk_len),
                               flags=(PF_RECORD_ANCESTORS if record_ancestors else 0)
                               | (PF_ALL_STAGES if all_stages else 0) | (PF_ADAPTIVE if adaptive else 0)
                               | (PF_ROTATE if rotate else 0)
                               | (PF_ISLANDS if islands else 0) | (PF_ISLANDS_PLAIN if islands == "plain" else 0)
                               | (PF_DIGIT_SETS if digit_sets else 0) | int(extra_flags),
                               grid=int(grid),
                               stream=ctypes.c_void_p(self.stream.cuda_stream),
                               ess_threshold=float(ess_threshold) if adaptive else 0.0)
        self.record_ancestors = record_ancestors
        self.all_stages = bool(all_stages)
        self.adaptive = bool(adaptive)
        self.islands = islands
        self.digit_sets = bool(digit_sets)
        with torch.cuda.device(self.device):
            nbytes = ctypes.c_size_t(0)
            _check(lib.pf_workspace_size(ctypes.byref(self._pm), self.N, self._rad, self.m,
                                         ctypes.byref(self._opts), ctypes.byref(nbytes)))
            self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            _check(lib.pf_create(ctypes.byref(self._pm), self.N, self._rad, self.m, ctypes.c_uint64(self.seed),
                                 ctypes.byref(self._opts), _cuda_ptr(self.workspace),
                                 int(nbytes.value), ctypes.byref(h)))
        self._h = h
        self.steps = 0

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.pf_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- filtering -------------------------------------------------------
    def step(self, y_n):
        """One time step; returns (mean (d,), loglik increment, ess) as host values."""
        y = np.ascontiguousarray(np.asarray(y_n, dtype=np.float32).reshape(self.dy))
        mean = np.empty(self.d, dtype=np.float32)
        inc = ctypes.c_double(0.0)
        ess = ctypes.c_float(0.0)
        _check(_lib.pf_step(self._h, y.ctypes.data_as(ctypes.c_void_p), mean.ctypes.data_as(ctypes.c_void_p),
                            ctypes.cast(ctypes.byref(inc), ctypes.c_void_p),
                            ctypes.cast(ctypes.byref(ess), ctypes.c_void_p)), self._h)
        self.steps += 1
        return mean, inc.value, ess.value

    def run(self, y, outputs: bool = True):
        """Filter the observations y (T x dy; numpy array or torch tensor, host or device).

        With outputs=True returns dict(mean (T,d) float32, inc (T,) float64, ess (T,) float32)
        as numpy arrays (for host inputs) or torch tensors on the input's device.
        """
        torch = _torch()
        if isinstance(y, torch.Tensor):
            yt = y.to(dtype=torch.float32).contiguous().reshape(-1, self.dy)
            T = yt.shape[0]
            ptr = ctypes.c_void_p(yt.data_ptr())
            on_dev = yt.is_cuda
            keep = yt
        else:
            ya = np.ascontiguousarray(np.asarray(y, dtype=np.float32).reshape(-1, self.dy))
            T = ya.shape[0]
            ptr = ya.ctypes.data_as(ctypes.c_void_p)
            on_dev = False
            keep = ya
        res = None
        mp = ip = ep = None
        if outputs:
            if on_dev:
                res = dict(mean=torch.empty((T, self.d), dtype=torch.float32, device=self.device),
                           inc=torch.empty(T, dtype=torch.float64, device=self.device),
                           ess=torch.empty(T, dtype=torch.float32, device=self.device))
                mp, ip, ep = (ctypes.c_void_p(res[k].data_ptr()) for k in ("mean", "inc", "ess"))
            else:
                res = dict(mean=np.empty((T, self.d), dtype=np.float32), inc=np.empty(T, dtype=np.float64),
                           ess=np.empty(T, dtype=np.float32))
                mp, ip, ep = (res[k].ctypes.data_as(ctypes.c_void_p) for k in ("mean", "inc", "ess"))
        _check(_lib.pf_run(self._h, ptr, int(T), mp, ip, ep), self._h)
        del keep
        self.steps += T
        return res

    def push(self, y_dev):
        """Copy observations (a contiguous float32 torch tensor or numpy array, T x dy)
        into the device ring for the next steps (pf_push_observations)."""
        torch = _torch()
        if isinstance(y_dev, torch.Tensor):
            assert y_dev.dtype == torch.float32 and y_dev.is_contiguous()
            ptr, T = ctypes.c_void_p(y_dev.data_ptr()), y_dev.numel() // self.dy
        else:
            a = np.ascontiguousarray(np.asarray(y_dev, dtype=np.float32))
            ptr, T = a.ctypes.data_as(ctypes.c_void_p), a.size // self.dy
        _check(_lib.pf_push_observations(self._h, ptr, int(T)), self._h)

    def advance(self, T: int = 1):
        """Take T steps on pushed observations without reading outputs (pf_advance)."""
        _check(_lib.pf_advance(self._h, int(T), None, None, None), self._h)
        self.steps += T

    def loglik(self) -> float:
        out = ctypes.c_double(0.0)
        _check(_lib.pf_loglik(self._h, ctypes.byref(out)), self._h)
        return out.value

    def state(self):
        """(x (N, d) float32, lV (N / a_prev,) float32, dict(n, loglik, mu, mu_used))."""
        t = self.steps * (self.m if (self.all_stages or self.islands) else 1)    # stage counter
        kp = (t - 1) % self.m
        if self.adaptive and self.islands:      # AIRPF2: one weight per island
            nlv = self.N // self.radices[0]
        elif self.adaptive:
            nlv = self.N
        elif self.digit_sets:                   # groups of the last set {0, m-1}
            nlv = self.N // (self.radices[0] * self.radices[-1])
        else:
            nlv = self.N // self.radices[kp]
        x = np.empty((self.d, self.N), dtype=np.float32)
        lv = np.empty(nlv, dtype=np.float32)
        sc = np.empty(4, dtype=np.float64)
        _check(_lib.pf_get_state(self._h, x.ctypes.data_as(ctypes.c_void_p), lv.ctypes.data_as(ctypes.c_void_p),
                                 sc.ctypes.data_as(ctypes.c_void_p)), self._h)
        return x.T.copy(), lv, dict(n=int(sc[0]), loglik=float(sc[1]), mu=float(sc[2]), mu_used=float(sc[3]))

    def describe(self) -> dict:
        """The launch plan: per digit the kernel ('group' or 'tile'), lanes/tile and grid."""
        import json
        buf = ctypes.create_string_buffer(8192)
        _check(_lib.pf_describe(self._h, buf, len(buf)), self._h)
        return json.loads(buf.value.decode())

    def ancestors(self) -> np.ndarray:
        anc = np.empty(self.N, dtype=np.int32)
        _check(_lib.pf_get_ancestors(self._h, anc.ctypes.data_as(ctypes.c_void_p)), self._h)
        return anc

    def draw_prefix(self) -> np.ndarray:
        """Integer prefix sums of the last step's draws (pf_get_draw_prefix), uint64 (N,)."""
        out = np.empty(self.N, dtype=np.uint64)
        _check(_lib.pf_get_draw_prefix(self._h, out.ctypes.data_as(ctypes.c_void_p)), self._h)
        return out

    def status(self) -> int:
        b = ctypes.c_uint32(0)
        _check(_lib.pf_get_status(self._h, ctypes.byref(b)), self._h)
        return b.value

    def save(self) -> np.ndarray:
        """Checkpoint (uint8 array): the whole filter state; see pf_save."""
        n = ctypes.c_size_t(0)
        _check(_lib.pf_checkpoint_size(self._h, ctypes.byref(n)), self._h)
        buf = np.empty(int(n.value), dtype=np.uint8)
        _check(_lib.pf_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes), self._h)
        return buf

    def load(self, buf) -> None:
        """Restore a checkpoint taken with save() from a filter with the same model,
        N, radices, seed and options; the run continues bit for bit."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(_lib.pf_load(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes), self._h)
        n = ctypes.c_double * 4
        sc = n()
        _check(_lib.pf_get_state(self._h, None, None, sc), self._h)
        self.steps = int(sc[0])

    def stage_count(self) -> int:
        """Resampling stages executed so far (with adaptive=True, those the ESS test let run)."""
        c = ctypes.c_uint64(0)
        _check(_lib.pf_stage_count(self._h, ctypes.byref(c)), self._h)
        return int(c.value)


class FilterBatch:
    """F independent filters (own model, N, radices, seed) advanced together, one
    kernel launch per time step for the whole batch (pf_batch_*)."""

    def __init__(self, specs, *, chunk_len: int = 0, device=None, stream=None, tile: int = 0, unit_work: int = 0,
                 tune: bool = False):
        """specs: sequence of (model, N, radices, seed).  tile: particles per tile of
        the shared-memory tile code (0 = by state dimension); unit_work: work of one
        thread block in particle-dimensions (a filter's step is split over
        ceil(N (d + 1) / unit_work) blocks; 0 = the library's default); tune=True
        takes both from the autotuner (cached per device and batch shape)."""
        torch = _torch()
        lib = load_library()
        if not torch.cuda.is_available():
            raise PFError(PF_ECUDA, "no CUDA device: the butterfly filter runs only on the GPU")
        if tune:
            from . import autotune
            best = autotune.tune_batch(specs, device=device)
            tile, unit_work = int(best["tile"]), int(best["unit_work"])
        self.tile, self.unit_work = int(tile), int(unit_work)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.F = len(specs)
        self._keep = []
        models = (PFModel * self.F)()
        for f, (model, N, radices, seed) in enumerate(specs):
            pm, keep = make_model(model)
            models[f] = pm
            self._keep.append(keep)
        self._models = models
        self.N = [int(s[1]) for s in specs]
        self.radices = [tuple(int(a) for a in s[2]) for s in specs]
        self.d = [models[f].d for f in range(self.F)]
        self.dy = [models[f].dy for f in range(self.F)]
        self.d_max, self.dy_max = max(self.d), max(self.dy)
        self._N = (ctypes.c_int64 * self.F)(*self.N)
        flat = [a for r in self.radices for a in r]
        self._rad = (ctypes.c_int32 * len(flat))(*flat)
        self._m = (ctypes.c_int32 * self.F)(*[len(r) for r in self.radices])
        self._seeds = (ctypes.c_uint64 * self.F)(*[int(s[3]) for s in specs])
        self._opts = PFOptions(tile=int(tile), chunk_len=int(chunk_len), flags=0, grid=int(unit_work),
                               stream=ctypes.c_void_p(self.stream.cuda_stream))
        with torch.cuda.device(self.device):
            nbytes = ctypes.c_size_t(0)
            _check(lib.pf_batch_workspace_size(self.F, models, self._N, self._rad, self._m, ctypes.byref(self._opts),
                                               ctypes.byref(nbytes)))
            self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            st = lib.pf_batch_create(self.F, models, self._N, self._rad, self._m, self._seeds, ctypes.byref(self._opts),
                                     _cuda_ptr(self.workspace), int(nbytes.value), ctypes.byref(h))
            if st != PF_OK:
                raise PFError(st, lib.pf_batch_last_error(None).decode(errors="replace"))
        self._h = h
        self.steps = 0

    def _check(self, st):
        if st != PF_OK:
            raise PFError(st, _lib.pf_batch_last_error(self._h).decode(errors="replace"))

    def close(self):
        if getattr(self, "_h", None):
            self._check(_lib.pf_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, y, outputs: bool = True):
        """y: (F, T, dy_max) float32 (numpy, or torch on host or device).  Returns
        dict(inc (F, T), mean (F, T, d_max), ess (F, T)) (numpy for host input, torch otherwise)."""
        torch = _torch()
        if isinstance(y, torch.Tensor):
            yt = y.to(torch.float32).contiguous()
            T = yt.shape[1]
            ptr, keep, on_dev = ctypes.c_void_p(yt.data_ptr()), yt, yt.is_cuda
        else:
            ya = np.ascontiguousarray(np.asarray(y, dtype=np.float32))
            T = ya.shape[1]
            ptr, keep, on_dev = ya.ctypes.data_as(ctypes.c_void_p), ya, False
        res = None
        ip = mp = ep = None
        if outputs:
            if on_dev:
                res = dict(inc=torch.empty((self.F, T), dtype=torch.float64, device=self.device),
                           mean=torch.empty((self.F, T, self.d_max), dtype=torch.float32, device=self.device),
                           ess=torch.empty((self.F, T), dtype=torch.float32, device=self.device))
                ip, mp, ep = (ctypes.c_void_p(res[k].data_ptr()) for k in ("inc", "mean", "ess"))
            else:
                res = dict(inc=np.empty((self.F, T)), mean=np.empty((self.F, T, self.d_max), dtype=np.float32),
                           ess=np.empty((self.F, T), dtype=np.float32))
                ip, mp, ep = (res[k].ctypes.data_as(ctypes.c_void_p) for k in ("inc", "mean", "ess"))
        self._check(_lib.pf_batch_run(self._h, ptr, int(T), ip, mp, ep))
        del keep
        self.steps += T
        return res

    def loglik(self) -> np.ndarray:
        out = np.empty(self.F)
        self._check(_lib.pf_batch_loglik(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def state(self, f: int):
        """(x (N, d), lV, dict(n, loglik, mu, mu_used)) of filter f."""
        m = len(self.radices[f])
        kp = (self.steps - 1) % m
        x = np.empty((self.d[f], self.N[f]), dtype=np.float32)
        lv = np.empty(self.N[f] // self.radices[f][kp], dtype=np.float32)
        sc = np.empty(4)
        self._check(_lib.pf_batch_get_state(self._h, int(f), x.ctypes.data_as(ctypes.c_void_p),
                                            lv.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p)))
        return x.T.copy(), lv, dict(n=int(sc[0]), loglik=float(sc[1]), mu=float(sc[2]), mu_used=float(sc[3]))


def philox_blocks(seed: int, counter, count: int, device=None):
    """Philox4x32-7 words for counters (c0 + j, c1, c2, c3), j < count: a (count, 4) int64
    tensor of uint32 values (computed on the GPU by the library)."""
    torch = _torch()
    lib = load_library()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(4 * count, dtype=torch.int32, device=dev)
    c0, c1, c2, c3 = (int(v) & 0xFFFFFFFF for v in counter)
    _check(lib.pf_philox_blocks(ctypes.c_uint64(seed), c0, c1, c2, c3, int(count), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
    return (out.to(torch.int64) & 0xFFFFFFFF).reshape(count, 4)


__all__ = ["ButterflyFilter", "FilterBatch", "PFError", "philox_blocks", "load_library", "make_model", "LIB_PATH"]
