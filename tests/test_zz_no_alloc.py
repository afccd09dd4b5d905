"""pf_step_noalloc: the time step for callers that may not allocate device memory.

Some callers run inside an engine or framework that owns every device
allocation, or in a real-time loop with a fixed memory budget; they cannot
call cudaMalloc and cannot keep a pf_create workspace.  pf_step_noalloc takes
their particle buffers as they are and keeps its temporaries in a scratch area
compiled into the library.  This test calls it through the C ABI for m + 1
steps in a row (so the digit wraps round and the carried weights of digit
m - 1 feed digit 0) and checks each step against the handle API (pf_create /
pf_step) from the same state, within the parity tolerances of the other GPU
tests; a NaN observation must come back as status bit 0.  It lives in a file
of its own so that it is collected last.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S
import lockstep as LS

pytestmark = pytest.mark.gpu


def _bind(lib, bfpf):
    fn = lib.pf_step_noalloc
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.POINTER(bfpf.PFModel), ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                   ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return fn


@pytest.mark.parametrize("name,model,radices", [
    ("sv_group_kernel", S.sv_model(), (16, 16, 16, 16)),
    ("lg4_tile_kernel", S.lg_dense(4, seed=3), (3, 5, 4, 8)),
    ("sv_two_digits", S.sv_model(), (16, 32)),
])
def test_noalloc_step_matches_handle_api(bfpf, name, model, radices):
    import torch
    lib = bfpf.load_library()
    step = _bind(lib, bfpf)
    N = int(np.prod(radices))
    seed = 2024
    d = model.d
    steps = len(radices) + 1
    y = S.simulate(model, steps, seed=31)[1]
    f = bfpf.ButterflyFilter(model, N, radices, seed)
    x0, _, _ = f.state()                                   # pi_0 draw of the handle
    dev = f.device
    stream = torch.cuda.current_stream(dev)
    x = torch.tensor(np.ascontiguousarray(x0.T), dtype=torch.float32, device=dev)   # state-major
    lv = [torch.zeros(N // radices[-1], dtype=torch.float32, device=dev)]
    pm, keep = bfpf.make_model(model)
    rad = (ctypes.c_int32 * len(radices))(*radices)
    mu = 0.0
    for n in range(steps):
        mean_h, inc_h, ess_h = f.step(y[n])
        xh, lvh, sch = f.state()
        lv_out = torch.empty(N // radices[n % len(radices)], dtype=torch.float32, device=dev)
        yn = np.ascontiguousarray(y[n], dtype=np.float32)
        out = np.zeros(3, dtype=np.float64)
        mean = np.zeros(d, dtype=np.float32)
        bits = ctypes.c_uint32(0xFFFF)
        st = step(ctypes.byref(pm), N, rad, len(radices), seed, n, mu,
                  ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lv[-1].data_ptr()),
                  ctypes.c_void_p(lv_out.data_ptr()), yn.ctypes.data_as(ctypes.c_void_p),
                  out.ctypes.data_as(ctypes.c_void_p), mean.ctypes.data_as(ctypes.c_void_p),
                  ctypes.byref(bits), ctypes.c_void_p(stream.cuda_stream))
        assert st == bfpf.PF_OK, lib.pf_last_error(None).decode()
        assert bits.value == 0
        lv.append(lv_out)
        mu = out[1]
        assert LS.rel_err(x.cpu().numpy().T, xh) <= LS.TOL_STATE
        assert LS.rel_err(lv_out.cpu().numpy(), lvh) <= LS.TOL_STATE
        assert abs(out[0] - inc_h) <= LS.TOL_INC * max(1.0, abs(inc_h))
        assert abs(out[1] - sch["mu"]) <= LS.TOL_INC * max(1.0, abs(sch["mu"]))
        assert LS.rel_err(mean, mean_h) <= LS.TOL_STATE
        assert abs(out[2] - ess_h) <= 1e-4 * ess_h
    f.close()
    del keep


def test_noalloc_reports_non_finite_weights(bfpf):
    """A NaN observation makes every log-weight NaN: the step treats them as weight
    zero, keeps the particles of the all-zero groups, and says so in status_out."""
    import torch
    lib = bfpf.load_library()
    step = _bind(lib, bfpf)
    model = S.sv_model()
    radices = (16, 16)
    N = 256
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.linspace(-1.0, 1.0, N, dtype=torch.float32, device=dev)
    lv_in = torch.zeros(N // 16, dtype=torch.float32, device=dev)
    lv_out = torch.empty(N // 16, dtype=torch.float32, device=dev)
    pm, keep = bfpf.make_model(model)
    rad = (ctypes.c_int32 * 2)(*radices)
    out = np.zeros(3)
    bits = ctypes.c_uint32(0)
    yn = np.array([np.nan], dtype=np.float32)
    st = step(ctypes.byref(pm), N, rad, 2, 5, 0, 0.0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lv_in.data_ptr()),
              ctypes.c_void_p(lv_out.data_ptr()), yn.ctypes.data_as(ctypes.c_void_p),
              out.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(bits),
              ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert st == bfpf.PF_OK, lib.pf_last_error(None).decode()
    assert bits.value & 1 and bits.value & 2, bits.value
    # the next call clears the bits: a finite observation reports none
    yn[0] = 0.3
    st = step(ctypes.byref(pm), N, rad, 2, 5, 0, 0.0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lv_in.data_ptr()),
              ctypes.c_void_p(lv_out.data_ptr()), yn.ctypes.data_as(ctypes.c_void_p),
              out.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(bits),
              ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert st == bfpf.PF_OK and bits.value == 0
    del keep


def test_noalloc_rejects_bad_sizes(bfpf):
    lib = bfpf.load_library()
    step = _bind(lib, bfpf)
    pm, keep = bfpf.make_model(S.lg_scalar())
    rad = (ctypes.c_int32 * 2)(4, 4)
    dummy = ctypes.c_void_p(1)
    out = np.zeros(3)
    st = step(ctypes.byref(pm), 32, rad, 2, 1, 0, 0.0, dummy, dummy, dummy,
              np.zeros(1, np.float32).ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
              None, None, None)
    assert st == bfpf.PF_EINVAL
    assert "product" in lib.pf_last_error(None).decode()
