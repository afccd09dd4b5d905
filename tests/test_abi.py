"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/bfpf.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "bfpf.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("pf_create", "pf_step", "pf_run", "pf_loglik", "pf_destroy", "pf_workspace_size",
              "pf_last_error", "pf_get_state"):
        assert n in names


def test_library_exports_every_declared_symbol(bfpf):
    lib = ctypes.CDLL(bfpf.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name


def test_library_targets_sm103a(bfpf):
    # the fatbinary of an sm_103a build names the architecture
    data = open(bfpf.LIB_PATH, "rb").read()
    assert b"sm_103a" in data


def _model_and_radices(bfpf, radices, N):
    import synthetic as S
    pm, keep = bfpf.make_model(S.lg_scalar())
    rad = (ctypes.c_int32 * len(radices))(*radices)
    return pm, keep, rad


@pytest.mark.parametrize("radices,N,msg", [
    ((4, 4, 2), 64, "product"),
    ((1, 64), 64, ">= 2"),
    ((2048, 2), 4096, "1024"),
])
def test_argument_checks_without_gpu(bfpf, radices, N, msg):
    lib = bfpf.load_library()
    pm, keep, rad = _model_and_radices(bfpf, radices, N)
    nbytes = ctypes.c_size_t(0)
    st = lib.pf_workspace_size(ctypes.byref(pm), N, rad, len(radices), None, ctypes.byref(nbytes))
    assert st == bfpf.PF_EINVAL
    assert msg in lib.pf_last_error(None).decode()


def test_null_arguments(bfpf):
    lib = bfpf.load_library()
    assert lib.pf_destroy(None) == bfpf.PF_OK
    assert lib.pf_loglik(None, None) == bfpf.PF_EINVAL
    assert lib.pf_step(None, None, None, None, None) == bfpf.PF_EINVAL


def test_binding_flags_match_the_header(bfpf):
    """Every PF_* flag and status code the header defines has the same value in the binding."""
    text = open(HEADER).read()
    defines = {name: int(val.rstrip("uU"), 0)
               for name, val in re.findall(r"#define\s+(PF_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+u?|\d+u?)\b", text)}
    assert "PF_ALL_STAGES" in defines and "PF_TEST_SMALL_BUCKETS" in defines
    for name, val in defines.items():
        if hasattr(bfpf, name):
            assert getattr(bfpf, name) == val, name
    for name in ("PF_RECORD_ANCESTORS", "PF_ALL_STAGES", "PF_ADAPTIVE", "PF_ROTATE", "PF_ISLANDS",
                 "PF_ISLANDS_PLAIN", "PF_DIGIT_SETS", "PF_TEST_SMALL_BUCKETS", "PF_TEST_STAGE_PER_LAUNCH"):
        assert getattr(bfpf, name) == defines[name], name
