"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every function declared in include/*.h, and rejects
invalid arguments before touching the device."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

import paper_2608_09102_b300 as ll
from paper_2608_09102_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*\s*\**\s+)+\**\s*(ll_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ll.load_library()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert {"ll_mg_setup", "ll_mg_solve", "ll_step", "ll_mg_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(ll.EXPORTS) <= declared


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)
    assert os.path.exists(build.LIB)


def test_default_params_match_the_header(lib):
    p = ll.default_params()
    assert p == ll.Params()


def test_status_strings(lib):
    for st in (0, 1, 2, -1, -2, -3, -4, -5):
        assert ll.status_string(st)
    assert ll.status_string(12345) == "unknown status"
    import threading

    seen = []  # a fresh thread: no CUDA call of it has failed, so no error text
    t = threading.Thread(target=lambda: seen.append(ll.last_cuda_error()))
    t.start()
    t.join()
    assert seen == [""]
    d = ll.Params()  # the binding's defaults mirror the library's
    c = ll._Params()
    ll.load_library().ll_mg_default_params(ctypes.byref(c))
    assert (c.stall_window, c.stall_ratio) == (d.stall_window, d.stall_ratio) == (0, 0.99)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    out = ctypes.c_void_p()
    g = ll._Grid(8, 8, 1)
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert lib.ll_mg_setup(None, 0.1, 1e-3, 0.1, g, None, None, ctypes.byref(out)) == ll.LL_EINVAL
    assert lib.ll_mg_setup(dummy, 0.1, 0.0, 0.1, g, None, None, ctypes.byref(out)) == ll.LL_EINVAL
    assert lib.ll_mg_setup(dummy, -1.0, 1e-3, 0.1, g, None, None, ctypes.byref(out)) == ll.LL_EINVAL
    assert lib.ll_mg_setup(dummy, 0.1, 1e-3, -0.1, g, None, None, ctypes.byref(out)) == ll.LL_EINVAL
    assert lib.ll_mg_setup(dummy, 0.1, 1e-3, 0.1, ll._Grid(1, 1, 1), None, None, ctypes.byref(out)) == ll.LL_EINVAL
    bad = ll.Params(restart=0)._c()
    assert lib.ll_mg_setup(dummy, 0.1, 1e-3, 0.1, g, ctypes.byref(bad), None, ctypes.byref(out)) == ll.LL_EINVAL
    bad = ll.Params(precision=7)._c()
    assert lib.ll_mg_setup(dummy, 0.1, 1e-3, 0.1, g, ctypes.byref(bad), None, ctypes.byref(out)) == ll.LL_EINVAL
    bad = ll.Params(kcycle=-1)._c()
    assert lib.ll_mg_setup(dummy, 0.1, 1e-3, 0.1, g, ctypes.byref(bad), None, ctypes.byref(out)) == ll.LL_EINVAL
    for kw in (dict(stall_window=-1), dict(stall_window=20, stall_ratio=0.0),
               dict(stall_window=20, stall_ratio=float("nan"))):
        bad = ll.Params(**kw)._c()
        assert lib.ll_mg_setup(dummy, 0.1, 1e-3, 0.1, g, ctypes.byref(bad), None, ctypes.byref(out)) == ll.LL_EINVAL
    assert lib.ll_mg_solve(None, dummy, dummy, 0.0, None, None) == ll.LL_EINVAL
    assert lib.ll_step(None, 1, 0.1, 1e-3, 0.1, g, None, None, None, None) == ll.LL_EINVAL
    assert lib.ll_mg_levels(None) == -1
    lib.ll_mg_destroy(None)


def test_binding_refuses_cpu_tensors_for_device_arguments(lib):
    import torch

    with pytest.raises(TypeError):
        ll.Hierarchy(torch.zeros(3 * 64, dtype=torch.float64), 0.1, 1e-3, 1 / 8, (8, 8, 1))
