"""The allocation-free residual entry point (ll_residual_noalloc), for
callers that cannot allocate device memory, checked through the C ABI
against the residual the hierarchy-based entry points give for the same
inputs (ll_mg_apply, and the true relative residual ll_mg_solve reports),
on two calls in a row.  Collected last on purpose."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_09102_b300 as ll  # noqa: E402
from paper_2608_09102_b300 import inputs  # noqa: E402

DEV = "cuda:0"
TOL = 1e-12  # float64 rounding of two summation orders of the same residual


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=DEV)


def test_noalloc_residual_matches_existing_entry_points_twice():
    grid, h, alpha, dt = (40, 36, 20), 1 / 40, 0.05, 2e-3
    m = _t(inputs.vortex(*grid, seed=3))
    H = ll.Hierarchy(m, alpha, dt, h, grid, ll.Params(rtol=1e-9))
    b = _t(inputs.rhs_field(*grid, seed=4))
    xs = [_t(inputs.rhs_field(*grid, seed=5)), m.clone()]
    st, it, rr = H.solve(b, xs[1])  # the second input is a converged solution
    assert st == ll.LL_OK
    norms = torch.empty(2, dtype=torch.float64, device=DEV)
    r = torch.empty_like(b)
    y = torch.empty_like(b)
    lib = ll.load_library()
    g = ll._Grid(*grid)

    def call(x):
        return lib.ll_residual_noalloc(ctypes.c_void_p(m.data_ptr()), alpha, dt, h, g, ctypes.c_void_p(b.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                       ctypes.c_void_p(norms.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    # the first call on a device does the one-time set-up (looking up the
    # scratch array's address, which may load the library's device code);
    # after it, calls leave the device's free memory unchanged
    assert call(xs[0]) == ll.LL_OK
    torch.cuda.synchronize()
    for k, x in enumerate(xs):
        free0 = torch.cuda.mem_get_info()[0]
        st = call(x)
        assert st == ll.LL_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        H.apply(x, y)  # existing entry point: y = A x
        r_ref = b - y
        scale = float(r_ref.abs().max())
        assert float((r - r_ref).abs().max()) <= TOL * max(scale, float(b.abs().max()))
        rn2, bn2 = float(norms[0]), float(norms[1])
        assert abs(bn2 - float((b * b).sum())) <= TOL * bn2
        # |r|^2 inherits the cancellation in b - A x: relative error about
        # eps |b| / |r|, i.e. 1e-12 for the random x and ~1e-7 once converged
        rel = TOL if k == 0 else 1e-5
        assert abs(rn2 - float((r_ref * r_ref).sum())) <= rel * rn2
        if k == 1:  # agrees with the true relative residual ll_mg_solve reported
            assert abs(np.sqrt(rn2 / bn2) - rr) <= 1e-5 * rr


def test_noalloc_rejects_grids_beyond_its_scratch():
    lib = ll.load_library()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    st = lib.ll_residual_noalloc(dummy, 0.1, 1e-3, 0.1, ll._Grid(4096, 2049, 1), dummy, dummy, None, dummy, None)
    assert st == ll.LL_ELIMIT
    st = lib.ll_residual_noalloc(dummy, 0.1, 0.0, 0.1, ll._Grid(8, 8, 8), dummy, dummy, None, dummy, None)
    assert st == ll.LL_EINVAL
