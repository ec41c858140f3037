"""B300-native aggregation-multigrid solver for the semi-implicit BDF1
Landau-Lifshitz system (Python binding of the C ABI in ``include/ll_mg.h``).

The binding only marshals arguments: every step of the solve runs in the
hand-written sm_103a kernels of ``_lib/libllmg.so``.  PyTorch provides the
device memory and the current CUDA stream.  There is no CPU fallback: if the
library is missing or no CUDA device is present the calls raise.

Fields are float64 tensors holding 3*N values in component-major order (m1 of
all cells, then m2, then m3; cell (x, y, z) at x + nx*(y + ny*z)), e.g. of
shape (3, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libllmg.so")

LL_OK, LL_NOT_CONVERGED, LL_BREAKDOWN = 0, 1, 2
LL_EINVAL, LL_ECUDA, LL_ENOMEM, LL_SINGULAR_COARSE, LL_ELIMIT = -1, -2, -3, -4, -5
LL_FP64, LL_MIXED_FP32, LL_MIXED_BF16 = 0, 1, 2

# every symbol declared in include/ll_mg.h
EXPORTS = (
    "ll_mg_default_params", "ll_mg_setup", "ll_mg_update", "ll_mg_solve", "ll_step", "ll_mg_destroy",
    "ll_status_string", "ll_mg_levels", "ll_mg_level_cells", "ll_mg_level_aggregates",
    "ll_mg_level_colours", "ll_mg_level_blocks", "ll_mg_level_operator", "ll_mg_apply", "ll_mg_vcycle",
    "ll_mg_smooth", "ll_mg_step", "ll_launch_count", "ll_mg_profile", "ll_mg_profile_read",
    "ll_residual_noalloc", "ll_mg_step_llg", "ll_mg_batch_setup", "ll_mg_batch_update", "ll_mg_batch_solve",
    "ll_mg_batch_count", "ll_mg_batch_levels", "ll_mg_batch_level_rows", "ll_mg_batch_level_colours",
    "ll_mg_batch_instance_levels", "ll_mg_batch_destroy", "ll_mg_step_save", "ll_mg_batch_subbatches", "ll_mg_adjoint_setup",
    "ll_mg_step_vjp", "ll_mg_step_host", "ll_fp64_fma_probe", "ll_mg_batch_setup_groups", "ll_mg_batch_groups",
    "ll_mg_batch_instance_group", "ll_mg_batch_autotune", "ll_mg_tune_octave", "ll_mg_tune_lookup",
    "ll_last_cuda_error",
)


class LLError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = "%s failed: %s (status %d)" % (what, status_string(status), status)
        if status in (LL_ECUDA, LL_ENOMEM):
            detail = last_cuda_error()
            if detail:
                msg += ": " + detail
        super().__init__(msg)
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [
        ("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("restart", ctypes.c_int),
        ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("coarsest_cells", ctypes.c_int),
        ("max_levels", ctypes.c_int), ("rounds", ctypes.c_int), ("seed", ctypes.c_uint),
        ("precision", ctypes.c_int), ("kcycle", ctypes.c_int), ("coarse_lanes", ctypes.c_int),
        ("coarse_block", ctypes.c_int), ("stall_window", ctypes.c_int), ("stall_ratio", ctypes.c_double),
    ]


@dataclass
class Params:
    """Mirror of ``ll_mg_params`` with the library's defaults."""

    rtol: float = 1e-8
    maxit: int = 1000
    restart: int = 10
    nu_pre: int = 1
    nu_post: int = 1
    coarsest_cells: int = 64
    max_levels: int = 20
    rounds: int = 32
    seed: int = 0
    precision: int = LL_FP64
    kcycle: int = 0
    coarse_lanes: int = 0
    coarse_block: int = 0
    stall_window: int = 0
    stall_ratio: float = 0.99

    def _c(self) -> _Params:
        return _Params(self.rtol, self.maxit, self.restart, self.nu_pre, self.nu_post, self.coarsest_cells,
                       self.max_levels, self.rounds, self.seed & 0xFFFFFFFF, self.precision, self.kcycle,
                       self.coarse_lanes, self.coarse_block, self.stall_window, self.stall_ratio)

    @classmethod
    def _from_c(cls, c: "_Params") -> "Params":
        return cls(c.rtol, c.maxit, c.restart, c.nu_pre, c.nu_post, c.coarsest_cells, c.max_levels, c.rounds,
                   c.seed, c.precision, c.kcycle, c.coarse_lanes, c.coarse_block, c.stall_window, c.stall_ratio)


_lib = None


def load_library():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("the sm_103a library %s is missing; build it with "
                           "paper_2608_09102_b300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    ip, dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER(_Params)
    sig = {
        "ll_mg_default_params": (None, [P]),
        "ll_mg_setup": (i, [vp, d, d, d, _Grid, P, vp, ctypes.POINTER(vp)]),
        "ll_mg_update": (i, [vp, vp, d, d]),
        "ll_mg_solve": (i, [vp, vp, vp, d, ip, dp]),
        "ll_step": (i, [vp, i, d, d, d, _Grid, P, vp, ip, dp]),
        "ll_mg_destroy": (None, [vp]),
        "ll_status_string": (ctypes.c_char_p, [i]),
        "ll_mg_levels": (i, [vp]),
        "ll_mg_level_cells": (i, [vp, i]),
        "ll_mg_level_aggregates": (i, [vp, i, vp]),
        "ll_mg_level_colours": (i, [vp, i, vp]),
        "ll_mg_level_blocks": (i, [vp, i]),
        "ll_mg_level_operator": (i, [vp, i, vp, vp, vp]),
        "ll_mg_apply": (i, [vp, vp, vp]),
        "ll_mg_vcycle": (i, [vp, vp, vp]),
        "ll_mg_smooth": (i, [vp, i, vp, vp, i]),
        "ll_mg_step": (i, [vp, vp, i, ip, dp]),
        "ll_launch_count": (ctypes.c_longlong, []),
        "ll_mg_profile": (i, [vp, ctypes.c_uint]),
        "ll_mg_profile_read": (i, [vp, i, dp, ctypes.POINTER(ctypes.c_longlong), dp, dp]),
        "ll_residual_noalloc": (i, [vp, d, d, d, _Grid, vp, vp, vp, vp, vp]),
        "ll_mg_step_llg": (i, [vp, vp, i, d, vp, ip, dp]),
        "ll_mg_batch_setup": (i, [i, vp, vp, vp, vp, vp, P, vp, ctypes.POINTER(vp)]),
        "ll_mg_batch_update": (i, [vp, vp, vp, vp]),
        "ll_mg_batch_solve": (i, [vp, vp, vp, d, vp, vp, vp]),
        "ll_mg_batch_count": (i, [vp]),
        "ll_mg_batch_levels": (i, [vp]),
        "ll_mg_batch_level_rows": (ctypes.c_longlong, [vp, i]),
        "ll_mg_batch_level_colours": (i, [vp, i]),
        "ll_mg_batch_instance_levels": (i, [vp, i]),
        "ll_mg_batch_subbatches": (i, [vp]),
        "ll_mg_batch_destroy": (None, [vp]),
        "ll_mg_step_save": (i, [vp, vp, i, vp, ip, dp]),
        "ll_mg_adjoint_setup": (i, [vp, d, d, d, _Grid, P, vp, ctypes.POINTER(vp)]),
        "ll_mg_step_vjp": (i, [vp, vp, d, d, vp, vp, vp, dp, d, ip, dp]),
        "ll_mg_step_host": (i, [vp, vp, i, ip, dp]),
        "ll_fp64_fma_probe": (i, [vp, ctypes.c_longlong, i, vp, dp]),
        "ll_mg_batch_setup_groups": (i, [i, vp, vp, vp, vp, vp, P, vp, ctypes.POINTER(vp)]),
        "ll_mg_batch_groups": (i, [vp]),
        "ll_mg_batch_instance_group": (i, [vp, i]),
        "ll_mg_batch_autotune": (i, [i, vp, vp, vp, vp, vp, P, ctypes.c_char_p, vp, P, ip]),
        "ll_mg_tune_octave": (i, [d, d]),
        "ll_mg_tune_lookup": (i, [ctypes.c_char_p, _Grid, d, d, P]),
        "ll_last_cuda_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load_library().ll_status_string(int(status)).decode()


def last_cuda_error() -> str:
    """The CUDA call behind this thread's last LL_ECUDA / LL_ENOMEM ("" if none)."""
    return load_library().ll_last_cuda_error().decode()


def default_params() -> Params:
    c = _Params()
    load_library().ll_mg_default_params(ctypes.byref(c))
    return Params._from_c(c)


def _grid(grid) -> _Grid:
    g = [int(v) for v in grid] + [1] * (3 - len(grid))
    return _Grid(*g)


def _field(t, n, name):
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("%s must be a float64 CUDA tensor" % name)
    if not t.is_contiguous() or t.numel() != 3 * n:
        raise ValueError("%s must be contiguous with 3*N = %d values" % (name, 3 * n))
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(st, what, ok=(LL_OK, LL_NOT_CONVERGED, LL_BREAKDOWN)):
    if st not in ok:
        raise LLError(st, what)
    return st


class Hierarchy:
    """Library-owned multigrid hierarchy for one grid (``ll_mg_setup``)."""

    def __init__(self, m_tilde, alpha, dt, h, grid, params: Params | None = None):
        lib = load_library()
        g = _grid(grid)
        self.grid = (g.nx, g.ny, g.nz)
        nx, ny, nz = self.grid
        self.n = nx * ny * nz
        self.params = params or Params()
        self._h = ctypes.c_void_p()
        self._cp = self.params._c()
        st = lib.ll_mg_setup(_field(m_tilde, self.n, "m_tilde"), float(alpha), float(dt), float(h), _grid(grid),
                             ctypes.byref(self._cp), _stream(), ctypes.byref(self._h))
        _check(st, "ll_mg_setup", ok=(LL_OK,))

    def close(self):
        if self._h:
            load_library().ll_mg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, m_tilde, alpha, dt):
        st = load_library().ll_mg_update(self._h, _field(m_tilde, self.n, "m_tilde"), float(alpha), float(dt))
        _check(st, "ll_mg_update", ok=(LL_OK,))

    def solve(self, rhs, x, rtol: float = 0.0):
        """Solve in place (x: initial guess in, solution out); returns
        (status, iterations, true relative residual)."""
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load_library().ll_mg_solve(self._h, _field(rhs, self.n, "rhs"), _field(x, self.n, "x"), float(rtol),
                                        ctypes.byref(it), ctypes.byref(rr))
        _check(st, "ll_mg_solve")
        return st, it.value, rr.value

    def step(self, m, n_steps: int = 1):
        """n_steps time steps on this hierarchy (``ll_mg_step``), in place.

        ``m`` may be a CUDA tensor or a CPU tensor (copied to the device and
        back).  Returns (status, iterations per step, relres per step)."""
        dev = m if m.is_cuda else m.to("cuda", non_blocking=True)
        its = (ctypes.c_int * max(1, n_steps))()
        rrs = (ctypes.c_double * max(1, n_steps))()
        st = load_library().ll_mg_step(self._h, _field(dev, self.n, "m"), int(n_steps), its, rrs)
        _check(st, "ll_mg_step")
        if dev is not m:
            m.copy_(dev, non_blocking=False)
        return st, list(its[:n_steps]), list(rrs[:n_steps])

    def step_host(self, m, n_steps: int = 1):
        """n_steps steps of a field in HOST memory (``ll_mg_step_host``): the
        library copies ``m`` (a contiguous float64 CPU tensor, best pinned) to
        the device, steps it and copies the result back into ``m``.  Returns
        (status, iterations per step, relres per step)."""
        import torch

        if not isinstance(m, torch.Tensor) or m.is_cuda or m.dtype != torch.float64:
            raise TypeError("m must be a float64 CPU tensor")
        if not m.is_contiguous() or m.numel() != 3 * self.n:
            raise ValueError("m must be contiguous with 3*N = %d values" % (3 * self.n))
        its = (ctypes.c_int * max(1, n_steps))()
        rrs = (ctypes.c_double * max(1, n_steps))()
        st = load_library().ll_mg_step_host(self._h, ctypes.c_void_p(m.data_ptr()), int(n_steps), its, rrs)
        _check(st, "ll_mg_step_host")
        return st, list(its[:n_steps]), list(rrs[:n_steps])

    def step_save(self, m, x_save, n_steps: int = 1):
        """n_steps steps in place (``ll_mg_step_save``); x_save (CUDA,
        3*N*n_steps) receives each step's solution before the projection."""
        import torch

        if x_save.dtype != torch.float64 or not x_save.is_cuda:
            raise TypeError("x_save must be a float64 CUDA tensor")
        if x_save.numel() != 3 * self.n * n_steps or not x_save.is_contiguous():
            raise ValueError("x_save must hold 3*N*n_steps contiguous values")
        its = (ctypes.c_int * max(1, n_steps))()
        rrs = (ctypes.c_double * max(1, n_steps))()
        st = load_library().ll_mg_step_save(self._h, _field(m, self.n, "m"), int(n_steps),
                                            ctypes.c_void_p(x_save.data_ptr()), its, rrs)
        _check(st, "ll_mg_step_save")
        return st, list(its[:n_steps]), list(rrs[:n_steps])

    def step_llg(self, m, n_steps: int = 1, q: float = 0.0, he=(0.0, 0.0, 0.0)):
        """Time steps with the explicit anisotropy and external-field terms
        (``ll_mg_step_llg``); set the hierarchy up with h/sqrt(eps)."""
        dev = m if m.is_cuda else m.to("cuda", non_blocking=True)
        its = (ctypes.c_int * max(1, n_steps))()
        rrs = (ctypes.c_double * max(1, n_steps))()
        hev = (ctypes.c_double * 3)(*[float(v) for v in he])
        st = load_library().ll_mg_step_llg(self._h, _field(dev, self.n, "m"), int(n_steps), float(q), hev, its, rrs)
        _check(st, "ll_mg_step_llg")
        if dev is not m:
            m.copy_(dev, non_blocking=False)
        return st, list(its[:n_steps]), list(rrs[:n_steps])

    # -- introspection ---------------------------------------------------
    @property
    def levels(self) -> int:
        return load_library().ll_mg_levels(self._h)

    def level_cells(self, l: int) -> int:
        return load_library().ll_mg_level_cells(self._h, l)

    def aggregates(self, l: int):
        import numpy as np

        out = np.zeros(self.level_cells(l), np.int32)
        _check(load_library().ll_mg_level_aggregates(self._h, l, out.ctypes.data), "ll_mg_level_aggregates")
        return out

    def colours(self, l: int):
        import numpy as np

        out = np.zeros(self.level_cells(l), np.int32)
        _check(load_library().ll_mg_level_colours(self._h, l, out.ctypes.data), "ll_mg_level_colours")
        return out

    def operator(self, l: int):
        """BSR operator of level l >= 1 as (rowptr, col, val[nnzb, 3, 3])."""
        import numpy as np

        lib = load_library()
        n = self.level_cells(l)
        nb = lib.ll_mg_level_blocks(self._h, l)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nb, np.int32)
        va = np.zeros(9 * nb, np.float64)
        _check(lib.ll_mg_level_operator(self._h, l, rp.ctypes.data, ci.ctypes.data, va.ctypes.data),
               "ll_mg_level_operator")
        return rp, ci, va.reshape(nb, 3, 3)

    def apply(self, x, y):
        _check(load_library().ll_mg_apply(self._h, _field(x, self.n, "x"), _field(y, self.n, "y")), "ll_mg_apply",
               ok=(LL_OK,))

    def vcycle(self, r, z):
        _check(load_library().ll_mg_vcycle(self._h, _field(r, self.n, "r"), _field(z, self.n, "z")),
               "ll_mg_vcycle", ok=(LL_OK,))

    def smooth(self, l: int, b, x, forward: bool = True):
        n = self.n if l == 0 else self.level_cells(l)
        st = load_library().ll_mg_smooth(self._h, l, _field(b, n, "b"), _field(x, n, "x"), 1 if forward else 0)
        _check(st, "ll_mg_smooth", ok=(LL_OK,))


def residual_noalloc(m_tilde, alpha, dt, h, grid, rhs, x, r=None, norms2=None):
    """``ll_residual_noalloc``: r = rhs - A x and (|r|^2, |rhs|^2) into the
    2-element float64 CUDA tensor ``norms2`` without any device allocation
    inside the library.  Returns ``norms2`` (enqueued on the current stream)."""
    import torch

    g = _grid(grid)
    n = g.nx * g.ny * g.nz
    if norms2 is None:
        norms2 = torch.empty(2, dtype=torch.float64, device=rhs.device)
    rp = _field(r, n, "r") if r is not None else None
    st = load_library().ll_residual_noalloc(_field(m_tilde, n, "m_tilde"), float(alpha), float(dt), float(h), g,
                                            _field(rhs, n, "rhs"), _field(x, n, "x"), rp,
                                            ctypes.c_void_p(norms2.data_ptr()), _stream())
    _check(st, "ll_residual_noalloc", ok=(LL_OK,))
    return norms2


class Adjoint:
    """Solves with A(m~)^T and vector-Jacobian products of single steps
    (``ll_mg_adjoint_setup`` / ``ll_mg_step_vjp``)."""

    def __init__(self, m_tilde, alpha, dt, h, grid, params: Params | None = None):
        lib = load_library()
        g = _grid(grid)
        self.grid = (g.nx, g.ny, g.nz)
        self.n = g.nx * g.ny * g.nz
        self.params = params or Params()
        self._cp = self.params._c()
        self._h = ctypes.c_void_p()
        st = lib.ll_mg_adjoint_setup(_field(m_tilde, self.n, "m_tilde"), float(alpha), float(dt), float(h), g,
                                     ctypes.byref(self._cp), _stream(), ctypes.byref(self._h))
        _check(st, "ll_mg_adjoint_setup", ok=(LL_OK,))

    def close(self):
        if self._h:
            load_library().ll_mg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, m_tilde, alpha, dt):
        a = (ctypes.c_double * 1)(float(alpha))
        d = (ctypes.c_double * 1)(float(dt))
        st = load_library().ll_mg_batch_update(self._h, _ptrs([m_tilde], [self.n], "m_tilde"), a, d)
        _check(st, "ll_mg_batch_update", ok=(LL_OK,))

    def solve(self, rhs, lam, rtol: float = 0.0):
        """A^T lam = rhs in place; returns (status, iterations, relres)."""
        its = (ctypes.c_int * 1)()
        rrs = (ctypes.c_double * 1)()
        sts = (ctypes.c_int * 1)()
        st = load_library().ll_mg_batch_solve(self._h, _ptrs([rhs], [self.n], "rhs"), _ptrs([lam], [self.n], "x"),
                                              float(rtol), its, rrs, sts)
        _check(st, "ll_mg_batch_solve")
        return st, its[0], rrs[0]

    def vjp(self, m, alpha, dt, x, g, m_bar=None, rtol: float = 0.0):
        """(dL/dm^n, dL/dalpha part, status, iterations, relres) of one step
        m^n -> x/|x| for g = dL/dm^{n+1}."""
        import torch

        if m_bar is None:
            m_bar = torch.empty_like(m)
        ab = ctypes.c_double(0.0)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = load_library().ll_mg_step_vjp(self._h, _field(m, self.n, "m"), float(alpha), float(dt),
                                           _field(x, self.n, "x"), _field(g, self.n, "g"),
                                           _field(m_bar, self.n, "m_bar"), ctypes.byref(ab), float(rtol),
                                           ctypes.byref(it), ctypes.byref(rr))
        _check(st, "ll_mg_step_vjp")
        return m_bar, ab.value, st, it.value, rr.value


def _steps_function():
    import torch

    class _Steps(torch.autograd.Function):
        """m^N of n_steps semi-implicit steps, differentiable in m^0 and
        alpha; the backward pass recomputes each segment of `checkpoint`
        steps from its stored initial state, then runs the step VJPs
        backwards through it."""

        @staticmethod
        def forward(ctx, m0, alpha, n_steps, dt, h, grid, params, checkpoint):
            a = float(alpha)
            H = Hierarchy(m0.detach(), a, dt, h, grid, params)
            m = m0.detach().clone()
            x = torch.empty_like(m)
            ckpt = {0: m.clone()}
            for k in range(n_steps):
                H.step_save(m, x)
                if (k + 1) % checkpoint == 0 and k + 1 < n_steps:
                    ckpt[k + 1] = m.clone()
            ctx.H, ctx.ckpt, ctx.cfg = H, ckpt, (a, n_steps, dt, h, grid, params, checkpoint)
            ctx.save_for_backward(m0)
            return m

        @staticmethod
        def backward(ctx, g_out):
            (m0,) = ctx.saved_tensors
            a, n_steps, dt, h, grid, params, checkpoint = ctx.cfg
            H = ctx.H
            T = Adjoint(m0.detach(), a, dt, h, grid, params)
            g = g_out.detach().contiguous().clone()
            abar = 0.0
            x = torch.empty_like(g)
            for s0 in sorted(ctx.ckpt, reverse=True):
                s1 = min(s0 + checkpoint, n_steps)
                m = ctx.ckpt[s0].clone()
                ms, xs = [], []
                for _ in range(s0, s1):  # recompute the segment's states and solutions
                    ms.append(m.clone())
                    H.step_save(m, x)
                    xs.append(x.clone())
                for k in range(len(ms) - 1, -1, -1):
                    g, ak, st, it, rr = T.vjp(ms[k], a, dt, xs[k], g)
                    abar += ak
            T.close()
            galpha = torch.tensor(abar, dtype=torch.float64) if ctx.needs_input_grad[1] else None
            return g, galpha, None, None, None, None, None, None

    return _Steps


_STEPS = None


def steps_autograd(m0, alpha, n_steps: int, dt, h, grid, params: Params | None = None, checkpoint: int = 5):
    """m^N after n_steps steps from m0 (float64 CUDA tensor), differentiable
    with respect to m0 and alpha (a float or a 0-dim float64 tensor) through
    the library's adjoint; states are stored every `checkpoint` steps and the
    rest recomputed in the backward pass."""
    import torch

    global _STEPS
    if _STEPS is None:
        _STEPS = _steps_function()
    if not isinstance(alpha, torch.Tensor):
        alpha = torch.tensor(float(alpha), dtype=torch.float64)
    return _STEPS.apply(m0, alpha, int(n_steps), float(dt), float(h), tuple(grid), params or Params(),
                        int(checkpoint))


def _ptrs(tensors, ns, name):
    arr = (ctypes.c_void_p * len(tensors))()
    for k, (t, n) in enumerate(zip(tensors, ns)):
        arr[k] = _field(t, n, "%s[%d]" % (name, k)).value
    return arr


class Batch:
    """Independent instances solved together (``ll_mg_batch_setup``): one
    hierarchy per instance, concatenated level by level, GCR in lockstep.

    ``params`` is one Params for every instance, or a list of one Params per
    instance (``ll_mg_batch_setup_groups``: instances with equal parameters
    form a group, and the groups run concurrently), e.g. the list
    ``autotune`` returns."""

    def __init__(self, m_tildes, alphas, dts, hs, grids, params=None):
        lib = load_library()
        self.count = len(m_tildes)
        gs = [_grid(g) for g in grids]
        self.grids = [(g.nx, g.ny, g.nz) for g in gs]
        self.ns = [g.nx * g.ny * g.nz for g in gs]
        garr = (_Grid * self.count)(*gs)
        dv = lambda v: (ctypes.c_double * self.count)(*[float(a) for a in v])  # noqa: E731
        self._h = ctypes.c_void_p()
        if isinstance(params, (list, tuple)):
            if len(params) != self.count:
                raise ValueError("one Params per instance")
            self.params = list(params)
            self._cp = (_Params * self.count)(*[q._c() for q in self.params])
            st = lib.ll_mg_batch_setup_groups(self.count, _ptrs(m_tildes, self.ns, "m_tilde"), dv(alphas), dv(dts),
                                              dv(hs), garr, self._cp, _stream(), ctypes.byref(self._h))
            _check(st, "ll_mg_batch_setup_groups", ok=(LL_OK,))
            return
        self.params = params or Params()
        self._cp = self.params._c()
        st = lib.ll_mg_batch_setup(self.count, _ptrs(m_tildes, self.ns, "m_tilde"), dv(alphas), dv(dts), dv(hs),
                                   garr, ctypes.byref(self._cp), _stream(), ctypes.byref(self._h))
        _check(st, "ll_mg_batch_setup", ok=(LL_OK,))

    def close(self):
        if self._h:
            load_library().ll_mg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, m_tildes, alphas, dts):
        dv = lambda v: (ctypes.c_double * self.count)(*[float(a) for a in v])  # noqa: E731
        st = load_library().ll_mg_batch_update(self._h, _ptrs(m_tildes, self.ns, "m_tilde"), dv(alphas), dv(dts))
        _check(st, "ll_mg_batch_update", ok=(LL_OK,))

    def solve(self, rhs, x, rtol: float = 0.0):
        """Solve every instance in place; returns (status, iterations,
        true relative residuals, per-instance statuses)."""
        its = (ctypes.c_int * self.count)()
        rrs = (ctypes.c_double * self.count)()
        sts = (ctypes.c_int * self.count)()
        st = load_library().ll_mg_batch_solve(self._h, _ptrs(rhs, self.ns, "rhs"), _ptrs(x, self.ns, "x"),
                                              float(rtol), its, rrs, sts)
        _check(st, "ll_mg_batch_solve")
        return st, list(its), list(rrs), list(sts)

    @property
    def levels(self) -> int:
        return load_library().ll_mg_batch_levels(self._h)

    def level_rows(self, level: int) -> int:
        return int(load_library().ll_mg_batch_level_rows(self._h, level))

    def level_colours(self, level: int) -> int:
        return load_library().ll_mg_batch_level_colours(self._h, level)

    def instance_levels(self, i: int) -> int:
        return load_library().ll_mg_batch_instance_levels(self._h, i)

    @property
    def subbatches(self) -> int:
        """Compacted sub-batches built so far (ll_mg_batch_subbatches)."""
        return load_library().ll_mg_batch_subbatches(self._h)

    @property
    def groups(self) -> int:
        """Groups of equal parameters (1 for a single parameter set)."""
        return load_library().ll_mg_batch_groups(self._h)

    def instance_group(self, i: int) -> int:
        return load_library().ll_mg_batch_instance_group(self._h, i)


def autotune(m_tildes, alphas, dts, hs, grids, base: Params | None = None, cache_path: str | None = None):
    """Per-class choice of cycle and coarse-kernel launch shape for a batch
    (``ll_mg_batch_autotune``); returns (one Params per instance, classes
    timed by this call)."""
    lib = load_library()
    count = len(m_tildes)
    gs = [_grid(g) for g in grids]
    ns = [g.nx * g.ny * g.nz for g in gs]
    garr = (_Grid * count)(*gs)
    dv = lambda v: (ctypes.c_double * count)(*[float(a) for a in v])  # noqa: E731
    bp = (base or Params())._c()
    out = (_Params * count)()
    tuned = ctypes.c_int(0)
    st = lib.ll_mg_batch_autotune(count, _ptrs(m_tildes, ns, "m_tilde"), dv(alphas), dv(dts), dv(hs), garr,
                                  ctypes.byref(bp), cache_path.encode() if cache_path else None, _stream(), out,
                                  ctypes.byref(tuned))
    _check(st, "ll_mg_batch_autotune", ok=(LL_OK,))
    return [Params._from_c(out[k]) for k in range(count)], tuned.value


def tune_octave(dt: float, h: float) -> int:
    """The autotuner's class octave floor(log2(dt/h^2)) (host only)."""
    return int(load_library().ll_mg_tune_octave(float(dt), float(h)))


def tune_lookup(cache_path: str, grid, dt: float, h: float, base: Params | None = None):
    """The autotuner's cached choice for one instance (host only): base
    with the choice applied, or None when the cache does not hold its class."""
    c = (base or Params())._c()
    st = load_library().ll_mg_tune_lookup(cache_path.encode(), _grid(grid), float(dt), float(h), ctypes.byref(c))
    if st < 0:
        raise LLError(st, "ll_mg_tune_lookup")
    return Params._from_c(c) if st == 1 else None


def fp64_fma_probe(sink, iters: int, blocks: int):
    """One launch of the library's float64 multiply-add probe on the current
    stream (``ll_fp64_fma_probe``); ``sink`` is a float64 CUDA tensor of at
    least one element.  Returns the launch's floating-point operations."""
    fl = ctypes.c_double(0.0)
    st = load_library().ll_fp64_fma_probe(ctypes.c_void_p(sink.data_ptr()), int(iters), int(blocks), _stream(),
                                          ctypes.byref(fl))
    _check(st, "ll_fp64_fma_probe", ok=(LL_OK,))
    return fl.value


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(load_library().ll_launch_count())


def step(m, n_steps: int, alpha, dt, h, grid, params: Params | None = None):
    """n_steps semi-implicit steps with projection (``ll_step``), in place.

    ``m`` may be a CUDA tensor, or a CPU tensor (then it is copied to the
    device through pinned memory and back).  Returns (status, iterations per
    step, relative residual per step)."""
    import torch

    lib = load_library()
    params = params or Params()
    g = _grid(grid)
    n = g.nx * g.ny * g.nz
    dev = m
    if not m.is_cuda:
        dev = m.pin_memory().to("cuda", non_blocking=True) if not m.is_pinned() else m.to("cuda", non_blocking=True)
    its = (ctypes.c_int * max(1, n_steps))()
    rrs = (ctypes.c_double * max(1, n_steps))()
    cp = params._c()
    st = lib.ll_step(_field(dev, n, "m"), int(n_steps), float(alpha), float(dt), float(h), g, ctypes.byref(cp),
                     _stream(), its, rrs)
    _check(st, "ll_step")
    if dev is not m:
        m.copy_(dev, non_blocking=False)
    return st, list(its[:n_steps]), list(rrs[:n_steps])
