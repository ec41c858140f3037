"""Python harness of the FP64 CPU oracle (``ll_oracle.c``).

TEST INFRASTRUCTURE ONLY: the product path never imports this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

The oracle restates, slowly and in plain code, what the solver computes:

* the operator of the damped semi-implicit BDF1 scheme (Sec. 2.1, component
  form), divided by dt:  (A x)_k = x_k/dt + C(m_k) (Delta_h x)_k with
  C(m) = [m]_x + alpha (m m^T - |m|^2 I), assembled as a scalar CSR matrix in
  the component-major order [m1; m2; m3];
* aggregation by two passes of pairwise matching per level (Sec. 3.1.1), the
  Boolean prolongation of Eq. (Pagg), Galerkin products P^T A P
  (Eq. galerkin) by explicit sparse products;
* block Gauss-Seidel smoothing, V-cycle, dense LU at the coarsest level
  (Sec. 3);
* preconditioned GCR as Algorithm 1 (modified Gram-Schmidt);
* the time step with projection m <- m/|m| (Sec. 4).

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ll_oracle.c")
_LIB = os.path.join(_HERE, "_ll_oracle.so")

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("rtol", ctypes.c_double),
        ("maxit", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("nu_pre", ctypes.c_int),
        ("nu_post", ctypes.c_int),
        ("coarsest_cells", ctypes.c_int),
        ("max_levels", ctypes.c_int),
        ("rounds", ctypes.c_int),
        ("seed", ctypes.c_uint32),
        ("prec", ctypes.c_int),
        ("kcycle", ctypes.c_int),
        ("stall_window", ctypes.c_int),
        ("stall_ratio", ctypes.c_double),
    ]


@dataclass
class Params:
    """Solver parameters; defaults mirror the library's documented defaults.

    prec: 0 = aggregation V-cycle, 1 = none (plain GCR), 2 = exact (dense LU
    of the whole operator, tiny grids only).
    kcycle: coarse levels 1..kcycle are solved by two inner GCR steps (K-cycle).
    stall_window, stall_ratio: stagnation stop (not in the paper; 0 = off): at
    a restart, stop as not converged when the true residual norm exceeds
    stall_ratio times its value at the latest restart at least stall_window
    iterations earlier.
    """

    rtol: float = 1e-8
    maxit: int = 1000
    restart: int = 10
    nu_pre: int = 1
    nu_post: int = 1
    coarsest_cells: int = 64
    max_levels: int = 20
    rounds: int = 32
    seed: int = 0
    prec: int = 0
    kcycle: int = 0
    stall_window: int = 0
    stall_ratio: float = 0.99

    def _c(self) -> _Params:
        return _Params(self.rtol, self.maxit, self.restart, self.nu_pre, self.nu_post,
                       self.coarsest_cells, self.max_levels, self.rounds, self.seed & 0xFFFFFFFF,
                       self.prec, self.kcycle, self.stall_window, self.stall_ratio)


_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _load():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def bind(lib):
    """Declare the argument and result types of the oracle's exports on a
    loaded copy of the library (the tests also bind copies with a planted
    mistake, to show that the pins catch it)."""
    vp, i, d, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint32
    sig = {
        "orc_setup": (vp, [i, i, i, d, d, d, _dp, ctypes.POINTER(_Params)]),
        "orc_setup_adjoint": (vp, [i, i, i, d, d, d, _dp, ctypes.POINTER(_Params)]),
        "orc_step_vjp": (i, [i, i, i, d, d, d, ctypes.POINTER(_Params), _dp, _dp, _dp, _dp, ctypes.POINTER(d),
                             ctypes.POINTER(i), ctypes.POINTER(d)]),
        "orc_free": (None, [vp]),
        "orc_solve": (i, [vp, _dp, _dp, d, ctypes.POINTER(i), ctypes.POINTER(d), vp]),
        "orc_step": (i, [_dp, i, i, i, i, d, d, d, ctypes.POINTER(_Params), i, _ip, _dp]),
        "orc_step_llg": (i, [_dp, i, i, i, i, d, d, d, ctypes.POINTER(_Params), d, _dp, _ip, _dp]),
        "orc_nlevels": (i, [vp]),
        "orc_level_cells": (i, [vp, i]),
        "orc_level_nnz": (i, [vp, i]),
        "orc_level_ncolours": (i, [vp, i]),
        "orc_singular": (i, [vp]),
        "orc_level_csr": (None, [vp, i, _ip, _ip, _dp]),
        "orc_level_agg": (None, [vp, i, _ip]),
        "orc_level_colours": (None, [vp, i, _ip]),
        "orc_level_graph_nnz": (i, [vp, i]),
        "orc_level_graph": (None, [vp, i, _ip, _ip, _ip]),
        "orc_apply": (None, [vp, i, _dp, _dp]),
        "orc_smooth": (None, [vp, i, _dp, _dp, i]),
        "orc_vcycle": (None, [vp, _dp, _dp]),
        "orc_vcycle_level": (None, [vp, i, _dp, _dp]),
        "orc_coarse_solve": (None, [vp, _dp]),
        "orc_kinner": (None, [vp, i, _dp, _dp]),
        "orc_aggregate_graph": (i, [i, _ip, _ip, _ip, i, u32, _ip]),
        "orc_matching_pass": (i, [i, _ip, _ip, _ip, i, u32, i, _ip]),
        "orc_colour_graph": (i, [i, _ip, _ip, u32, _ip]),
        "orc_edge_hash": (u32, [u32, u32, u32]),
        "orc_operator_apply": (None, [i, i, i, d, d, d, _dp, _dp, _dp]),
        "orc_grid_aggregates": (i, [i, i, i, i, u32, _ip]),
        "orc_vertex_hash": (u32, [u32, u32]),
        "orc_step_guess": (i, [i, i, _dp, _dp, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _grid3(grid):
    g = tuple(int(v) for v in grid)
    while len(g) < 3:
        g = g + (1,)
    return g


def _soa(m, n):
    a = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(-1))
    if a.size != 3 * n:
        raise ValueError("expected 3*N values in component-major order")
    return a


class Hierarchy:
    """Oracle hierarchy for one time step: operator, aggregates, Galerkin
    levels, colourings and the coarsest LU."""

    def __init__(self, grid, h, alpha, dt, m_tilde, params: Params | None = None, adjoint: bool = False):
        """adjoint=True: the hierarchy of A^T (same aggregation, every level
        operator transposed), for adjoint solves."""
        self.grid = _grid3(grid)
        nx, ny, nz = self.grid
        self.n = nx * ny * nz
        self.h, self.alpha, self.dt = float(h), float(alpha), float(dt)
        self.params = params or Params()
        self._cp = self.params._c()
        lib = _load()
        setup = lib.orc_setup_adjoint if adjoint else lib.orc_setup
        self._h = setup(nx, ny, nz, self.h, self.alpha, self.dt, _soa(m_tilde, self.n), ctypes.byref(self._cp))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_free(self._h)
            self._h = None

    # -- structure -------------------------------------------------------
    @property
    def nlevels(self) -> int:
        return _lib.orc_nlevels(self._h)

    def cells(self, l: int) -> int:
        return _lib.orc_level_cells(self._h, l)

    def matrix(self, l: int) -> sp.csr_matrix:
        n3 = 3 * self.cells(l)
        nnz = _lib.orc_level_nnz(self._h, l)
        rp = np.zeros(n3 + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        va = np.zeros(nnz, np.float64)
        _lib.orc_level_csr(self._h, l, rp, ci, va)
        return sp.csr_matrix((va, ci, rp), shape=(n3, n3))

    def agg(self, l: int) -> np.ndarray:
        out = np.zeros(self.cells(l), np.int32)
        _lib.orc_level_agg(self._h, l, out)
        return out

    def colours(self, l: int) -> np.ndarray:
        out = np.zeros(self.cells(l), np.int32)
        _lib.orc_level_colours(self._h, l, out)
        return out

    def ncolours(self, l: int) -> int:
        return _lib.orc_level_ncolours(self._h, l)

    def graph(self, l: int):
        n = self.cells(l)
        nnz = _lib.orc_level_graph_nnz(self._h, l)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        w = np.zeros(nnz, np.int32)
        _lib.orc_level_graph(self._h, l, rp, ci, w)
        return rp, ci, w

    @property
    def singular(self) -> bool:
        return bool(_lib.orc_singular(self._h))

    # -- operations ------------------------------------------------------
    def apply(self, x, l: int = 0) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float64).reshape(-1)
        y = np.zeros_like(x)
        _lib.orc_apply(self._h, l, x, y)
        return y

    def smooth(self, b, x, forward: bool = True, l: int = 0) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64).reshape(-1)
        x = np.array(x, np.float64, copy=True).reshape(-1)
        _lib.orc_smooth(self._h, l, b, x, 1 if forward else 0)
        return x

    def vcycle(self, r, l: int = 0) -> np.ndarray:
        r = np.ascontiguousarray(r, np.float64).reshape(-1)
        z = np.zeros_like(r)
        _lib.orc_vcycle_level(self._h, l, r, z)
        return z

    def kinner(self, r, l: int) -> np.ndarray:
        """Two preconditioned GCR steps on level l from zero (K-cycle)."""
        r = np.ascontiguousarray(r, np.float64).reshape(-1)
        e = np.zeros_like(r)
        _lib.orc_kinner(self._h, l, r, e)
        return e

    def coarse_solve(self, b) -> np.ndarray:
        x = np.array(b, np.float64, copy=True).reshape(-1)
        _lib.orc_coarse_solve(self._h, x)
        return x

    def solve(self, b, x0=None, rtol: float | None = None, history: bool = False):
        """GCR solve; returns (x, status, iterations, true relres[, history])."""
        b = np.ascontiguousarray(b, np.float64).reshape(-1)
        x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64, copy=True).reshape(-1)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        hist = np.full(self.params.maxit + 1, np.nan) if history else None
        st = _lib.orc_solve(self._h, b, x, self.params.rtol if rtol is None else float(rtol),
                            ctypes.byref(it), ctypes.byref(rr),
                            hist.ctypes.data_as(ctypes.c_void_p) if history else None)
        if history:
            return x, st, it.value, rr.value, hist[: it.value + 1]
        return x, st, it.value, rr.value


def step(m, n_steps, grid, h, alpha, dt, params: Params | None = None, project: bool = True):
    """n_steps semi-implicit steps; returns (m, iterations per step, relres per step, status)."""
    params = params or Params()
    nx, ny, nz = _grid3(grid)
    mm = np.array(m, np.float64, copy=True).reshape(-1)
    its = np.zeros(max(n_steps, 1), np.int32)
    rrs = np.zeros(max(n_steps, 1), np.float64)
    cp = params._c()
    st = _load().orc_step(mm, int(n_steps), nx, ny, nz, float(h), float(alpha), float(dt),
                          ctypes.byref(cp), 1 if project else 0, its, rrs)
    return mm, its[:n_steps], rrs[:n_steps], st


def step_guess(m, prev):
    """The initial approximation of a step's solve from m = m^n and the
    earlier states prev (newest first, at most 6): returns (guess, order)."""
    mm = np.ascontiguousarray(np.asarray(m, np.float64).reshape(-1))
    d = len(prev)
    pp = np.ascontiguousarray(np.stack([np.asarray(p, np.float64).reshape(-1) for p in prev])
                              if d else np.zeros(1)).reshape(-1)
    x = np.zeros_like(mm)
    k = _load().orc_step_guess(mm.size, d, mm, pp, x)
    if k < 0:
        raise ValueError("at most 6 earlier states")
    return x, k


def step_vjp(m, x, g, grid, h, alpha, dt, params: Params | None = None):
    """Vector-Jacobian product of one step m -> x/|x| (A(m) x = m/dt):
    returns (dL/dm, dL/dalpha, status, adjoint iterations, relres) for
    g = dL/dm^{n+1} and the step's solution x."""
    params = params or Params()
    nx, ny, nz = _grid3(grid)
    n = nx * ny * nz
    mbar = np.zeros(3 * n)
    abar = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    cp = params._c()
    st = _load().orc_step_vjp(nx, ny, nz, float(h), float(alpha), float(dt), ctypes.byref(cp), _soa(m, n),
                              _soa(x, n), _soa(g, n), mbar, ctypes.byref(abar), ctypes.byref(it),
                              ctypes.byref(rr))
    return mbar, abar.value, st, it.value, rr.value


def forward_states(m0, n_steps, grid, h, alpha, dt, params: Params | None = None):
    """n_steps plain steps from m0 keeping every state and every solution x:
    returns (ms, xs) with ms[0] = m0, ms[k+1] = xs[k]/|xs[k]|."""
    params = params or Params()
    nx, ny, nz = _grid3(grid)
    n = nx * ny * nz
    ms = [np.array(m0, np.float64).reshape(-1)]
    xs = []
    for _ in range(n_steps):
        H = Hierarchy(grid, h, alpha, dt, ms[-1], params)
        b = ms[-1] / dt
        x, st, it, rr = H.solve(b, ms[-1].copy())
        xs.append(x)
        v = x.reshape(3, n)
        ms.append((v / np.sqrt(np.sum(v * v, axis=0))).reshape(-1))
    return ms, xs


def loss_gradient(m0, m_target, n_steps, grid, h, alpha, dt, params: Params | None = None):
    """L = 0.5 |m^N - m_target|^2 after n_steps steps, and its gradients with
    respect to m0 and alpha by the adjoint recursion (step_vjp backwards)."""
    ms, xs = forward_states(m0, n_steps, grid, h, alpha, dt, params)
    diff = ms[-1] - np.asarray(m_target, np.float64).reshape(-1)
    loss = 0.5 * float(diff @ diff)
    g = diff.copy()
    abar = 0.0
    for k in range(n_steps - 1, -1, -1):
        g, a, st, it, rr = step_vjp(ms[k], xs[k], g, grid, h, alpha, dt, params)
        abar += a
    return loss, g, abar


def step_llg(m, n_steps, grid, h, alpha, dt, q=0.0, he=(0.0, 0.0, 0.0), params: Params | None = None):
    """Steps of the full model with explicit anisotropy and external field
    (eps folded into h); returns (m, iterations, relres, status)."""
    params = params or Params()
    nx, ny, nz = _grid3(grid)
    mm = np.array(m, np.float64, copy=True).reshape(-1)
    its = np.zeros(max(n_steps, 1), np.int32)
    rrs = np.zeros(max(n_steps, 1), np.float64)
    cp = params._c()
    st = _load().orc_step_llg(mm, int(n_steps), nx, ny, nz, float(h), float(alpha), float(dt), ctypes.byref(cp),
                              float(q), np.asarray(he, np.float64), its, rrs)
    return mm, its[:n_steps], rrs[:n_steps], st


def aggregate_graph(rowptr, col, w, rounds: int = 32, seed: int = 0):
    """Aggregation (two matching passes) of an arbitrary weighted graph."""
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.int32)
    n = rowptr.size - 1
    agg = np.zeros(max(n, 1), np.int32)
    nc = _load().orc_aggregate_graph(n, rowptr, col, w, rounds, seed & 0xFFFFFFFF, agg)
    return agg[:n], nc


def matching_pass(rowptr, col, w, rounds: int = 32, seed: int = 0, attach: bool = False):
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.int32)
    n = rowptr.size - 1
    grp = np.zeros(max(n, 1), np.int32)
    ng = _load().orc_matching_pass(n, rowptr, col, w, rounds, seed & 0xFFFFFFFF, 1 if attach else 0, grp)
    return grp[:n], ng


def colour_graph(rowptr, col, seed: int = 0):
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    n = rowptr.size - 1
    c = np.zeros(max(n, 1), np.int32)
    nc = _load().orc_colour_graph(n, rowptr, col, seed & 0xFFFFFFFF, c)
    return c[:n], nc


def operator_apply(grid, h, alpha, dt, m, x):
    """y = A x for the operator alone (assembled CSR, no hierarchy)."""
    nx, ny, nz = _grid3(grid)
    n = nx * ny * nz
    y = np.zeros(3 * n)
    _load().orc_operator_apply(nx, ny, nz, float(h), float(alpha), float(dt), _soa(m, n), _soa(x, n), y)
    return y


def grid_aggregates(grid, rounds: int = 32, seed: int = 0):
    """Level-0 aggregates of the grid graph (natural cell order)."""
    nx, ny, nz = _grid3(grid)
    agg = np.zeros(nx * ny * nz, np.int32)
    nc = _load().orc_grid_aggregates(nx, ny, nz, rounds, seed & 0xFFFFFFFF, agg)
    return agg, nc


def edge_hash(a: int, b: int, seed: int = 0) -> int:
    return int(_load().orc_edge_hash(a, b, seed & 0xFFFFFFFF))


def vertex_hash(v: int, seed: int = 0) -> int:
    return int(_load().orc_vertex_hash(v, seed & 0xFFFFFFFF))
