"""Parity with the FP64 oracle where the dominant kernels run, through the
C ABI.

The small grids of ``test_gpu_parity.py`` put every coarse level inside the
cluster tail.  Here the grids are large enough that the per-class coarse
kernels run: at 48^3 levels 1 and 2 (27,598 and 6,842 cells) are above the
tail's limit of 5,000 cells and their colour classes take 8 lanes per row,
and the tail runs levels 3-4 on the whole cluster; at 128^3 levels 1-4 run
per class and the level-1 classes (over 20,000 rows each) take 4 lanes per
row.  Tolerances
as in ``test_gpu_parity.py``: single sweeps to 1e-12 of the largest entry, a
V-cycle to 1e-11 relative, float64 solves to 1e-10 relative of the oracle's,
mixed-precision solves to 1e-8 of the oracle's.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2608_09102_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2608_09102_b300 as ll  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _cm_to_aos(v, n):
    return np.ascontiguousarray(np.asarray(v).reshape(3, n).T).reshape(-1)


def _aos_to_cm(v, n):
    return np.ascontiguousarray(np.asarray(v).reshape(n, 3).T).reshape(-1)


def _vortex_case(side, kcycle=0, precision=ll.LL_FP64, rtol=1e-12):
    grid = (side,) * 3
    h, alpha = 1.0 / side, 0.02
    dt = 8.19 * h * h  # the time-stepping workload's dt/h^2
    m = inputs.vortex(*grid, seed=0).reshape(-1)
    O = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=rtol, kcycle=kcycle))
    G = ll.Hierarchy(_t(m), alpha, dt, h, grid, ll.Params(rtol=rtol, kcycle=kcycle, precision=precision))
    return grid, h, alpha, dt, m, O, G


@pytest.fixture(scope="module")
def case48():
    return _vortex_case(48)


@pytest.fixture(scope="module")
def case128():
    return _vortex_case(128)


def _check_coarse_sweeps(O, G, levels):
    rng = np.random.default_rng(6)
    for l in levels:
        n = O.cells(l)
        b, x = rng.standard_normal(3 * n), rng.standard_normal(3 * n)
        for fwd in (True, False):
            xg = torch.tensor(_cm_to_aos(x, n), device=DEV)
            G.smooth(l, torch.tensor(_cm_to_aos(b, n), device=DEV), xg, fwd)
            ref = O.smooth(b, x, fwd, l=l)
            err = np.abs(_aos_to_cm(_np(xg), n) - ref).max() / np.abs(ref).max()
            assert err <= 1e-12, (l, fwd, err)


def test_48cube_hierarchy_and_per_class_sweeps(case48):
    grid, h, alpha, dt, m, O, G = case48
    assert G.levels == O.nlevels
    assert O.cells(1) > 5000  # level 1 runs per colour class, outside the tail
    for l in range(O.nlevels - 1):
        assert np.array_equal(G.aggregates(l), O.agg(l))
        assert np.array_equal(G.colours(l + 1), O.colours(l + 1))
    _check_coarse_sweeps(O, G, [1, 2])


def test_48cube_vcycle(case48):
    grid, h, alpha, dt, m, O, G = case48
    r = inputs.rhs_field(*grid, seed=8).reshape(-1)
    z = torch.empty_like(_t(r))
    G.vcycle(_t(r), z)
    ref = O.vcycle(r)
    assert np.linalg.norm(_np(z) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("nu", [(2, 2), (2, 1), (1, 2), (0, 1), (1, 0)])
def test_48cube_vcycle_sweep_counts(nu):
    """Other smoothing counts take other kernels on level 0 (the full
    residual with the restriction after two forward sweeps, the restriction
    of b alone without pre-sweeps, the prolongation alone without
    post-sweeps) and on the per-class and tail levels."""
    grid = (48,) * 3
    h, alpha = 1.0 / 48, 0.02
    dt = 8.19 * h * h
    m = inputs.vortex(*grid, seed=0).reshape(-1)
    O = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-12, nu_pre=nu[0], nu_post=nu[1]))
    G = ll.Hierarchy(_t(m), alpha, dt, h, grid, ll.Params(rtol=1e-12, nu_pre=nu[0], nu_post=nu[1]))
    r = inputs.rhs_field(*grid, seed=8).reshape(-1)
    z = torch.empty_like(_t(r))
    G.vcycle(_t(r), z)
    ref = O.vcycle(r)
    assert np.linalg.norm(_np(z) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_48cube_kcycle_preconditioner():
    grid, h, alpha, dt, m, O, G = _vortex_case(48, kcycle=1)
    r = inputs.rhs_field(*grid, seed=8).reshape(-1)
    z = torch.empty_like(_t(r))
    G.vcycle(_t(r), z)
    ref = O.vcycle(r)
    assert np.linalg.norm(_np(z) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_48cube_solve(case48):
    grid, h, alpha, dt, m, O, G = case48
    b = m / dt
    xo, sto, ito, rro = O.solve(b, np.zeros_like(b))
    x = torch.zeros(b.size, dtype=torch.float64, device=DEV)
    st, it, rr = G.solve(_t(b), x)
    assert st == ll.LL_OK and sto == oracle.OK and rr < 1e-12
    assert abs(it - ito) <= 1, (it, ito)
    assert np.linalg.norm(_np(x) - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("precision", [ll.LL_MIXED_FP32, ll.LL_MIXED_BF16])
def test_48cube_mixed_solution_against_oracle(case48, precision):
    """float32 / bfloat16 V-cycle inside float64 GCR to rtol 1e-10: within
    1e-8 of the oracle's float64 solution."""
    grid, h, alpha, dt, m, O, G = case48
    b = m / dt
    xo, sto, ito, rro = O.solve(b, np.zeros_like(b))
    Gm = ll.Hierarchy(_t(m), alpha, dt, h, grid, ll.Params(rtol=1e-10, precision=precision))
    x = torch.zeros(b.size, dtype=torch.float64, device=DEV)
    st, it, rr = Gm.solve(_t(b), x)
    assert st == ll.LL_OK and rr < 1e-10
    assert np.linalg.norm(_np(x) - xo) <= 1e-8 * np.linalg.norm(xo)


def test_128cube_per_class_sweeps_and_vcycle(case128):
    """The time-stepping workload's hierarchy: the level-1 classes take the
    4-lane path, levels 2-4 the 8-lane path; one V-cycle through all of them
    and the cluster tail."""
    grid, h, alpha, dt, m, O, G = case128
    assert G.levels == O.nlevels
    assert O.cells(1) > 20000 * 4  # several level-1 classes above the 4-lane threshold
    for l in range(1, 5):
        assert np.array_equal(G.colours(l), O.colours(l))
    _check_coarse_sweeps(O, G, [1, 2, 3, 4])
    r = inputs.rhs_field(*grid, seed=8).reshape(-1)
    z = torch.empty_like(_t(r))
    G.vcycle(_t(r), z)
    ref = O.vcycle(r)
    assert np.linalg.norm(_np(z) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_128cube_ordered_galerkin_levels(case128):
    """Levels 2 and 3 of the 128^3 hierarchy (over 200,000 blocks each) are
    built with the Galerkin threads in slot-list-length order: every block
    within 1e-12 of the oracle's P^T A P (compared as sparse matrices)."""
    import scipy.sparse as sp

    grid, h, alpha, dt, m, O, G = case128
    for l in (2, 3):
        n = O.cells(l)
        rp, ci, val = G.operator(l)
        assert rp[-1] >= 200000, (l, rp[-1])
        bsr = sp.bsr_matrix((val, ci, rp), shape=(3 * n, 3 * n)).tocsr()
        perm = np.array([3 * I + c for c in range(3) for I in range(n)])  # component-major -> cell-major
        mine = bsr[perm][:, perm]
        ref = O.matrix(l).tocsr()
        diff = (mine - ref).tocsr()
        scale = np.abs(ref.data).max()
        assert (np.abs(diff.data).max() if diff.nnz else 0.0) <= 1e-12 * scale, l


def test_graphs_equal_eager_iterations():
    """GCR iterations replayed from their CUDA graphs give bit for bit the
    iterates, counts and residuals of eager launches (no graphs) and of the
    graphs with kernel timing (event nodes) on.  Restart 4 with a short last
    cycle: maxit 7 stops inside the second cycle."""
    import ctypes
    import os

    grid, h, alpha, dt = (32, 32, 32), 1 / 32, 0.02, 8.19 / 32 ** 2
    m = inputs.vortex(*grid, seed=0).reshape(-1)
    b = _t(m / dt)
    out = {}
    for maxit in (1000, 7):
        p = ll.Params(rtol=1e-10, restart=4, maxit=maxit)
        for mode in ("graphs", "eager", "timed"):
            if mode == "eager":
                os.environ["LLMG_NO_GRAPHS"] = "1"
            try:
                G = ll.Hierarchy(_t(m), alpha, dt, h, grid, p)
            finally:
                os.environ.pop("LLMG_NO_GRAPHS", None)
            if mode == "timed":
                ll.load_library().ll_mg_profile(G._h, ctypes.c_uint(0xFFFF))
            x = torch.zeros_like(b)
            st, it, rr = G.solve(b, x)
            out[(maxit, mode)] = (st, it, rr, x)
        ref = out[(maxit, "graphs")]
        for mode in ("eager", "timed"):
            st, it, rr, x = out[(maxit, mode)]
            assert (st, it, rr) == ref[:3], (maxit, mode)
            assert torch.equal(x, ref[3]), (maxit, mode)
    assert out[(1000, "graphs")][0] == ll.LL_OK and out[(1000, "graphs")][1] > 8
    assert out[(7, "graphs")][0] == ll.LL_NOT_CONVERGED and out[(7, "graphs")][1] == 7


def test_iteration_counts_stay_bounded_under_refinement():
    """Mesh independence on the GPU (3-D, dt/h^2 = 8.19, alpha = 0.02):
    32^3 -> 128^3 grows the iteration count by at most 30 %."""
    its = []
    for side in (32, 64, 128):
        grid = (side,) * 3
        h = 1.0 / side
        dt = 8.19 * h * h
        m = inputs.vortex(*grid, seed=0).reshape(-1)
        G = ll.Hierarchy(_t(m), 0.02, dt, h, grid, ll.Params(rtol=1e-8))
        x = _t(m)
        st, it, rr = G.solve(_t(m / dt), x)
        assert st == ll.LL_OK
        its.append(it)
    assert max(its) <= 1.3 * its[0], its


def test_step_host_equals_device_steps():
    """ll_mg_step_host (a field in host memory, copied by the library) gives
    the same steps as ll_mg_step on a device field."""
    grid, h, alpha, dt = (24, 20, 8), 1 / 24, 0.05, 2e-3
    m0 = inputs.vortex(*grid, seed=0).reshape(-1)
    p = ll.Params(rtol=1e-10)
    md = _t(m0)
    Gd = ll.Hierarchy(md, alpha, dt, h, grid, p)
    std, itd, rrd = Gd.step(md, 2)
    mh = torch.tensor(m0).pin_memory()
    Gh = ll.Hierarchy(_t(m0), alpha, dt, h, grid, p)
    sth, ith, rrh = Gh.step_host(mh, 2)
    assert std == sth == ll.LL_OK and itd == ith
    assert torch.equal(mh, md.cpu())
    mp = torch.tensor(m0)  # pageable host memory works too
    Gp = ll.Hierarchy(_t(m0), alpha, dt, h, grid, p)
    Gp.step_host(mp, 2)
    assert torch.equal(mp, md.cpu())


def test_continued_integration_keeps_the_extrapolation_history():
    """Steps split over several calls equal the same steps in one call (the
    field passed in is the hierarchy's last output, so the history of earlier
    states carries over); a field that is not that output starts a fresh
    history, as a new hierarchy would.  Against the oracle's one-call steps."""
    grid, h, alpha, dt = (24, 20, 8), 1 / 24, 0.05, 2e-3
    m0 = inputs.vortex(*grid, seed=0).reshape(-1)
    p = ll.Params(rtol=1e-12)
    ma = _t(m0)
    Ga = ll.Hierarchy(ma, alpha, dt, h, grid, p)
    sa, ita, _ = Ga.step(ma, 6)
    mb = _t(m0)
    Gb = ll.Hierarchy(mb, alpha, dt, h, grid, p)
    itb = []
    for k in (1, 2, 3):
        st, its, _ = Gb.step(mb, k)
        itb += its
    assert torch.equal(ma, mb) and ita == itb
    mo, ito, rro, sto = oracle.step(m0, 6, grid, h, alpha, dt, oracle.Params(rtol=1e-12))
    assert np.abs(_np(ma) - mo).max() <= 1e-10
    assert all(abs(a - b) <= 1 for a, b in zip(ita, ito)), (ita, ito)
    # a field that is not the last output: no history (as on a fresh hierarchy)
    mc = _t(m0)
    st, itc, _ = Gb.step(mc, 2)
    md = _t(m0)
    Gd = ll.Hierarchy(md, alpha, dt, h, grid, p)
    st, itd, _ = Gd.step(md, 2)
    assert torch.equal(mc, md) and itc == itd
    # another dt through ll_mg_update: the kept states are dropped, so the
    # next steps equal those of a fresh hierarchy with the new dt
    Gd.update(md, alpha, 2 * dt)
    me = md.clone()
    st, ite, _ = Gd.step(md, 3)
    Ge = ll.Hierarchy(me, alpha, 2 * dt, h, grid, p)
    st, itf, _ = Ge.step(me, 3)
    assert torch.equal(md, me) and ite == itf


def test_fp64_probe_runs():
    sink = torch.zeros(1, dtype=torch.float64, device=DEV)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fl = ll.fp64_fma_probe(sink, 4096, 148 * 4)
    e1.record()
    torch.cuda.synchronize()
    assert fl == 2.0 * 8 * 4096 * 148 * 4 * 256
    tflops = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
    assert 0.05 < tflops < 5.0, tflops
    assert float(sink[0]) == 0.0
