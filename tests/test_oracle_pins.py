"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the
paper's component form (Sec. 2.1), textbook Neumann Laplacians, the DCT
closed form for a constant field, dense direct solves, the Galerkin
identity (Eq. galerkin / Eq. Ac_direct) by an independent sparse product,
the GCR identity r_m = b - A u_m (Sec. 3.1.2), first-order convergence in
time on a manufactured solution, and an independent restatement of the
aggregation rule.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2608_09102_b300 import inputs
from tests import aggregation_bruteforce as bf
from tests import reference_forms as rf


def _rand_m(n, seed, unit=False):
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((3, n))
    if unit:
        m /= np.linalg.norm(m, axis=0)
    return m.reshape(-1)


# --------------------------------------------------------------------------
# operator (Sec. 2.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("grid", [(3, 3, 3), (4, 3, 1), (5, 1, 1), (2, 3, 2)])
def test_operator_matches_component_form(grid):
    nx, ny, nz = grid
    n = nx * ny * nz
    h, alpha, dt = 0.37, 0.3, 0.011
    m = _rand_m(n, 1)  # deliberately not unit length
    H = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(coarsest_cells=10 ** 6))
    A = H.matrix(0).toarray()
    ref = rf.operator_dense(nx, ny, nz, h, alpha, dt, m)
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_constant_vectors_see_only_the_mass_term():
    """Delta_h c = 0 under Neumann conditions, so A c = c/dt for any m~."""
    grid = (6, 5, 4)
    n = 120
    H = oracle.Hierarchy(grid, 0.1, 0.05, 1e-3, _rand_m(n, 2, unit=True), oracle.Params())
    c = np.repeat(np.array([0.3, -1.2, 2.0]), n)
    np.testing.assert_allclose(H.apply(c), c / 1e-3, rtol=1e-12)


def test_pointwise_orthogonality_of_the_solution():
    """m_k^T C(m_k) = 0, so m_k.(A x)_k = m_k.x_k/dt: with b = m/dt the
    solution satisfies m_k.x_k - 1 = -dt m_k.r_k in every cell."""
    grid = (24, 24, 1)
    n = 576
    h, alpha, dt = 1 / 24, 0.1, 2e-3
    m = inputs.smooth_field(24, 24, 1, seed=3).reshape(-1)
    H = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-9))
    b = m / dt
    x, st, it, rr = H.solve(b, np.zeros_like(b))
    assert st == oracle.OK and rr < 1e-9
    r = b - H.apply(x)
    mx = (m.reshape(3, n) * x.reshape(3, n)).sum(0)
    mr = (m.reshape(3, n) * r.reshape(3, n)).sum(0)
    np.testing.assert_allclose(mx - 1.0, -dt * mr, rtol=0, atol=1e-12)
    assert np.all(np.linalg.norm(x.reshape(3, n), axis=0) >= 1.0 - 1e-7)


# --------------------------------------------------------------------------
# whole solve against exact solutions
# --------------------------------------------------------------------------

@pytest.mark.parametrize("grid,mdir,alpha", [((32, 32, 1), (0, 0, 1), 0.1),
                                             ((12, 10, 8), (0.3, -0.4, 0.8), 0.02),
                                             ((40, 1, 1), (1, 2, 2), 1.0)])
def test_solve_matches_dct_closed_form(grid, mdir, alpha):
    nx, ny, nz = grid
    n = nx * ny * nz
    h, dt = 1.0 / nx, 4.0 / nx ** 2
    m = inputs.constant_field(nx, ny, nz, mdir).reshape(-1)
    b = inputs.rhs_field(nx, ny, nz, seed=5).reshape(-1)
    H = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-13, coarsest_cells=8))
    x, st, it, rr = H.solve(b)
    assert st == oracle.OK
    xe = rf.dct_solve(nx, ny, nz, h, alpha, dt, mdir, b)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)


@pytest.mark.parametrize("grid,alpha,seed", [((4, 4, 2), 0.3, 0), ((6, 5, 1), 0.02, 1), ((7, 1, 1), 1.0, 2)])
def test_solve_matches_dense_direct(grid, alpha, seed):
    nx, ny, nz = grid
    n = nx * ny * nz
    h, dt = 1.0 / nx, 2.0 / nx ** 2
    m = _rand_m(n, seed, unit=True)
    b = np.random.default_rng(seed + 7).standard_normal(3 * n)
    H = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-14, coarsest_cells=2))
    assert H.nlevels >= 2
    x, st, it, rr = H.solve(b)
    xe = np.linalg.solve(rf.operator_dense(nx, ny, nz, h, alpha, dt, m), b)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)


def test_constant_field_is_a_fixed_point():
    """For constant m~ = m^n the system returns x = m^n exactly (Sec. 4's
    trivial initial state): 0 iterations from the guess m^n."""
    nx = ny = 16
    m = inputs.trivial_state(nx, ny, 1).reshape(-1)
    dt = 1e-3
    H = oracle.Hierarchy((nx, ny, 1), 1 / nx, 0.01, dt, m, oracle.Params(rtol=1e-10))
    x, st, it, rr = H.solve(m / dt, m)
    assert st == oracle.OK and it == 0 and rr < 1e-14
    x0, st0, it0, rr0 = H.solve(m / dt)
    assert st0 == oracle.OK and it0 <= 3
    np.testing.assert_allclose(x0, m, atol=1e-9)


# --------------------------------------------------------------------------
# Galerkin (Eq. galerkin, Eq. Ac_direct) and aggregation (Eq. Pagg)
# --------------------------------------------------------------------------

def _boolean_p(agg, nc):
    n = agg.size
    p = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
    return sp.kron(sp.eye(3), p).tocsr()  # component-major at both levels


@pytest.mark.parametrize("grid", [(12, 10, 1), (6, 6, 5)])
def test_galerkin_equals_independent_product(grid):
    nx, ny, nz = grid
    n = nx * ny * nz
    m = _rand_m(n, 4, unit=True)
    H = oracle.Hierarchy(grid, 0.2, 0.07, 1e-2, m, oracle.Params(coarsest_cells=4))
    assert H.nlevels >= 3
    for l in range(H.nlevels - 1):
        A = H.matrix(l)
        P = _boolean_p(H.agg(l), H.cells(l + 1))
        Ac = (P.T @ A @ P).toarray()
        got = H.matrix(l + 1).toarray()
        np.testing.assert_allclose(got, Ac, rtol=0, atol=1e-12 * np.abs(Ac).max())


def test_galerkin_entrywise_double_sum_on_tiny_grid():
    """(A_c)_ij = sum_{k in G_i} sum_{l in G_j} a_kl, evaluated by brute force."""
    grid = (4, 4, 1)
    n = 16
    m = _rand_m(n, 9)
    H = oracle.Hierarchy(grid, 0.5, 0.2, 0.1, m, oracle.Params(coarsest_cells=2))
    A = rf.operator_dense(4, 4, 1, 0.5, 0.2, 0.1, m)
    agg = H.agg(0)
    nc = H.cells(1)
    ref = np.zeros((3 * nc, 3 * nc))
    for c in range(3):
        for k in range(n):
            for c2 in range(3):
                for l in range(n):
                    ref[c * nc + agg[k], c2 * nc + agg[l]] += A[c * n + k, c2 * n + l]
    np.testing.assert_allclose(H.matrix(1).toarray(), ref, atol=1e-12 * np.abs(ref).max())


def test_galerkin_preserves_constants():
    """A_l (1 (x) c) = |G_I| c/dt: constants see only the mass term on every
    level, |G_I| the number of grid cells in the composite aggregate."""
    grid = (10, 9, 7)
    n = 630
    dt = 3e-3
    H = oracle.Hierarchy(grid, 0.1, 0.3, dt, _rand_m(n, 11, unit=True), oracle.Params(coarsest_cells=4))
    comp = np.arange(n)
    for l in range(H.nlevels):
        nl = H.cells(l)
        size = np.bincount(comp, minlength=nl).astype(float)
        c = np.array([1.5, -0.5, 0.25])
        v = np.repeat(c, nl)
        np.testing.assert_allclose(H.apply(v, l), np.kron(c, size) / dt, rtol=1e-10)
        if l < H.nlevels - 1:
            comp = H.agg(l)[comp]


@pytest.mark.parametrize("grid", [(64, 64, 1), (16, 16, 16), (200, 1, 1)])
def test_aggregates_partition_and_coarsen_by_about_four(grid):
    nx, ny, nz = grid
    n = nx * ny * nz
    H = oracle.Hierarchy(grid, 1 / nx, 0.1, 1e-3, inputs.smooth_field(nx, ny, nz).reshape(-1),
                         oracle.Params(coarsest_cells=64))
    for l in range(H.nlevels - 1):
        agg = H.agg(l)
        nl, nc = H.cells(l), H.cells(l + 1)
        assert agg.min() == 0 and agg.max() == nc - 1
        sizes = np.bincount(agg, minlength=nc)
        assert sizes.min() >= 1
        # numbering = rank of the smallest member
        first = np.full(nc, nl)
        np.minimum.at(first, agg, np.arange(nl))
        assert np.all(np.diff(first) > 0)
        if l == 0:
            assert 2.5 < nl / nc <= 4.6, (l, nl, nc)


def _grid_adj(nx, ny, nz):
    H = oracle.Hierarchy((nx, ny, nz), 1.0, 0.1, 1.0, inputs.constant_field(nx, ny, nz).reshape(-1),
                         oracle.Params(coarsest_cells=10 ** 6))
    return H.graph(0)


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_aggregation_equals_independent_restatement(seed):
    rng = np.random.default_rng(seed)
    graphs = [_grid_adj(9, 7, 1), _grid_adj(4, 4, 4)]
    # a random symmetric weighted graph
    n = 60
    W = np.zeros((n, n), np.int32)
    for _ in range(180):
        i, j = rng.integers(0, n, 2)
        if i != j:
            W[i, j] = W[j, i] = rng.integers(1, 9)
    S = sp.csr_matrix(W)
    S.sort_indices()
    graphs.append((S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.int32)))
    # and a coarse level of a real hierarchy (weights > 1)
    H = oracle.Hierarchy((12, 12, 6), 0.1, 0.1, 1e-3, inputs.smooth_field(12, 12, 6).reshape(-1),
                         oracle.Params(coarsest_cells=8, seed=seed))
    graphs.append(H.graph(1))
    for rp, ci, w in graphs:
        adj = bf.to_adj(rp, ci, w)
        got, nc = oracle.aggregate_graph(rp, ci, w, seed=seed)
        ref, nref = bf.aggregate(adj, seed=seed)
        assert nc == nref
        assert got.tolist() == ref
        g1, n1 = oracle.matching_pass(rp, ci, w, seed=seed)
        r1, m1 = bf.matching_pass(adj, seed=seed)
        assert n1 == m1 and g1.tolist() == r1
        col, _ = oracle.colour_graph(rp, ci, seed=seed)
        assert col.tolist() == bf.colour(adj, seed=seed)


def test_round_cap_is_respected():
    rp, ci, w = _grid_adj(16, 16, 1)
    adj = bf.to_adj(rp, ci, w)
    for R in (1, 2, 3):
        got, nc = oracle.matching_pass(rp, ci, w, rounds=R)
        ref, nref = bf.matching_pass(adj, rounds=R)
        assert got.tolist() == ref
    one, n_one = oracle.matching_pass(rp, ci, w, rounds=1)
    full, n_full = oracle.matching_pass(rp, ci, w, rounds=32)
    assert n_full < n_one


def test_hash_functions_match_restatement():
    for a, b, s in [(0, 1, 0), (7, 12345, 3), (2 ** 20, 2 ** 30 + 5, 0xDEADBEEF)]:
        assert oracle.edge_hash(a, b, s) == bf.edge_hash(a, b, s)
        assert oracle.vertex_hash(a, s) == bf.vertex_hash(a, s)
    assert bf.fmix32(0) == 0


def test_colourings_are_proper():
    grid = (20, 20, 1)
    H = oracle.Hierarchy(grid, 0.05, 0.1, 1e-3, inputs.smooth_field(20, 20, 1).reshape(-1),
                         oracle.Params(coarsest_cells=4))
    c0 = H.colours(0).reshape(20, 20)
    yy, xx = np.mgrid[0:20, 0:20]
    assert np.array_equal(c0, (xx + yy) % 2)
    for l in range(H.nlevels):
        rp, ci, _ = H.graph(l)
        col = H.colours(l)
        for i in range(H.cells(l)):
            for p in range(rp[i], rp[i + 1]):
                assert col[i] != col[ci[p]]


# --------------------------------------------------------------------------
# smoother, coarse solve, V-cycle
# --------------------------------------------------------------------------

def test_gauss_seidel_fixed_point_and_convergence():
    grid = (8, 6, 1)
    n = 48
    m = _rand_m(n, 13, unit=True)
    H = oracle.Hierarchy(grid, 1.0, 0.5, 0.05, m, oracle.Params(coarsest_cells=2))
    A = rf.operator_dense(8, 6, 1, 1.0, 0.5, 0.05, m)
    b = np.random.default_rng(3).standard_normal(3 * n)
    xe = np.linalg.solve(A, b)
    for fwd in (True, False):
        np.testing.assert_allclose(H.smooth(b, xe, fwd), xe, rtol=0, atol=1e-12 * np.abs(xe).max())
    x = np.zeros(3 * n)
    for _ in range(60):
        x = H.smooth(b, x, True)
    assert np.linalg.norm(x - xe) < 1e-8 * np.linalg.norm(xe)


def test_gauss_seidel_on_coarse_level_converges():
    grid = (10, 10, 1)
    H = oracle.Hierarchy(grid, 0.1, 0.3, 1e-2, _rand_m(100, 14, unit=True), oracle.Params(coarsest_cells=4))
    A1 = H.matrix(1).toarray()
    b = np.random.default_rng(5).standard_normal(A1.shape[0])
    xe = np.linalg.solve(A1, b)
    np.testing.assert_allclose(H.smooth(b, xe, True, l=1), xe, atol=1e-11 * np.abs(xe).max())
    x = np.zeros_like(b)
    for _ in range(200):
        x = H.smooth(b, x, True, l=1)
    assert np.linalg.norm(x - xe) < 1e-6 * np.linalg.norm(xe)


def test_coarsest_lu_is_exact():
    H = oracle.Hierarchy((16, 16, 1), 1 / 16, 0.1, 1e-3, inputs.smooth_field(16, 16, 1).reshape(-1),
                         oracle.Params(coarsest_cells=40))
    L = H.nlevels - 1
    Ac = H.matrix(L).toarray()
    b = np.random.default_rng(1).standard_normal(Ac.shape[0])
    np.testing.assert_allclose(H.coarse_solve(b), np.linalg.solve(Ac, b), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(H.vcycle(b, l=L), np.linalg.solve(Ac, b), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("grid,mdir,alpha", [((16, 16, 1), None, 0.1), ((8, 8, 1), (0, 0, 1), 0.02),
                                             ((6, 6, 6), (0.6, 0, 0.8), 0.1)])
def test_vcycle_contracts(grid, mdir, alpha):
    """Spectral radius of the V-cycle error propagation I - B A below one
    (constant fields, and a vortex resolved by the grid)."""
    nx, ny, nz = grid
    n = nx * ny * nz
    m = (inputs.vortex(nx, ny, nz) if mdir is None else inputs.constant_field(nx, ny, nz, mdir)).reshape(-1)
    H = oracle.Hierarchy(grid, 1 / nx, alpha, 8.0 / nx ** 2, m, oracle.Params(coarsest_cells=4))
    assert H.nlevels >= 3
    A = H.matrix(0).toarray()
    B = np.column_stack([H.vcycle(e) for e in np.eye(3 * n)])
    rho = np.abs(np.linalg.eigvals(np.eye(3 * n) - B @ A)).max()
    assert rho < 0.9


# --------------------------------------------------------------------------
# GCR (Algorithm 1)
# --------------------------------------------------------------------------

def test_gcr_recurrence_equals_true_residual():
    """r_m = b - A u_m (Sec. 3.1.2): stop after j iterations (no restart) and
    compare the recurrence residual with the true residual."""
    grid = (20, 20, 1)
    m = inputs.smooth_field(20, 20, 1, seed=2).reshape(-1)
    b = inputs.rhs_field(20, 20, 1, seed=2).reshape(-1)
    for j in (1, 3, 7):
        H = oracle.Hierarchy(grid, 0.05, 0.1, 1e-2, m, oracle.Params(maxit=j, restart=j, rtol=1e-30))
        x, st, it, rr, hist = H.solve(b, history=True)
        assert it == j and st == oracle.NOT_CONVERGED
        assert abs(hist[-1] - rr) <= 1e-9 * rr


def test_gcr_with_exact_preconditioner_takes_one_iteration():
    grid = (5, 4, 3)
    n = 60
    m = _rand_m(n, 21, unit=True)
    b = np.random.default_rng(2).standard_normal(3 * n)
    H = oracle.Hierarchy(grid, 0.3, 0.05, 0.02, m, oracle.Params(prec=2, rtol=1e-12))
    x, st, it, rr = H.solve(b)
    assert st == oracle.OK and it == 1 and rr < 1e-12


def test_unpreconditioned_gcr_reaches_dense_solution():
    grid = (6, 6, 1)
    m = _rand_m(36, 22, unit=True)
    b = np.random.default_rng(3).standard_normal(108)
    H = oracle.Hierarchy(grid, 1 / 6, 0.1, 0.05, m, oracle.Params(prec=1, rtol=1e-13, restart=200))
    x, st, it, rr = H.solve(b)
    xe = np.linalg.solve(rf.operator_dense(6, 6, 1, 1 / 6, 0.1, 0.05, m), b)
    assert st == oracle.OK and np.linalg.norm(x - xe) < 1e-10 * np.linalg.norm(xe)


def test_zero_rhs_and_breakdown_free_statuses():
    H = oracle.Hierarchy((8, 8, 1), 1 / 8, 0.1, 1e-2, inputs.smooth_field(8, 8, 1).reshape(-1), oracle.Params())
    x, st, it, rr = H.solve(np.zeros(192), np.ones(192))
    assert st == oracle.OK and it == 0 and np.all(x == 0)
    bad = np.full(192, np.nan)
    _, st2, _, _ = H.solve(bad)
    assert st2 == oracle.BREAKDOWN


# --------------------------------------------------------------------------
# iteration counts and time stepping (Sec. 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("grids", [[(n, n, 1) for n in (32, 64, 128, 256)],
                                   [(n, n, n) for n in (16, 32, 64)]], ids=["2d", "3d"])
def test_iteration_counts_stay_bounded_under_refinement(grids):
    """Mesh-independent convergence (the paper's claim for the aggregation
    solver, abstract and Tables 4-13): at fixed dt/h^2 = 8.19 the iteration
    count to 1e-8 grows by at most 30 % from the coarsest to the finest grid
    (2-D 32^2 -> 256^2, 3-D 16^3 -> 64^3; measured 26 -> 33 and 34 -> 42)."""
    its = []
    for g in grids:
        n = g[0]
        m = inputs.vortex(*g, seed=0).reshape(-1)
        dt = 8.19 / n ** 2
        H = oracle.Hierarchy(g, 1 / n, 0.02, dt, m, oracle.Params(rtol=1e-8))
        _, st, it, _ = H.solve(m / dt, m)
        assert st == oracle.OK
        its.append(it)
    assert max(its) <= 1.3 * its[0], its


def test_projection_leaves_iteration_counts_unchanged():
    """The paper observes that the projection m <- m/|m| does not change
    the iteration numbers."""
    n = 24
    m0 = inputs.smooth_field(n, n, 1, seed=4).reshape(-1)
    p = oracle.Params(rtol=1e-10)
    m1, it1, _, s1 = oracle.step(m0, 4, (n, n, 1), 1 / n, 0.01, 1e-3, p, project=True)
    m2, it2, _, s2 = oracle.step(m0, 4, (n, n, 1), 1 / n, 0.01, 1e-3, p, project=False)
    assert s1 == s2 == oracle.OK
    assert np.all(np.abs(it1 - it2) <= 2), (it1, it2)
    assert np.allclose(np.linalg.norm(m1.reshape(3, -1), axis=0), 1.0, atol=1e-14)


def test_first_order_convergence_in_time():
    """BDF1 with first-order extrapolation of m~: the error of a manufactured
    solution halves with dt (h fixed and fine)."""
    n, alpha, T = 48, 0.1, 0.2
    ms = rf.Manufactured(n, alpha)
    errs = []
    for nsteps in (10, 20, 40):
        dt = T / nsteps
        m = ms.m(0.0).reshape(-1)
        for s in range(nsteps):
            H = oracle.Hierarchy((n, n, 1), 1 / n, alpha, dt, m, oracle.Params(rtol=1e-12))
            b = m / dt + ms.forcing((s + 1) * dt).reshape(-1)
            m, st, it, rr = H.solve(b, m)
            assert st == oracle.OK
        errs.append(np.abs(m - ms.m(T).reshape(-1)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.7 < r1 < 2.3 and 1.7 < r2 < 2.3, errs


# --------------------------------------------------------------------------
# source terms of the full model (Sec. 2.1: anisotropy, external field)
# --------------------------------------------------------------------------

def _llg_rhs_uniform_step(m, dt, alpha, q, he):
    """A uniform field has Delta_h m = 0, so one step is the explicit update
    m - dt (m x f + alpha m x (m x f)), f = -q (0, m2, m3) + he, then the
    projection (cross products written out with numpy, independently of the
    oracle's 3x3 coefficient)."""
    f = np.array([he[0], he[1] - q * m[1], he[2] - q * m[2]])
    c1 = np.cross(m, f)
    v = m - dt * (c1 + alpha * np.cross(m, c1))
    return v / np.linalg.norm(v)


def test_source_terms_on_a_uniform_field_match_the_explicit_update():
    grid, h, alpha, dt, q, he = (6, 5, 4), 0.1, 0.3, 2e-2, 0.7, (0.2, -0.4, 0.5)
    d = np.array([0.3, 0.5, -0.8])
    d /= np.linalg.norm(d)
    m = inputs.constant_field(*grid, direction=d).reshape(-1)
    out, its, rrs, st = oracle.step_llg(m, 3, grid, h, alpha, dt, q, he, oracle.Params(rtol=1e-13))
    assert st == oracle.OK
    ref = d.copy()
    for _ in range(3):
        ref = _llg_rhs_uniform_step(ref, dt, alpha, q, he)
    np.testing.assert_allclose(out.reshape(3, -1), np.repeat(ref[:, None], 120, axis=1), atol=1e-12)


def test_damping_turns_the_field_towards_the_applied_field():
    """With alpha > 0 the term -alpha m x (m x h_e) pulls m towards h_e:
    the mean of m . h_e grows step by step."""
    n = 16
    m = inputs.smooth_field(n, n, 1, seed=6).reshape(-1)
    he = np.array([0.0, 0.0, 40.0])
    dots = []
    for _ in range(4):
        m, its, rrs, st = oracle.step_llg(m, 1, (n, n, 1), 1 / n, 0.5, 1e-3, 0.0, he, oracle.Params(rtol=1e-12))
        assert st == oracle.OK
        dots.append(float((m.reshape(3, -1).T @ he).mean()))
    assert all(b > a for a, b in zip(dots, dots[1:])), dots


def test_zero_sources_reduce_to_the_plain_step():
    n = 12
    m = inputs.vortex(n, n, 1, seed=1).reshape(-1)
    a, _, _, _ = oracle.step_llg(m, 2, (n, n, 1), 1 / n, 0.1, 1e-3, 0.0, (0, 0, 0), oracle.Params(rtol=1e-12))
    b, _, _, _ = oracle.step(m, 2, (n, n, 1), 1 / n, 0.1, 1e-3, oracle.Params(rtol=1e-12))
    np.testing.assert_allclose(a, b, atol=1e-13)


# --------------------------------------------------------------------------
# K-cycle (Krylov acceleration of the coarse levels, Sec. 3.1)
# --------------------------------------------------------------------------

def test_kcycle_inner_steps_minimise_the_residual():
    """Two GCR steps return the e in span{z1, z2} (z1 = B r, z2 = B r1) that
    minimises |r - A e|: checked by an independent least-squares solve."""
    grid = (20, 18, 1)
    m = inputs.vortex(*grid, seed=2).reshape(-1)
    H = oracle.Hierarchy(grid, 1 / 20, 0.1, 2e-3, m, oracle.Params(coarsest_cells=8, kcycle=1))
    assert H.nlevels >= 3
    A = H.matrix(1)
    r = np.random.default_rng(4).standard_normal(A.shape[0])
    e = H.kinner(r, 1)
    z1 = H.vcycle(r, l=1)
    Az1 = A @ z1
    a1 = (Az1 @ r) / (Az1 @ Az1)
    r1 = r - a1 * Az1
    z2 = H.vcycle(r1, l=1)
    Z = np.column_stack([z1, z2])
    y, *_ = np.linalg.lstsq(A @ Z, r, rcond=None)
    np.testing.assert_allclose(e, Z @ y, rtol=0, atol=1e-10 * np.abs(Z @ y).max())


@pytest.mark.parametrize("kcycle", [1, 3])
def test_kcycle_solve_matches_dct_closed_form(kcycle):
    grid, mdir, alpha = (24, 20, 12), (0.3, -0.4, 0.8), 0.05
    nx, ny, nz = grid
    h, dt = 1.0 / nx, 6.0 / nx ** 2
    m = inputs.constant_field(*grid, mdir).reshape(-1)
    b = inputs.rhs_field(*grid, seed=7).reshape(-1)
    H = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-13, coarsest_cells=8, kcycle=kcycle))
    x, st, it, rr = H.solve(b)
    assert st == oracle.OK
    xe = rf.dct_solve(nx, ny, nz, h, alpha, dt, mdir, b)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)


def test_kcycle_reduces_iterations():
    grid = (24, 24, 24)
    m = inputs.vortex(*grid, seed=0).reshape(-1)
    dt = 8.19 / 24 ** 2
    its = []
    for k in (0, 2):
        H = oracle.Hierarchy(grid, 1 / 24, 0.02, dt, m, oracle.Params(kcycle=k))
        _, st, it, _ = H.solve(m / dt, m)
        assert st == oracle.OK
        its.append(it)
    assert its[1] < its[0], its


# --------------------------------------------------------------------------
# known limit: i.i.d. random unit vectors at dt/h^2 = 6.55
# --------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.01, 0.1, 1.0])
def test_random_unit_vectors_limit_of_the_vcycle(alpha):
    """The 256 x 256 x 128 workload's field and dt/h^2 on a 16 x 16 x 8 grid.
    The system is well posed for every alpha: plain GCR reaches 1e-8.  The
    V-cycle-preconditioned GCR converges for alpha = 1 and stagnates for
    alpha <= 0.1, where the symmetric part of the level-1 Galerkin operator
    has a large share of negative eigenvalues (2 % for alpha = 1, over 25 %
    below)."""
    grid, h = (16, 16, 8), 1.0 / 16
    dt = 6.5536 * h * h
    m = inputs.random_sphere(*grid, seed=0).reshape(-1)
    b = m / dt
    plain = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(prec=1, maxit=3000, rtol=1e-8))
    x, st, it, rr = plain.solve(b)
    assert st == oracle.OK and rr < 1e-8
    H = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-8, maxit=60))
    x, st, it, rr = H.solve(b)
    A1 = H.matrix(1).toarray()
    neg = np.mean(np.linalg.eigvalsh(0.5 * (A1 + A1.T)) < 0)
    if alpha == 1.0:
        assert st == oracle.OK and it <= 40
        assert neg < 0.05
    else:
        assert st == oracle.NOT_CONVERGED and rr > 0.5
        assert neg > 0.25


def _adaptive_guess(states):
    """The reading restated: Newton's backward-difference series of
    states[0] = m^n, states[l] = m^{n-l}, its terms D^j m^n taken while their
    norms shrink (D m^n always), summed as the polynomial extrapolation of
    that degree."""
    from math import comb

    d = len(states) - 1
    if d == 0:
        return states[0].copy(), 0
    t = [s.copy() for s in states]
    s2 = [0.0] * (d + 1)
    for j in range(1, d + 1):
        for l in range(d - j + 1):
            t[l] = t[l] - t[l + 1]
        s2[j] = float(np.dot(t[0], t[0]))
    k = 1
    for j in range(2, d + 1):
        if s2[j] < s2[j - 1]:
            k = j
        else:
            break
    c = [(-1) ** l * comb(k + 1, l + 1) for l in range(k + 1)]
    return sum(c[l] * states[l] for l in range(k + 1)), k


def step_guess_violations():
    """The closed-form pins of the step guess, as a list of violations (empty
    when the oracle passes).  States sampled from a vector polynomial of
    degree q in time, with shrinking terms: the backward differences shrink
    up to D^q (D^{q+1} is rounding), so the guess is the polynomial's next
    value; with d < q earlier states the degree-d extrapolation misses it.
    A series whose differences grow keeps the linear extrapolation."""
    bad = []
    rng = np.random.default_rng(3)
    n3 = 300
    for q in (1, 2, 3, 4, 5):
        a = [rng.standard_normal(n3) * 0.05 ** j for j in range(q + 1)]

        def P(t):
            return sum(a[j] * t ** j for j in range(q + 1))

        states = [P(-float(l)) for l in range(7)]  # m^n at t = 0, earlier at -1, -2, ...
        nxt = P(1.0)
        for d in range(7):
            x, k = oracle.step_guess(states[0], states[1:d + 1])
            err = np.abs(x - nxt).max()
            if d == 0 and not (k == 0 and np.array_equal(x, states[0])):
                bad.append(("m^n", q, d, k))
            elif d >= q and not (k >= q and err <= 1e-12 * np.abs(nxt).max()):
                bad.append(("exact", q, d, k, err))
            elif 0 < d < q and not (k == d and err > 1e-8):
                bad.append(("degree", q, d, k, err))
    m = np.ones(n3)
    prev = [m + (-2.0) ** l * 1e-3 for l in range(1, 4)]
    x, k = oracle.step_guess(m, prev)
    if not (k == 1 and np.array_equal(x, 2 * m - prev[0])):
        bad.append(("growing", k))
    return bad


def test_step_guess_extrapolates_polynomials_in_time_exactly():
    assert step_guess_violations() == []


def test_step_guess_matches_the_restated_rule():
    rng = np.random.default_rng(5)
    base = rng.standard_normal(600)
    drift = rng.standard_normal(600)
    for d in range(7):
        states = [base + (1 + 0.3 * l) ** 2 * 1e-2 * drift + 1e-9 * rng.standard_normal(600) for l in range(d + 1)]
        x, k = oracle.step_guess(states[0], states[1:])
        xr, kr = _adaptive_guess(states)
        assert k == kr, (d, k, kr)
        assert np.array_equal(x, xr), d


def test_step_initial_approximation_is_the_extrapolated_state():
    """Reading of the time loop (Algorithm 1 takes u_0 as an input): step k of
    a call starts from the extrapolation of m^n and the min(k, 6) states
    before it, with as many backward-difference terms as keep shrinking.  An
    eight-step call equals eight explicit solves with those guesses, the order
    grows past cubic, and each extrapolated guess starts closer to the
    solution than m^n does."""
    n = 16
    grid, h, alpha, dt = (n, n, 1), 1 / n, 0.05, 2e-3
    m0 = inputs.smooth_field(*grid, seed=4).reshape(-1)
    p = oracle.Params(rtol=1e-12)
    ms = [m0]
    gains, orders = [], []
    for k in range(8):
        states = ms[::-1][:7]
        guess, order = _adaptive_guess(states)
        orders.append(order)
        H = oracle.Hierarchy(grid, h, alpha, dt, ms[-1], p)
        x, st, it, rr = H.solve(ms[-1] / dt, guess.copy())
        assert st == oracle.OK
        if k > 0:
            gains.append(np.linalg.norm(x - guess) / np.linalg.norm(x - ms[-1]))
        v = x.reshape(3, -1)
        ms.append((v / np.linalg.norm(v, axis=0)).reshape(-1))
    out, its, rrs, st = oracle.step(m0, 8, grid, h, alpha, dt, p)
    assert st == oracle.OK
    assert np.abs(out - ms[-1]).max() <= 1e-13
    assert max(orders) >= 4, orders
    assert max(gains) < 0.5, gains


def _stall_stop(hist, restart, window, ratio, maxit):
    """The stagnation stop restated on a residual history of a run without
    it: the restarts fall every `restart` iterations; at a restart t the
    solve stops when hist[t] exceeds `ratio` times its value at the latest
    restart t0 <= t - window.  Returns the iteration it stops at, or None."""
    for t in range(restart, maxit, restart):
        earlier = [t0 for t0 in range(0, t, restart) if t0 <= t - window]
        if earlier and hist[t] > ratio * hist[earlier[-1]]:
            return t
    return None


@pytest.mark.parametrize("alpha", [0.01, 0.1, 1.0])
def test_stagnation_stop(alpha):
    """The optional stagnation stop (stall_window, stall_ratio; not in the
    paper): on the random-unit-vector field, where the V-cycle-preconditioned
    GCR stagnates for alpha <= 0.1 and converges for alpha = 1, the stop
    point follows from the stated rule applied to the residual history of a
    run without it, and the stopped solve equals a run with maxit set to that
    point, bit for bit.  Windows that are not multiples of the restart length
    and a ratio under which the converging solve stops too check which
    earlier restart the rule compares with and the direction of the test."""
    grid, h = (16, 16, 8), 1.0 / 16
    dt = 6.5536 * h * h
    m = inputs.random_sphere(*grid, seed=0).reshape(-1)
    b = m / dt
    maxit = 60
    _, st0, it0, rr0, hist = oracle.Hierarchy(grid, h, alpha, dt, m,
                                              oracle.Params(rtol=1e-8, maxit=maxit)).solve(b, history=True)
    cases = [(20, 0.99), (15, 0.99), (25, 0.99), (10, 0.5), (20, 1e-9)]
    stops = []
    for window, ratio in cases:
        p = oracle.Params(rtol=1e-8, maxit=maxit, stall_window=window, stall_ratio=ratio)
        x, st, it, rr = oracle.Hierarchy(grid, h, alpha, dt, m, p).solve(b)
        t = _stall_stop(hist, 10, window, ratio, min(maxit, it0))
        stops.append(t)
        if t is None:  # the stop never fires: the run is unchanged
            assert (st, it, rr) == (st0, it0, rr0)
            continue
        assert st == oracle.NOT_CONVERGED and it == t
        xr, str_, itr, rrr = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-8, maxit=t)).solve(b)
        assert itr == t and np.array_equal(x, xr) and rr == rrr
    if alpha < 1:
        assert stops[:3] == [20, 20, 30]  # a window of 25 compares iteration 30 with 0
    else:
        assert stops[:4] == [None] * 4 and stops[4] == 20


# the paper's closed-form initial states (Sec. 4.4) and the symmetries that
# the exchange-only step must keep: the cell-centred Neumann Laplacian
# commutes with the grid's mirrors, and the step with proper rotations of
# every spin, so a state with m(mirror p) = R m(p) keeps it at every step
_ROT_X = np.array([1.0, -1.0, -1.0])  # rotation by pi about the x axis


def _paper_state_symmetries(M, name):
    """Largest deviation from each symmetry the state has (M: (3, nz, ny, nx))."""
    R = _ROT_X[:, None, None, None]
    if name == "s":  # (0,1,0) | (1,0,0) | (0,1,0) across x: mirror symmetric
        return [np.abs(M[..., ::-1] - M).max()]
    if name == "c":  # (0,1,0) | (1,0,0) | (0,-1,0): the mirror in x turns m2
        return [np.abs(R * M[..., ::-1] - M).max()]
    if name == "flower":  # as C, and the same about the mirror in y
        return [np.abs(R * M[..., ::-1] - M).max(), np.abs(R * M[:, :, ::-1, :] - M).max()]
    # c1: g = cos(pi x) cos(pi y) [cos(pi z)] is even under (x, y) -> (1-x, 1-y)
    return [np.abs(M[:, :, ::-1, ::-1] - M).max()]


@pytest.mark.parametrize("grid", [(40, 30, 1), (16, 12, 8)])
@pytest.mark.parametrize("name", ["c1", "s", "c", "flower"])
def test_paper_initial_states_keep_their_symmetries(name, grid):
    """Three steps from each closed-form initial state of Sec. 4.4 (C1, S,
    C, Flower) converge, leave every spin of unit length, change the field,
    and keep the state's mirror symmetries to the solve's accuracy (a wrong
    neighbour at a boundary, or an operator term that does not commute with
    the mirrors, breaks them)."""
    nx, ny, nz = grid
    h = 1.0 / nx
    dt, alpha = 8 * h * h, 0.05
    m0 = getattr(inputs, name + "_state")(nx, ny, nz).reshape(-1)
    M0 = m0.reshape(3, nz, ny, nx)
    assert max(_paper_state_symmetries(M0, name)) <= 1e-15  # C1: cosines of mirrored points round apart
    m, its, rrs, st = oracle.step(m0, 3, grid, h, alpha, dt, oracle.Params(rtol=1e-12))
    assert st == oracle.OK and min(its) > 0
    assert np.abs(m - m0).max() > 1e-3
    np.testing.assert_allclose(np.linalg.norm(m.reshape(3, -1), axis=0), 1.0, atol=1e-14)
    assert max(_paper_state_symmetries(m.reshape(3, nz, ny, nx), name)) <= 1e-9
