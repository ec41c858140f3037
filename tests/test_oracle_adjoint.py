"""Pins of the oracle's adjoint (differentiation of the time step).

The oracle's gradient comes from its adjoint hierarchy (every level operator
transposed) and the vector-Jacobian product of one step.  It is checked
against things it does not use:

* the transpose of the operator written out independently from the paper's
  component form (``reference_forms.operator_dense``);
* a dense solve with that transpose;
* central finite differences of a dense forward map (dense solve of the same
  independently written operator, then the projection) -- for the gradient
  with respect to the initial state and to alpha, through several steps.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2608_09102_b300 import inputs
from tests import reference_forms as rf


def _dense_forward(m0, n_steps, grid, h, alpha, dt):
    m = np.array(m0, np.float64).reshape(-1)
    n = int(np.prod(grid))
    for _ in range(n_steps):
        A = rf.operator_dense(*grid, h, alpha, dt, m)
        x = np.linalg.solve(A, m / dt).reshape(3, n)
        m = (x / np.sqrt(np.sum(x * x, axis=0))).reshape(-1)
    return m


def _dense_loss(m0, mt, n_steps, grid, h, alpha, dt):
    d = _dense_forward(m0, n_steps, grid, h, alpha, dt) - mt
    return 0.5 * float(d @ d)


CASES = [((5, 4, 1), 0.1, 2e-2), ((4, 3, 3), 0.3, 1e-2), ((12, 10, 1), 0.05, 4e-3)]


@pytest.mark.parametrize("grid,alpha,dt", CASES)
def test_adjoint_levels_are_transposes(grid, alpha, dt):
    h = 1.0 / grid[0]
    m = inputs.smooth_field(*grid, seed=2).reshape(-1)
    p = oracle.Params(coarsest_cells=4)
    H = oracle.Hierarchy(grid, h, alpha, dt, m, p)
    T = oracle.Hierarchy(grid, h, alpha, dt, m, p, adjoint=True)
    assert T.nlevels == H.nlevels
    A0 = rf.operator_dense(*grid, h, alpha, dt, m)
    np.testing.assert_allclose(T.matrix(0).toarray(), A0.T, rtol=0, atol=1e-12 * np.abs(A0).max())
    for l in range(T.nlevels - 1):
        assert np.array_equal(T.agg(l), H.agg(l))
    for l in range(T.nlevels):
        d = T.matrix(l).toarray() - H.matrix(l).toarray().T
        assert np.abs(d).max() == 0.0


@pytest.mark.parametrize("grid,alpha,dt", CASES)
def test_adjoint_solve_matches_dense(grid, alpha, dt):
    h = 1.0 / grid[0]
    n = int(np.prod(grid))
    m = inputs.smooth_field(*grid, seed=3).reshape(-1)
    T = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-13, coarsest_cells=4), adjoint=True)
    g = inputs.rhs_field(*grid, seed=4).reshape(-1)
    lam, st, it, rr = T.solve(g, np.zeros(3 * n))
    assert st == oracle.OK and rr < 1e-13
    ref = np.linalg.solve(rf.operator_dense(*grid, h, alpha, dt, m).T, g)
    assert np.linalg.norm(lam - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [2, 0])  # exact preconditioner; the V-cycle of A^T
@pytest.mark.parametrize("grid,alpha,dt", CASES[:2])
def test_gradient_matches_finite_differences(grid, alpha, dt, prec):
    h = 1.0 / grid[0]
    n_steps = 3
    m0 = inputs.smooth_field(*grid, seed=5).reshape(-1)
    mt = inputs.smooth_field(*grid, seed=6).reshape(-1)
    p = oracle.Params(rtol=1e-14, maxit=400, coarsest_cells=4, prec=prec)
    loss, gm, ga = oracle.loss_gradient(m0, mt, n_steps, grid, h, alpha, dt, p)
    assert abs(loss - _dense_loss(m0, mt, n_steps, grid, h, alpha, dt)) <= 1e-12 * max(loss, 1.0)
    rng = np.random.Generator(np.random.PCG64(11))
    eps = 1e-6
    for _ in range(3):
        d = rng.standard_normal(m0.size)
        fd = (_dense_loss(m0 + eps * d, mt, n_steps, grid, h, alpha, dt)
              - _dense_loss(m0 - eps * d, mt, n_steps, grid, h, alpha, dt)) / (2 * eps)
        assert abs(gm @ d - fd) <= 1e-6 * max(abs(fd), 1e-3), (gm @ d, fd)
    fda = (_dense_loss(m0, mt, n_steps, grid, h, alpha + eps, dt)
           - _dense_loss(m0, mt, n_steps, grid, h, alpha - eps, dt)) / (2 * eps)
    assert abs(ga - fda) <= 1e-6 * max(abs(fda), 1e-3), (ga, fda)


def test_single_step_vjp_matches_dense_jacobian():
    """One step on a 3x3x1 grid: the VJP equals g^T J with J the full
    Jacobian of the dense step map by central differences, column by column."""
    grid, alpha, dt = (3, 3, 1), 0.2, 5e-2
    h = 1.0 / 3
    n3 = 27
    m = inputs.smooth_field(*grid, seed=7).reshape(-1)
    g = inputs.rhs_field(*grid, seed=8).reshape(-1)
    ms, xs = oracle.forward_states(m, 1, grid, h, alpha, dt, oracle.Params(rtol=1e-14, prec=2))
    mbar, abar, st, it, rr = oracle.step_vjp(m, xs[0], g, grid, h, alpha, dt, oracle.Params(rtol=1e-14, prec=2))
    eps = 1e-6
    J = np.zeros((n3, n3))
    for j in range(n3):
        e = np.zeros(n3)
        e[j] = eps
        J[:, j] = (_dense_forward(m + e, 1, grid, h, alpha, dt) - _dense_forward(m - e, 1, grid, h, alpha, dt)) / (
            2 * eps)
    np.testing.assert_allclose(mbar, g @ J, rtol=0, atol=1e-7 * np.abs(g @ J).max())
    ja = (_dense_forward(m, 1, grid, h, alpha + eps, dt) - _dense_forward(m, 1, grid, h, alpha - eps, dt)) / (2 * eps)
    assert abs(abar - g @ ja) <= 1e-7 * max(abs(g @ ja), 1e-3)
