"""The adjoint on the GPU (A^T hierarchy, step VJPs, autograd through many
steps) against the FP64 oracle's adjoint and against central finite
differences of the GPU forward map."""
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

CASES = {
    "2d": ((24, 20, 1), 0.1, 4e-3),
    "3d": ((12, 10, 8), 0.02, 2.0 / 144),
    "odd": ((13, 7, 5), 0.3, 1e-3),
}


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=DEV)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_solve_matches_oracle(name):
    grid, alpha, dt = CASES[name]
    h = 1.0 / grid[0]
    m = inputs.smooth_field(*grid, seed=1).reshape(-1)
    g = inputs.rhs_field(*grid, seed=2).reshape(-1)
    T = ll.Adjoint(_t(m), alpha, dt, h, grid, ll.Params(rtol=1e-12, coarsest_cells=8))
    lam = torch.zeros(g.size, dtype=torch.float64, device=DEV)
    st, it, rr = T.solve(_t(g), lam)
    O = oracle.Hierarchy(grid, h, alpha, dt, m, oracle.Params(rtol=1e-12, coarsest_cells=8), adjoint=True)
    lo, sto, ito, rro = O.solve(g, np.zeros_like(g))
    assert st == ll.LL_OK and sto == oracle.OK and rr < 1e-12
    assert abs(it - ito) <= 1
    assert np.linalg.norm(_np(lam) - lo) <= 1e-10 * np.linalg.norm(lo)


@pytest.mark.parametrize("precision", [ll.LL_FP64, ll.LL_MIXED_FP32])
@pytest.mark.parametrize("name", list(CASES))
def test_step_vjp_matches_oracle(name, precision):
    grid, alpha, dt = CASES[name]
    h = 1.0 / grid[0]
    n = int(np.prod(grid))
    m = inputs.smooth_field(*grid, seed=3).reshape(-1)
    g = inputs.rhs_field(*grid, seed=4).reshape(-1)
    p = ll.Params(rtol=1e-12, coarsest_cells=8, precision=precision)
    H = ll.Hierarchy(_t(m), alpha, dt, h, grid, p)
    mg = _t(m)
    x = torch.empty(3 * n, dtype=torch.float64, device=DEV)
    H.step_save(mg, x)
    T = ll.Adjoint(_t(m), alpha, dt, h, grid, p)
    mbar, abar, st, it, rr = T.vjp(_t(m), alpha, dt, x, _t(g))
    assert st == ll.LL_OK
    mo, ao, sto, ito, rro = oracle.step_vjp(m, _np(x), g, grid, h, alpha, dt,
                                            oracle.Params(rtol=1e-12, coarsest_cells=8))
    assert np.linalg.norm(_np(mbar) - mo) <= 1e-9 * np.linalg.norm(mo)
    assert abs(abar - ao) <= 1e-9 * max(abs(ao), 1e-12)


def test_gradient_matches_oracle_through_steps():
    grid, alpha, dt = CASES["2d"]
    h = 1.0 / grid[0]
    m0 = inputs.smooth_field(*grid, seed=5).reshape(-1)
    mt = inputs.smooth_field(*grid, seed=6).reshape(-1)
    p = ll.Params(rtol=1e-12, coarsest_cells=8)
    m0t = _t(m0).requires_grad_(True)
    at = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    mN = ll.steps_autograd(m0t, at, 7, dt, h, grid, p, checkpoint=3)
    loss = 0.5 * torch.sum((mN - _t(mt)) ** 2)
    loss.backward()
    lo, go, gao = oracle.loss_gradient(m0, mt, 7, grid, h, alpha, dt, oracle.Params(rtol=1e-12, coarsest_cells=8))
    assert abs(float(loss.detach()) - lo) <= 1e-10 * lo
    assert np.linalg.norm(_np(m0t.grad) - go) <= 1e-8 * np.linalg.norm(go)
    assert abs(float(at.grad) - gao) <= 1e-8 * abs(gao)


def _loss_gpu(m0, mt, alpha, n_steps, dt, h, grid, p):
    m = _t(m0)
    ll.step(m, n_steps, alpha, dt, h, grid, p)
    d = m - mt
    return 0.5 * float(torch.dot(d, d))


def test_gradient_matches_finite_differences_96cube():
    """3-D 96^3, alpha 0.1, dt 1e-3, 20 steps, checkpoints every 5 steps;
    loss 0.5 |m^20 - m_target|^2 with smooth unit fields (seeds 0 and 1).
    The gradient along a random direction and with respect to alpha equals
    central differences (eps 1e-6) of the GPU forward map."""
    grid, alpha, dt, n_steps = (96, 96, 96), 0.1, 1e-3, 20
    h = 1.0 / 96
    m0 = inputs.smooth_field(*grid, seed=0).reshape(-1)
    mt = _t(inputs.smooth_field(*grid, seed=1).reshape(-1))
    p = ll.Params(rtol=1e-12)
    m0t = _t(m0).requires_grad_(True)
    at = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    mN = ll.steps_autograd(m0t, at, n_steps, dt, h, grid, p, checkpoint=5)
    loss = 0.5 * torch.sum((mN - mt) ** 2)
    loss.backward()
    rng = np.random.Generator(np.random.PCG64(12))
    d = rng.standard_normal(m0.size)
    eps = 1e-6
    fd = (_loss_gpu(m0 + eps * d, mt, alpha, n_steps, dt, h, grid, p)
          - _loss_gpu(m0 - eps * d, mt, alpha, n_steps, dt, h, grid, p)) / (2 * eps)
    gd = float(torch.dot(m0t.grad, _t(d)))
    assert abs(gd - fd) <= 1e-5 * abs(fd), (gd, fd)
    fda = (_loss_gpu(m0, mt, alpha + eps, n_steps, dt, h, grid, p)
           - _loss_gpu(m0, mt, alpha - eps, n_steps, dt, h, grid, p)) / (2 * eps)
    assert abs(float(at.grad) - fda) <= 1e-5 * abs(fda), (float(at.grad), fda)
