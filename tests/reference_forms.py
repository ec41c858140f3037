"""Closed forms written straight from the paper's statement of the problem,
used to pin the oracle to something other than itself.

* ``laplacian_dense``: the cell-centred Neumann Laplacian as a Kronecker sum
  of 1-D second differences (textbook construction, mirror ghost cells).
* ``operator_dense``: the damped semi-implicit system of Sec. 2.1, written
  row block by row block from its component expansion (three scalar
  equations, each holding the cross-product terms and the alpha-terms), then
  divided by dt.  Unknown order [m1; m2; m3] (component-major).
* ``dct_solve``: exact solution for a spatially constant unit m~ by the
  DCT-II diagonalisation of the Neumann Laplacian.
* ``manufactured``: an exact smooth unit field and the forcing that makes it
  solve the damped LL equation, for the time-convergence pin.
* ``block_gs_sweep``, ``vcycle_dense``: the block Gauss-Seidel sweep and the
  V-cycle of Sec. 3 on dense matrices, with Boolean prolongations made from
  the aggregate maps (``boolean_prolongation``, ``galerkin_levels``).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def second_difference_1d(n: int, h: float) -> np.ndarray:
    """1-D cell-centred second difference with homogeneous Neumann ends."""
    t = np.zeros((n, n))
    for i in range(n):
        if i > 0:
            t[i, i - 1] += 1.0
            t[i, i] -= 1.0
        if i < n - 1:
            t[i, i + 1] += 1.0
            t[i, i] -= 1.0
    return t / (h * h)


def laplacian_dense(nx: int, ny: int, nz: int, h: float) -> np.ndarray:
    ix, iy, iz = np.eye(nx), np.eye(ny), np.eye(nz)
    tx, ty, tz = (second_difference_1d(n, h) for n in (nx, ny, nz))
    return (np.kron(iz, np.kron(iy, tx)) + np.kron(iz, np.kron(ty, ix))
            + np.kron(tz, np.kron(iy, ix)))


def operator_dense(nx, ny, nz, h, alpha, dt, m) -> np.ndarray:
    """Dense system matrix from the component form of the damped scheme.

    Row 1 (Sec. 2.1): m1 + dt(m2 D m3 - m3 D m2)
                      + alpha dt[-(m2^2+m3^2) D m1 + m1 m2 D m2 + m1 m3 D m3]
    and rows 2, 3 as printed, all divided by dt (right-hand side m^n/dt).
    """
    n = nx * ny * nz
    m = np.asarray(m, np.float64).reshape(3, n)
    m1, m2, m3 = m
    L = laplacian_dense(nx, ny, nz, h)
    I = np.eye(n)

    def d(v):
        return np.diag(v) @ L

    a = alpha
    blocks = [
        [I / dt + d(-a * (m2 ** 2 + m3 ** 2)), d(-m3 + a * m1 * m2), d(m2 + a * m1 * m3)],
        [d(m3 + a * m1 * m2), I / dt + d(-a * (m1 ** 2 + m3 ** 2)), d(-m1 + a * m2 * m3)],
        [d(-m2 + a * m1 * m3), d(m1 + a * m2 * m3), I / dt + d(-a * (m1 ** 2 + m2 ** 2))],
    ]
    return np.block(blocks)


def _frame(mdir):
    """Right-handed orthonormal frame (e1, e2, m) with e1 x e2 = m."""
    m = np.asarray(mdir, np.float64)
    m = m / np.linalg.norm(m)
    t = np.array([1.0, 0.0, 0.0]) if abs(m[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = t - m * (m @ t)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(m, e1)
    return e1, e2, m


def dct_solve(nx, ny, nz, h, alpha, dt, mdir, b) -> np.ndarray:
    """Exact solution of A x = b for the constant unit field m~ = mdir.

    In the frame (e1, e2, m): C(m) maps e1 -> e2 - alpha e1 and
    e2 -> -e1 - alpha e2 and kills m, so w = x.e1 + i x.e2 obeys
    w/dt + (i - alpha) Delta_h w = b.e1 + i b.e2 and x.m = dt b.m.
    Delta_h is diagonal in the orthonormal DCT-II basis with eigenvalues
    -(4/h^2) sum_d sin^2(pi k_d / (2 n_d)).
    """
    e1, e2, m = _frame(mdir)
    b = np.asarray(b, np.float64).reshape(3, nz, ny, nx)
    be1 = np.tensordot(e1, b, axes=(0, 0))
    be2 = np.tensordot(e2, b, axes=(0, 0))
    bm = np.tensordot(m, b, axes=(0, 0))
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lam = -(4.0 / h ** 2) * (np.sin(np.pi * kx / (2 * nx)) ** 2 + np.sin(np.pi * ky / (2 * ny)) ** 2
                             + np.sin(np.pi * kz / (2 * nz)) ** 2)
    denom = 1.0 / dt + (1j - alpha) * lam
    beta_hat = sfft.dctn(be1, type=2, norm="ortho") + 1j * sfft.dctn(be2, type=2, norm="ortho")
    w_hat = beta_hat / denom
    wr = sfft.idctn(w_hat.real, type=2, norm="ortho")
    wi = sfft.idctn(w_hat.imag, type=2, norm="ortho")
    a3 = dt * bm
    x = (e1[:, None, None, None] * wr + e2[:, None, None, None] * wi
         + m[:, None, None, None] * a3)
    return x.reshape(-1)


class Manufactured:
    """m_e = (sin th cos phi, sin th sin phi, cos th), th = pi/4,
    phi = t + cos(pi x) cos(pi y) on the unit square (zero normal derivative
    on the boundary).  forcing(t) = d_t m_e + m_e x Delta m_e
    + alpha m_e x (m_e x Delta m_e), so that m_e solves
    d_t m = -m x Delta m - alpha m x (m x Delta m) + f."""

    def __init__(self, n: int, alpha: float):
        self.n, self.alpha = n, alpha
        s = (np.arange(n) + 0.5) / n
        self.Y, self.X = np.meshgrid(s, s, indexing="ij")
        self.th = np.pi / 4

    def phi(self, t):
        return t + np.cos(np.pi * self.X) * np.cos(np.pi * self.Y)

    def m(self, t):
        p = self.phi(t)
        s, c = np.sin(self.th), np.cos(self.th)
        return np.stack([s * np.cos(p), s * np.sin(p), c + 0 * p])[:, None]

    def forcing(self, t):
        X, Y = self.X, self.Y
        p = self.phi(t)
        s = np.sin(self.th)
        grad2 = np.pi ** 2 * (np.sin(np.pi * X) ** 2 * np.cos(np.pi * Y) ** 2
                              + np.cos(np.pi * X) ** 2 * np.sin(np.pi * Y) ** 2)
        lap = -2 * np.pi ** 2 * np.cos(np.pi * X) * np.cos(np.pi * Y)
        dcos = -np.sin(p) * lap - np.cos(p) * grad2
        dsin = np.cos(p) * lap - np.sin(p) * grad2
        me = self.m(t)[:, 0]
        lm = np.stack([s * dcos, s * dsin, 0 * p])
        dt_m = np.stack([-s * np.sin(p), s * np.cos(p), 0 * p])
        c1 = np.cross(me, lm, axis=0)
        c2 = np.cross(me, c1, axis=0)
        return (dt_m + c1 + self.alpha * c2)[:, None]


# --------------------------------------------------------------------------
# smoother and V-cycle (Sec. 3), written from their textbook definitions on
# dense matrices: an independent restatement of what the oracle's gs_sweep
# and vcycle compute
# --------------------------------------------------------------------------

def boolean_prolongation(agg, nc: int) -> np.ndarray:
    """Dense Boolean prolongation of Eq. (Pagg) for a component-major vector:
    P[(c, k), (c, agg[k])] = 1, i.e. I_3 (x) P_cell."""
    agg = np.asarray(agg)
    n = agg.size
    p = np.zeros((n, nc))
    p[np.arange(n), agg] = 1.0
    return np.kron(np.eye(3), p)


def galerkin_levels(A0: np.ndarray, aggs) -> list:
    """Level operators A_{l+1} = P_l^T A_l P_l (Eq. galerkin) as dense
    products, from the level-0 operator and the aggregate maps."""
    ops, ps = [np.asarray(A0)], []
    for agg in aggs:
        nc = int(np.max(agg)) + 1
        P = boolean_prolongation(agg, nc)
        ps.append(P)
        ops.append(P.T @ ops[-1] @ P)
    return ops, ps


def block_gs_sweep(A: np.ndarray, colours, b, x, forward: bool = True) -> np.ndarray:
    """One block Gauss-Seidel sweep on a component-major system A (3n x 3n).

    The cells are visited colour class by colour class, ascending colours
    for a forward sweep and descending for a backward one.  A cell k takes
    the exact solution of its own 3x3 equation,
        x_k <- D_k^{-1} (b_k - sum_{j != k} A_kj x_j),
    D_k = A_kk its diagonal block, with every other cell's current value.
    Cells of one colour share no off-diagonal block (checked), so updating
    a class all at once is the same as visiting its cells one by one."""
    colours = np.asarray(colours)
    n = colours.size
    x = np.array(x, np.float64, copy=True)
    b = np.asarray(b, np.float64)
    classes = sorted(set(colours.tolist()), reverse=not forward)
    for c in classes:
        cells = np.flatnonzero(colours == c)
        rows = np.concatenate([cells, n + cells, 2 * n + cells])
        owner = np.tile(cells, 3)
        assert not np.any(A[np.ix_(rows, rows)][owner[:, None] != owner[None, :]]), "cells of one colour are coupled"
        s = b[rows] - A[rows] @ x  # every cell's residual with the old values
        new = np.empty(rows.size)
        for i, k in enumerate(cells):
            mine = np.array([i, cells.size + i, 2 * cells.size + i])
            own = rows[mine]
            d = A[np.ix_(own, own)]
            # add back the cell's own diagonal-block term, then solve with it
            new[mine] = np.linalg.solve(d, s[mine] + d @ x[own])
        x[rows] = new
    return x


def vcycle_dense(ops, ps, colours, b, nu_pre: int = 1, nu_post: int = 1, level: int = 0,
                 kcycle: int = 0) -> np.ndarray:
    """One V(nu_pre, nu_post) cycle for ops[level] x = b from x = 0 (Sec. 3):
    forward block-GS sweeps, residual, restriction P^T, the coarse problem
    from a zero guess, prolongation x += P e, backward sweeps; an exact
    (dense) solve on the last level.  The coarse problem of levels
    1..kcycle (never the last) is solved by kcycle_inner, else by the same
    cycle one level down."""
    A = ops[level]
    if level == len(ops) - 1:
        return np.linalg.solve(A, b)
    x = np.zeros_like(np.asarray(b, np.float64))
    for _ in range(nu_pre):
        x = block_gs_sweep(A, colours[level], b, x, True)
    r = b - A @ x
    bc = ps[level].T @ r
    if level + 1 <= kcycle and level + 1 < len(ops) - 1:
        e = kcycle_inner(ops, ps, colours, bc, nu_pre, nu_post, level + 1, kcycle)
    else:
        e = vcycle_dense(ops, ps, colours, bc, nu_pre, nu_post, level + 1, kcycle)
    x = x + ps[level] @ e
    for _ in range(nu_post):
        x = block_gs_sweep(A, colours[level], b, x, False)
    return x


def kcycle_inner(ops, ps, colours, r, nu_pre: int, nu_post: int, level: int, kcycle: int) -> np.ndarray:
    """The Krylov-accelerated coarse solve of Sec. 3.1 (reading: two steps of
    Algorithm 1 on A e = r from e = 0, preconditioned by this level's cycle
    B): the correction e in span{B r, B r1} that minimises |r - A e|, with
    r1 = r - (c1.r) c1 the residual after the first step.  Written as the
    least-squares solve over the two directions (not the oracle's Gram-Schmidt
    recurrence); a direction whose image is zero is dropped."""
    A = ops[level]
    z1 = vcycle_dense(ops, ps, colours, r, nu_pre, nu_post, level, kcycle)
    c1 = A @ z1
    if not np.any(c1):
        return np.zeros_like(r)
    r1 = r - (c1 @ r) / (c1 @ c1) * c1
    z2 = vcycle_dense(ops, ps, colours, r1, nu_pre, nu_post, level, kcycle)
    W = np.column_stack([c1, A @ z2])
    if not np.any(W[:, 1]) or np.linalg.matrix_rank(W) < 2:
        return (c1 @ r) / (c1 @ c1) * z1
    y, *_ = np.linalg.lstsq(W, r, rcond=None)
    return y[0] * z1 + y[1] * z2
