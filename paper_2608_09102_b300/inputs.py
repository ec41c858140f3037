"""Seeded synthetic magnetisation fields (shared by the oracle tests and the
CUDA path; holds none of the solver's arithmetic).

Every generator returns a float64 array of shape (3, nz, ny, nx): the three
components in component-major (structure-of-arrays) order, each a C-ordered
grid with x fastest.  Coordinates are cell centres s_d = (i + 1/2)/n_d of the
unit-scaled domain.  Fields are normalised to unit length per cell.

The paper's data is not public; these fields stand in for its workloads:

* ``smooth_field``  sum of 8 random cosine (Neumann-compatible) modes per
  component, the "seeded smooth random field";
* ``vortex``        a vortex core (m_z = exp(-(r/0.1)^2)) plus Gaussian noise;
* ``random_sphere`` i.i.d. directions uniform on the sphere;
* ``c1_state``, ``s_state``, ``c_state``, ``flower_state``, ``trivial_state``:
  the closed-form initial states of Sec. 4 (Sec. 4.4 for C1, S, C, Flower).
"""
from __future__ import annotations

import numpy as np


def _coords(nx: int, ny: int, nz: int):
    sx = (np.arange(nx) + 0.5) / nx
    sy = (np.arange(ny) + 0.5) / ny
    sz = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(sz, sy, sx, indexing="ij")
    return X, Y, Z


def _normalise(v: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.sum(v * v, axis=0))
    bad = nrm < 1e-12
    if np.any(bad):
        v = v.copy()
        v[0][bad], v[1][bad], v[2][bad] = 0.0, 0.0, 1.0
        nrm = np.where(bad, 1.0, nrm)
    return v / nrm


def smooth_field(nx: int, ny: int = 1, nz: int = 1, seed: int = 0, modes: int = 8, kmax: int = 4):
    """Per component c: v_c = sum_q a_cq prod_d cos(pi k_cqd s_d), a ~ N(0,1),
    k uniform in {0..kmax} (only along dimensions with more than one cell);
    then m = v/|v|."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = _coords(nx, ny, nz)
    v = np.zeros((3, nz, ny, nx))
    for c in range(3):
        for _ in range(modes):
            a = rng.standard_normal()
            k = rng.integers(0, kmax + 1, size=3)
            if ny == 1:
                k[1] = 0
            if nz == 1:
                k[2] = 0
            v[c] += a * np.cos(np.pi * k[0] * X) * np.cos(np.pi * k[1] * Y) * np.cos(np.pi * k[2] * Z)
    return _normalise(v)


def vortex(nx: int, ny: int, nz: int = 1, seed: int = 0, noise: float = 1e-2, core: float = 0.1):
    """Vortex about the axis through (1/2, 1/2): m_z = exp(-(r/core)^2), the
    in-plane part circulates with length sqrt(1 - m_z^2); plus noise*N(0,1)
    per component; then normalised."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, _ = _coords(nx, ny, nz)
    dx, dy = X - 0.5, Y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    mz = np.exp(-((r / core) ** 2))
    inplane = np.sqrt(np.maximum(0.0, 1.0 - mz * mz))
    rs = np.where(r > 0, r, 1.0)
    v = np.stack([-dy / rs * inplane, dx / rs * inplane, mz])
    v = v + noise * rng.standard_normal(v.shape)
    return _normalise(v)


def random_sphere(nx: int, ny: int = 1, nz: int = 1, seed: int = 0):
    """Independent directions uniform on the unit sphere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _normalise(rng.standard_normal((3, nz, ny, nx)))


def constant_field(nx: int, ny: int = 1, nz: int = 1, direction=(0.0, 0.0, 1.0)):
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    return np.broadcast_to(d[:, None, None, None], (3, nz, ny, nx)).copy()


def trivial_state(nx: int, ny: int = 1, nz: int = 1):
    """m0 = [cos(g) sin(0), sin(g) sin(0), cos(0)] of Sec. 4 (g the product of
    cosines): identically (0, 0, 1)."""
    X, Y, Z = _coords(nx, ny, nz)
    g = np.cos(np.pi * X) * (np.cos(np.pi * Y) if ny > 1 else 1.0) * (np.cos(np.pi * Z) if nz > 1 else 1.0)
    return np.stack([np.cos(g) * np.sin(0.0), np.sin(g) * np.sin(0.0), np.cos(0.0) + 0.0 * g])


def c1_state(nx: int, ny: int = 1, nz: int = 1, theta: float = 0.01):
    """C1 state: [cos(g) sin(0.01), sin(g) sin(0.01), cos(0.01)], g the
    product of cos(pi x), cos(pi y), cos(pi z) over the grid's dimensions
    (a direction of one cell has no factor: its cell centre 1/2 would make g
    vanish, i.e. a constant field)."""
    X, Y, Z = _coords(nx, ny, nz)
    g = np.cos(np.pi * X) * (np.cos(np.pi * Y) if ny > 1 else 1.0) * (np.cos(np.pi * Z) if nz > 1 else 1.0)
    v = np.stack([np.cos(g) * np.sin(theta), np.sin(g) * np.sin(theta), np.cos(theta) + 0.0 * g])
    return _normalise(v)


def s_state(nx: int, ny: int = 1, nz: int = 1):
    """S state: (0,1,0) for x < 1/5 or x > 4/5, (1,0,0) otherwise."""
    X, _, _ = _coords(nx, ny, nz)
    edge = (X < 0.2) | (X > 0.8)
    return np.stack([np.where(edge, 0.0, 1.0), np.where(edge, 1.0, 0.0), np.zeros_like(X)])


def c_state(nx: int, ny: int = 1, nz: int = 1):
    """C state: (0,1,0) for x < 1/5, (0,-1,0) for x > 4/5, (1,0,0) otherwise."""
    X, _, _ = _coords(nx, ny, nz)
    m1 = np.where((X < 0.2) | (X > 0.8), 0.0, 1.0)
    m2 = np.where(X < 0.2, 1.0, np.where(X > 0.8, -1.0, 0.0))
    return np.stack([m1, m2, np.zeros_like(X)])


def flower_state(nx: int, ny: int = 1, nz: int = 1):
    """Flower state: (0, +-1, 0) in the strips x < 1/10 and x > 9/10 (sign by
    the half y < 1/2 or y > 1/2, as tabulated), (1,0,0) otherwise."""
    X, Y, _ = _coords(nx, ny, nz)
    lo, hi = X < 0.1, X > 0.9
    top = Y > 0.5
    m2 = np.where(lo, np.where(top, -1.0, 1.0), np.where(hi, np.where(top, 1.0, -1.0), 0.0))
    m1 = np.where(lo | hi, 0.0, 1.0)
    return np.stack([m1, m2, np.zeros_like(X)])


def rhs_field(nx: int, ny: int = 1, nz: int = 1, seed: int = 0):
    """A generic right-hand side: i.i.d. N(0,1) per unknown."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    return rng.standard_normal((3, nz, ny, nx))


BATCH_SIDES = (32, 48, 64, 96, 128, 192, 256)


def batch_instances(count: int, seed: int = 0, sides=BATCH_SIDES, alpha_range=(0.005, 1.0),
                    dt_range=(1e-5, 1e-2)):
    """Ragged batch of independent 2-D instances: side uniform from ``sides``
    (h = 1/side, square grid), alpha and dt log-uniform in their ranges, a
    smooth unit field per instance (seed = seed * 100003 + index).  Returns a
    list of dicts with keys grid, h, alpha, dt, seed."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    out = []
    for i in range(count):
        side = int(sides[rng.integers(len(sides))])
        a = float(np.exp(rng.uniform(np.log(alpha_range[0]), np.log(alpha_range[1]))))
        dt = float(np.exp(rng.uniform(np.log(dt_range[0]), np.log(dt_range[1]))))
        out.append({"grid": (side, side, 1), "h": 1.0 / side, "alpha": a, "dt": dt,
                    "seed": seed * 100003 + i})
    return out
