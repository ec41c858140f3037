"""Pins of the oracle's smoother and V-cycle (Sec. 3) against an independent
restatement on dense matrices.

The restatement (``reference_forms.block_gs_sweep`` / ``vcycle_dense``) is
built from the paper's component form of the operator
(``operator_dense``), Boolean prolongations made from the aggregate maps and
the colour vectors: none of the oracle's sparse matrices or loops.  The
aggregates and colours themselves are pinned against a pure-Python
restatement of the aggregation rule elsewhere.

The K-cycle of Sec. 3.1 (two GCR steps on a coarse level) is pinned the same
way, against a least-squares statement of the two steps.

The last tests plant plausible mistakes in a copy of the oracle (point
instead of block Gauss-Seidel, the backward sweep in ascending colour order,
a missing pre- or post-sweep, a non-zero coarse initial guess, a flipped
residual sign; one inner K-cycle step instead of two, no orthogonalisation
of the second image) and check that these pins catch every one of them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import reference_forms as rf

# (grid, h, alpha, dt, coarsest_cells): 2-D and 3-D, each with >= 3 levels
GRIDS = [
    ((12, 10, 1), 1 / 12, 0.1, 4e-3, 4),
    ((9, 7, 1), 1 / 9, 0.02, 0.05, 4),
    ((6, 5, 4), 1 / 6, 0.3, 0.02, 4),
    ((5, 4, 3), 1 / 5, 1.0, 0.1, 2),
]


def _unit_field(n, seed):
    v = np.random.default_rng(seed).standard_normal((3, n))
    return (v / np.linalg.norm(v, axis=0)).reshape(-1)


def _case(k, params=None):
    grid, h, alpha, dt, cc = GRIDS[k]
    n = int(np.prod(grid))
    m = _unit_field(n, 100 + k)
    H = oracle.Hierarchy(grid, h, alpha, dt, m, params or oracle.Params(coarsest_cells=cc))
    assert H.nlevels >= 3
    A0 = rf.operator_dense(*grid, h, alpha, dt, m)
    ops, ps = rf.galerkin_levels(A0, [H.agg(l) for l in range(H.nlevels - 1)])
    cols = [H.colours(l) for l in range(H.nlevels)]
    return H, ops, ps, cols


def _sweep_errors(H, ops, cols, seed=0):
    """Largest relative difference of one forward and one backward sweep
    on every level, oracle against the restatement."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for l in range(H.nlevels):
        nn = ops[l].shape[0]
        b, x0 = rng.standard_normal(nn), rng.standard_normal(nn)
        for fwd in (True, False):
            ref = rf.block_gs_sweep(ops[l], cols[l], b, x0, fwd)
            got = H.smooth(b, x0, fwd, l=l)
            worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
    return worst


def _vcycle_errors(H, ops, ps, cols, nu=(1, 1), seed=1):
    """Relative difference of a V-cycle from level 0 and from level 1."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for l in (0, 1):
        r = rng.standard_normal(ops[l].shape[0])
        ref = rf.vcycle_dense(ops, ps, cols, r, nu[0], nu[1], level=l)
        got = H.vcycle(r, l=l)
        worst = max(worst, np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return worst


@pytest.mark.parametrize("k", range(len(GRIDS)))
def test_gauss_seidel_sweeps_match_restatement(k):
    H, ops, ps, cols = _case(k)
    assert _sweep_errors(H, ops, cols) <= 1e-12


@pytest.mark.parametrize("k", range(len(GRIDS)))
def test_vcycle_matches_restatement(k):
    H, ops, ps, cols = _case(k)
    assert _vcycle_errors(H, ops, ps, cols) <= 1e-12


@pytest.mark.parametrize("nu", [(2, 2), (2, 1), (0, 1)])
def test_vcycle_sweep_counts_match_restatement(nu):
    grid, h, alpha, dt, cc = GRIDS[2]
    H, ops, ps, cols = _case(2, oracle.Params(coarsest_cells=cc, nu_pre=nu[0], nu_post=nu[1]))
    assert _vcycle_errors(H, ops, ps, cols, nu) <= 1e-12


@pytest.mark.parametrize("k,kcycle", [(0, 1), (2, 1), (2, 2), (3, 20)])
def test_kcycle_matches_restatement(k, kcycle):
    """The K-cycle (Sec. 3.1, reading: two GCR steps on levels 1..kcycle)
    against the least-squares restatement of the two steps."""
    grid, h, alpha, dt, cc = GRIDS[k]
    H, ops, ps, cols = _case(k, oracle.Params(coarsest_cells=cc, kcycle=kcycle))
    r = np.random.default_rng(7).standard_normal(ops[0].shape[0])
    ref = rf.vcycle_dense(ops, ps, cols, r, kcycle=kcycle)
    got = H.vcycle(r)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    if kcycle == 1:  # and it is not the plain V-cycle
        plain = rf.vcycle_dense(ops, ps, cols, r)
        assert np.linalg.norm(plain - ref) > 1e-6 * np.linalg.norm(ref)


# --------------------------------------------------------------------------
# planted mistakes: each must make a pin fail
# --------------------------------------------------------------------------

def _in_function(src, head, old, new):
    """Replace `old` (which must occur once) inside the function whose
    definition starts with `head`."""
    i = src.index(head)
    j = src.index("\n}\n", i)
    body = src[i:j]
    assert body.count(old) == 1, old
    return src[:i] + body.replace(old, new) + src[j:]


GS = "static void gs_sweep("
VC = "static void vcycle(const orc_hier *H, int l, const double *b, double *x) {"

MUTATIONS = {
    # point Gauss-Seidel: only the scalar diagonal is solved, the other two
    # components of the cell are taken from the previous iterate
    "point_gs": (GS, "if (j % n == k) d[c][j / n] += L->A.val[p];", "if (j == r) d[c][c] += L->A.val[p];"),
    # the backward sweep visits the colours in ascending order
    "backward_ascending": (GS, "int col = forward ? t : L->ncolours - 1 - t;", "int col = t;"),
    # the forward sweep visits the colours in descending order
    "forward_descending": (GS, "int col = forward ? t : L->ncolours - 1 - t;", "int col = L->ncolours - 1 - t;"),
    "no_pre_sweep": (VC, "s < H->prm.nu_pre;", "s < H->prm.nu_pre - 1;"),
    "no_post_sweep": (VC, "s < H->prm.nu_post;", "s < H->prm.nu_post - 1;"),
    # the coarse problem starts from its right-hand side instead of zero
    "nonzero_coarse_guess": (VC, "memset(x, 0, (size_t)nn * sizeof(double));",
                             "memcpy(x, b, (size_t)nn * sizeof(double));"),
    "residual_sign": (VC, "r[i] = b[i] - r[i];", "r[i] = r[i] - b[i];"),
}


KC = "static void kinner("

# mistakes in the K-cycle's two inner steps, caught by the K-cycle pin
KMUTATIONS = {
    # the second direction is dropped (one inner step)
    "kcycle_one_step": (KC, "double y2 = g22 > 0 ? a2 / g22 : 0.0", "double y2 = 0.0"),
    # the second image is not orthogonalised against the first
    "kcycle_no_orthogonalisation": (KC, "c2[i] -= g12 * c1[i];", "c2[i] -= 0.0 * c1[i];"),
}


SO = "static int step_order("
SG = "static void step_guess("

# mistakes in the time loop's initial approximation, caught by its closed-form
# pins (step_guess_violations in test_oracle_pins.py)
GMUTATIONS = {
    # the order stops at cubic
    "guess_cubic_cap": (SO, "j <= d && s2[j] < s2[j - 1]", "j <= d && j <= 3 && s2[j] < s2[j - 1]"),
    # every available term is taken, shrinking or not
    "guess_no_shrink_test": (SO, "j <= d && s2[j] < s2[j - 1]", "j <= d && s2[j] >= 0.0"),
    # the alternating signs of the extrapolation weights are lost
    "guess_weight_sign": (SG, "c[l] = (l % 2 ? -1.0 : 1.0) * b;", "c[l] = b;"),
    # C(k, l + 1) instead of C(k + 1, l + 1)
    "guess_binomial": (SG, "b = b * (double)(k + 1 - q) / (double)(q + 1);",
                       "b = b * (double)(k - q) / (double)(q + 1);"),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def _mutant(name, where):
    head, old, new = {**MUTATIONS, **KMUTATIONS, **GMUTATIONS}[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ll_oracle.c")).read()
    c = os.path.join(str(where), name + ".c")
    so = os.path.join(str(where), name + ".so")
    with open(c, "w") as f:
        f.write(_in_function(src, head, old, new))
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", so, c, "-lm"])
    return oracle.bind(ctypes.CDLL(so))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, mutant_dir):
    lib = _mutant(name, mutant_dir)
    saved = oracle._lib
    oracle._lib = lib
    try:
        sweep, cycle = [], []
        for k in range(len(GRIDS)):
            H, ops, ps, cols = _case(k)
            sweep.append(_sweep_errors(H, ops, cols))
            cycle.append(_vcycle_errors(H, ops, ps, cols))
            H.__del__()
    finally:
        oracle._lib = saved
    # a mistake in the sweep fails the sweep pin; every mistake fails the
    # V-cycle pin, on every grid
    if MUTATIONS[name][0] == GS:
        assert min(sweep) > 1e-6, sweep
    else:
        assert max(sweep) <= 1e-12, sweep
    assert min(cycle) > 1e-6, cycle


@pytest.mark.parametrize("name", sorted(KMUTATIONS))
def test_planted_kcycle_mistakes_are_caught(name, mutant_dir):
    lib = _mutant(name, mutant_dir)
    saved = oracle._lib
    oracle._lib = lib
    try:
        errs = []
        for k in (0, 2):
            grid, h, alpha, dt, cc = GRIDS[k]
            H, ops, ps, cols = _case(k, oracle.Params(coarsest_cells=cc, kcycle=1))
            r = np.random.default_rng(7).standard_normal(ops[0].shape[0])
            ref = rf.vcycle_dense(ops, ps, cols, r, kcycle=1)
            errs.append(np.linalg.norm(H.vcycle(r) - ref) / np.linalg.norm(ref))
            H.__del__()
    finally:
        oracle._lib = saved
    # far above the K-cycle pin's 1e-11 (the unorthogonalised second image
    # is nearly orthogonal to the first already, so that mistake moves the
    # result by a few 1e-8 only)
    assert min(errs) > 1e-9, errs


@pytest.mark.parametrize("name", sorted(GMUTATIONS))
def test_planted_step_guess_mistakes_are_caught(name, mutant_dir):
    from tests.test_oracle_pins import step_guess_violations

    lib = _mutant(name, mutant_dir)
    saved = oracle._lib
    oracle._lib = lib
    try:
        bad = step_guess_violations()
    finally:
        oracle._lib = saved
    assert bad, name
