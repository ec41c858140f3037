"""Batched solves of independent instances (ll_mg_batch_*), through the C ABI.

Each instance of a batch must give what a single solve gives: the same
hierarchy (aggregation per instance), a solution within 1e-10 of the FP64
oracle's for that instance and the same iteration count within one; the
float32 preconditioner path within 1e-8 of the float64 batch.  The
concatenated levels must hold exactly the instances' cells.
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

# ragged: 2-D and 3-D, odd sides (padding slots), different depths
SMALL = [
    {"grid": (16, 16, 1), "h": 1 / 16, "alpha": 0.1, "dt": 4.0 / 256, "kind": "smooth"},
    {"grid": (24, 20, 1), "h": 1 / 24, "alpha": 0.02, "dt": 1e-3, "kind": "vortex"},
    {"grid": (13, 7, 5), "h": 1 / 13, "alpha": 0.3, "dt": 1e-3, "kind": "smooth"},
    {"grid": (32, 32, 1), "h": 1 / 32, "alpha": 1.0, "dt": 1e-2, "kind": "smooth"},
    {"grid": (9, 9, 1), "h": 1 / 9, "alpha": 0.05, "dt": 1e-4, "kind": "smooth"},
    {"grid": (8, 8, 8), "h": 1 / 8, "alpha": 0.1, "dt": 8.0 / 64, "kind": "vortex"},
]
CC = 8


def _field(kind, grid, seed):
    if kind == "vortex":
        return inputs.vortex(*grid, seed=seed).reshape(-1)
    return inputs.smooth_field(*grid, seed=seed).reshape(-1)


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=DEV)


def _batch(cases, precision=ll.LL_FP64, rtol=1e-12, cc=CC, seed=0):
    ms = [_field(c.get("kind", "smooth"), c["grid"], seed + k) for k, c in enumerate(cases)]
    B = ll.Batch([_t(m) for m in ms], [c["alpha"] for c in cases], [c["dt"] for c in cases],
                 [c["h"] for c in cases], [c["grid"] for c in cases],
                 ll.Params(rtol=rtol, coarsest_cells=cc, precision=precision))
    return ms, B


def _solve(B, ms, cases, rtol=0.0):
    rhs = [_t(m / c["dt"]) for m, c in zip(ms, cases)]
    xs = [torch.zeros_like(r) for r in rhs]
    st, its, rrs, sts = B.solve(rhs, xs, rtol)
    return st, its, rrs, sts, [x.cpu().numpy() for x in xs]


def test_union_levels_hold_every_instance():
    ms, B = _batch(SMALL)
    singles = [ll.Hierarchy(_t(m), c["alpha"], c["dt"], c["h"], c["grid"], ll.Params(coarsest_cells=CC))
               for m, c in zip(ms, SMALL)]
    assert B.levels == max(H.levels for H in singles)
    for i, H in enumerate(singles):
        assert B.instance_levels(i) == H.levels
    rows0 = sum(2 * ((c["grid"][0] + 1) // 2) * c["grid"][1] * c["grid"][2] for c in SMALL)
    assert B.level_rows(0) == rows0  # red-black slots, padding included
    for l in range(1, B.levels):
        assert B.level_rows(l) == sum(H.level_cells(l) for H in singles if H.levels > l)


def test_batch_matches_oracle_per_instance():
    ms, B = _batch(SMALL)
    st, its, rrs, sts, xs = _solve(B, ms, SMALL)
    assert st == ll.LL_OK and all(s == ll.LL_OK for s in sts)
    for k, c in enumerate(SMALL):
        O = oracle.Hierarchy(c["grid"], c["h"], c["alpha"], c["dt"], ms[k],
                             oracle.Params(rtol=1e-12, coarsest_cells=CC))
        b = ms[k] / c["dt"]
        xo, sto, ito, rro = O.solve(b, np.zeros_like(b))
        assert sto == oracle.OK
        assert rrs[k] < 1e-12
        assert abs(its[k] - ito) <= 1, (k, its[k], ito)
        assert np.linalg.norm(xs[k] - xo) <= 1e-10 * np.linalg.norm(xo), k


def test_batch_matches_single_gpu_solves():
    ms, B = _batch(SMALL, rtol=1e-10)
    st, its, rrs, sts, xs = _solve(B, ms, SMALL)
    for k, c in enumerate(SMALL):
        H = ll.Hierarchy(_t(ms[k]), c["alpha"], c["dt"], c["h"], c["grid"],
                         ll.Params(rtol=1e-10, coarsest_cells=CC))
        x = torch.zeros(3 * int(np.prod(c["grid"])), dtype=torch.float64, device=DEV)
        s1, it1, rr1 = H.solve(_t(ms[k] / c["dt"]), x)
        assert abs(its[k] - it1) <= 1
        assert np.linalg.norm(xs[k] - x.cpu().numpy()) <= 1e-8 * np.linalg.norm(xs[k])


def test_mixed_precision_batch():
    ms, B64 = _batch(SMALL, rtol=1e-12)
    _, B32 = _batch(SMALL, precision=ll.LL_MIXED_FP32, rtol=1e-10)
    _, _, _, _, x64 = _solve(B64, ms, SMALL)
    st, its, rrs, sts, x32 = _solve(B32, ms, SMALL)
    assert st == ll.LL_OK and max(rrs) < 1e-10
    for a, b in zip(x32, x64):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)


def test_update_matches_fresh_batch():
    ms, B = _batch(SMALL, rtol=1e-11)
    ms2 = [_field("smooth", c["grid"], 100 + k) for k, c in enumerate(SMALL)]
    alphas = [c["alpha"] * 1.5 for c in SMALL]
    dts = [c["dt"] * 0.5 for c in SMALL]
    B.update([_t(m) for m in ms2], alphas, dts)
    cases2 = [dict(c, alpha=a, dt=d) for c, a, d in zip(SMALL, alphas, dts)]
    st, its, rrs, sts, xs = _solve(B, ms2, cases2)
    F = ll.Batch([_t(m) for m in ms2], alphas, dts, [c["h"] for c in SMALL], [c["grid"] for c in SMALL],
                 ll.Params(rtol=1e-11, coarsest_cells=CC))
    st2, its2, rrs2, sts2, xs2 = _solve(F, ms2, cases2)
    assert its == its2
    for a, b in zip(xs, xs2):
        assert np.array_equal(a, b)  # same arithmetic in the same order


def test_compaction_is_invisible(monkeypatch):
    """Compacting the still-iterating instances into sub-batches at restart
    boundaries changes nothing: iterations, residuals and solutions are
    bit-identical to the lockstep solve of the whole batch."""
    cases = SMALL + [dict(c, alpha=c["alpha"] * 0.3, dt=c["dt"] * 3) for c in SMALL[:3]]
    ms, B = _batch(cases, rtol=1e-12)
    monkeypatch.setenv("LLMG_BATCH_NO_COMPACT", "1")
    st1, its1, rrs1, sts1, xs1 = _solve(B, ms, cases)
    assert B.subbatches == 0
    monkeypatch.delenv("LLMG_BATCH_NO_COMPACT")
    st2, its2, rrs2, sts2, xs2 = _solve(B, ms, cases)
    assert B.subbatches >= 1
    assert its1 == its2 and sts1 == sts2 and rrs1 == rrs2
    for a, b in zip(xs1, xs2):
        assert np.array_equal(a, b)
    st3, its3, rrs3, sts3, xs3 = _solve(B, ms, cases)  # the cached sub-batches again
    assert its3 == its2 and all(np.array_equal(a, b) for a, b in zip(xs3, xs2))


def test_zero_rhs_instance_and_guess():
    ms, B = _batch(SMALL[:3], rtol=1e-10)
    rhs = [_t(ms[0] / SMALL[0]["dt"]), torch.zeros(3 * int(np.prod(SMALL[1]["grid"])), dtype=torch.float64,
                                                    device=DEV), _t(ms[2] / SMALL[2]["dt"])]
    xs = [torch.zeros_like(r) for r in rhs]
    xs[1] += 1.0  # a non-zero guess for the zero right-hand side
    st, its, rrs, sts = B.solve(rhs, xs)
    assert st == ll.LL_OK and sts == [ll.LL_OK] * 3
    assert float(xs[1].abs().max()) == 0.0 and its[1] == 0
    # a converged guess needs no iteration
    st, its2, rrs2, sts2 = B.solve(rhs, xs)
    assert its2[0] == 0 and its2[2] == 0


def test_invalid_batches():
    ms = [_t(_field("smooth", c["grid"], k)) for k, c in enumerate(SMALL[:2])]
    args = ([c["alpha"] for c in SMALL[:2]], [c["dt"] for c in SMALL[:2]], [c["h"] for c in SMALL[:2]],
            [c["grid"] for c in SMALL[:2]])
    for p in (ll.Params(kcycle=1, coarsest_cells=CC), ll.Params(precision=ll.LL_MIXED_BF16, coarsest_cells=CC)):
        with pytest.raises(ll.LLError):
            ll.Batch(ms, *args, params=p)
    with pytest.raises(ll.LLError):  # the 16x16 instance cannot coarsen below 1000 cells
        ll.Batch(ms, *args, params=ll.Params(coarsest_cells=1000))


def test_ragged_batch_sampled_against_oracle():
    """64 instances of the ragged recipe (sides 32..64, alpha and dt
    log-uniform): every instance reaches rtol by its true residual or reports
    otherwise, and three sampled instances match the oracle."""
    spec = inputs.batch_instances(64, seed=3, sides=(32, 48, 64))
    cases = [{"grid": s["grid"], "h": s["h"], "alpha": s["alpha"], "dt": s["dt"]} for s in spec]
    ms = [inputs.smooth_field(*s["grid"], seed=s["seed"]).reshape(-1) for s in spec]
    B = ll.Batch([_t(m) for m in ms], [c["alpha"] for c in cases], [c["dt"] for c in cases],
                 [c["h"] for c in cases], [c["grid"] for c in cases], ll.Params(rtol=1e-8, maxit=400))
    st, its, rrs, sts, xs = _solve(B, ms, cases)
    for k in range(len(cases)):
        if sts[k] == ll.LL_OK:
            assert rrs[k] < 1e-8
        else:
            assert sts[k] in (ll.LL_NOT_CONVERGED, ll.LL_BREAKDOWN)
    ok = [k for k in range(len(cases)) if sts[k] == ll.LL_OK]
    assert len(ok) >= len(cases) // 2
    for k in ok[:3]:
        c = cases[k]
        O = oracle.Hierarchy(c["grid"], c["h"], c["alpha"], c["dt"], ms[k], oracle.Params(rtol=1e-8, maxit=400))
        b = ms[k] / c["dt"]
        xo, sto, ito, rro = O.solve(b, np.zeros_like(b))
        assert sto == oracle.OK and abs(its[k] - ito) <= 1
        # both stop at relres < 1e-8: the solutions agree to the stopping level
        assert np.linalg.norm(xs[k] - xo) <= 1e-6 * np.linalg.norm(xo)
