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


def _batch(cases, precision=ll.LL_FP64, rtol=1e-12, cc=CC, seed=0, kcycle=0):
    ms = [_field(c.get("kind", "smooth"), c["grid"], seed + k) for k, c in enumerate(cases)]
    B = ll.Batch([_t(m) for m in ms], [c["alpha"] for c in cases], [c["dt"] for c in cases],
                 [c["h"] for c in cases], [c["grid"] for c in cases],
                 ll.Params(rtol=rtol, coarsest_cells=cc, precision=precision, kcycle=kcycle))
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
    boundaries changes each instance's arithmetic by rounding only (a
    sub-batch's smaller union may run a level in the cluster kernel that the
    whole batch runs as per-class launches): same statuses, iterations within
    one, solutions within 1e-10 of the lockstep solve of the whole batch
    where they converge; where an instance stagnates at maxit, its final
    residual (near 1, after hundreds of iterations that amplify rounding)
    within 1e-3.  A second solve reuses the sub-batches and repeats the first
    bit for bit."""
    cases = SMALL + [dict(c, alpha=c["alpha"] * 0.3, dt=c["dt"] * 3) for c in SMALL[:3]]
    ms, B = _batch(cases, rtol=1e-12)
    monkeypatch.setenv("LLMG_BATCH_NO_COMPACT", "1")
    st1, its1, rrs1, sts1, xs1 = _solve(B, ms, cases)
    assert B.subbatches == 0
    monkeypatch.delenv("LLMG_BATCH_NO_COMPACT")
    st2, its2, rrs2, sts2, xs2 = _solve(B, ms, cases)
    assert B.subbatches >= 1
    assert sts1 == sts2
    for k in range(len(cases)):
        assert abs(its1[k] - its2[k]) <= 1, (k, its1[k], its2[k])
        if sts1[k] == ll.LL_OK:
            assert rrs1[k] < 1e-12 and rrs2[k] < 1e-12
            assert np.linalg.norm(xs1[k] - xs2[k]) <= 1e-10 * np.linalg.norm(xs1[k]), k
        else:
            assert abs(rrs1[k] - rrs2[k]) <= 1e-3 * rrs1[k], (k, rrs1[k], rrs2[k])
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
    for p in (ll.Params(coarse_lanes=5, coarsest_cells=CC), ll.Params(precision=ll.LL_MIXED_BF16, coarsest_cells=CC)):
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


# ---------------------------------------------------------------------------
# the K-cycle in a batch, per-instance parameters (groups), the autotuner
# ---------------------------------------------------------------------------

def _oracle_solve(c, m, **kw):
    O = oracle.Hierarchy(c["grid"], c["h"], c["alpha"], c["dt"], m, oracle.Params(**kw))
    b = m / c["dt"]
    return O.solve(b, np.zeros_like(b))


@pytest.mark.parametrize("kcycle", [1, 2])
def test_kcycle_batch_matches_oracle_per_instance(kcycle):
    """The K-cycle on levels 1..kcycle of every instance, with each
    instance's own inner-step scalars: the oracle's K-cycle solve per
    instance (1e-10, iterations within one)."""
    ms, B = _batch(SMALL, kcycle=kcycle)
    st, its, rrs, sts, xs = _solve(B, ms, SMALL)
    assert st == ll.LL_OK
    for k, c in enumerate(SMALL):
        xo, sto, ito, rro = _oracle_solve(c, ms[k], rtol=1e-12, coarsest_cells=CC, kcycle=kcycle)
        assert sto == oracle.OK and rrs[k] < 1e-12
        assert abs(its[k] - ito) <= 1, (k, its[k], ito)
        assert np.linalg.norm(xs[k] - xo) <= 1e-10 * np.linalg.norm(xo), k


def test_kcycle_mixed_batch():
    ms, B64 = _batch(SMALL, rtol=1e-12, kcycle=1)
    _, B32 = _batch(SMALL, precision=ll.LL_MIXED_FP32, rtol=1e-10, kcycle=1)
    _, _, _, _, x64 = _solve(B64, ms, SMALL)
    st, its, rrs, sts, x32 = _solve(B32, ms, SMALL)
    assert st == ll.LL_OK and max(rrs) < 1e-10
    for a, b in zip(x32, x64):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)


# instances of the 512-instance recipe (seed 0) where V(1,1) stagnates
# (48^2, alpha 0.012, dt/h^2 18.9; 64^2, alpha 0.006, dt/h^2 39.2, where
# V(2,2) stagnates too and only the K-cycle converges) and two where it
# converges (64^2, dt/h^2 14.6; 96^2, dt/h^2 24.2): four tuning classes
HARD = [229, 196, 211, 80]


def _recipe(idx):
    spec = inputs.batch_instances(512, seed=0)
    cases = [{"grid": spec[k]["grid"], "h": spec[k]["h"], "alpha": spec[k]["alpha"], "dt": spec[k]["dt"]}
             for k in idx]
    ms = [inputs.smooth_field(*spec[k]["grid"], seed=spec[k]["seed"]).reshape(-1) for k in idx]
    return cases, ms


def _solve_from_guess(B, ms, cases, rtol=0.0):
    rhs = [_t(m / c["dt"]) for m, c in zip(ms, cases)]
    xs = [_t(m) for m in ms]
    st, its, rrs, sts = B.solve(rhs, xs, rtol)
    return st, its, rrs, sts, [x.cpu().numpy() for x in xs]


def test_groups_run_each_instance_with_its_parameters():
    """Per-instance parameters: instances with equal parameters share a
    group; every instance matches the oracle solve with its own cycle."""
    cycles = [dict(), dict(nu_pre=2, nu_post=2), dict(kcycle=1), dict(kcycle=1, nu_pre=2, nu_post=2)]
    per = [cycles[k % 4] for k in range(len(SMALL))]
    ms = [_field(c.get("kind", "smooth"), c["grid"], k) for k, c in enumerate(SMALL)]
    args = ([_t(m) for m in ms], [c["alpha"] for c in SMALL], [c["dt"] for c in SMALL], [c["h"] for c in SMALL],
            [c["grid"] for c in SMALL])
    B = ll.Batch(*args, params=[ll.Params(rtol=1e-12, coarsest_cells=CC, **kw) for kw in per])
    assert B.groups == 4
    assert [B.instance_group(k) for k in range(len(SMALL))] == [k % 4 for k in range(len(SMALL))]
    st, its, rrs, sts, xs = _solve(B, ms, SMALL)
    assert st == ll.LL_OK
    for k, c in enumerate(SMALL):
        xo, sto, ito, rro = _oracle_solve(c, ms[k], rtol=1e-12, coarsest_cells=CC, **per[k])
        assert sto == oracle.OK and abs(its[k] - ito) <= 1, (k, its[k], ito)
        assert np.linalg.norm(xs[k] - xo) <= 1e-10 * np.linalg.norm(xo), k
    # a single parameter set gives a plain batch
    assert ll.Batch(*args, params=[ll.Params(coarsest_cells=CC)] * len(SMALL)).groups == 1


def test_autotuner_rescues_the_stagnating_instances(tmp_path):
    """The autotuner times each class's candidates on its instances: the
    classes where V(1,1) stagnates get a cycle that converges, choices go to
    the cache and are reused, and the tuned batch converges everywhere with
    each instance matching the oracle run with its chosen cycle."""
    cases, ms = _recipe(HARD)
    args = ([_t(m) for m in ms], [c["alpha"] for c in cases], [c["dt"] for c in cases], [c["h"] for c in cases],
            [c["grid"] for c in cases])
    base = ll.Params(rtol=1e-8, maxit=300)
    plain = ll.Batch(*args, params=base)
    st, its, rrs, sts, xs = _solve_from_guess(plain, ms, cases)
    assert sts[0] != ll.LL_OK and sts[1] != ll.LL_OK  # V(1,1) stagnates on the first two
    cache = str(tmp_path / "tune.txt")
    chosen, tuned = ll.autotune(*args, base=base, cache_path=cache)
    assert tuned == 4
    lines = [ln for ln in open(cache) if ln.startswith("llmg-tune-v1")]
    assert len(lines) == 4
    for k in (0, 1):
        assert (chosen[k].nu_pre, chosen[k].kcycle) != (1, 0)
    assert chosen[1].kcycle == 1
    for p in chosen:
        assert (p.rtol, p.maxit) == (base.rtol, base.maxit)
    again, tuned2 = ll.autotune(*args, base=base, cache_path=cache)
    assert tuned2 == 0 and again == chosen
    for k, c in enumerate(cases):
        assert ll.tune_lookup(cache, c["grid"], c["dt"], c["h"], base) == chosen[k]
    B = ll.Batch(*args, params=chosen)
    st, its, rrs, sts, xs = _solve_from_guess(B, ms, cases)
    assert st == ll.LL_OK and all(r < 1e-8 for r in rrs)
    for k, c in enumerate(cases):
        p = chosen[k]
        O = oracle.Hierarchy(c["grid"], c["h"], c["alpha"], c["dt"], ms[k],
                             oracle.Params(rtol=1e-8, maxit=300, nu_pre=p.nu_pre, nu_post=p.nu_post, kcycle=p.kcycle))
        xo, sto, ito, rro = O.solve(ms[k] / c["dt"], ms[k].copy())
        assert sto == oracle.OK and abs(its[k] - ito) <= 1, (k, its[k], ito)
        assert np.linalg.norm(xs[k] - xo) <= 1e-6 * np.linalg.norm(xo)


def test_union_tail_matches_per_class_launches(monkeypatch):
    """The union's small levels in one cluster kernel (with every instance's
    dense solve at its own coarsest level) against the same levels as
    per-class launches: same iterations within one, solutions within 1e-10."""
    spec = inputs.batch_instances(24, seed=5, sides=(32, 48, 64, 96))
    cases = [{"grid": s["grid"], "h": s["h"], "alpha": s["alpha"], "dt": s["dt"]} for s in spec]
    ms = [inputs.smooth_field(*s["grid"], seed=s["seed"]).reshape(-1) for s in spec]
    args = ([_t(m) for m in ms], [c["alpha"] for c in cases], [c["dt"] for c in cases], [c["h"] for c in cases],
            [c["grid"] for c in cases])
    p = ll.Params(rtol=1e-12, maxit=400)
    B = ll.Batch(*args, params=p)
    monkeypatch.setenv("LLMG_NO_TAIL", "1")
    N = ll.Batch(*args, params=p)
    monkeypatch.delenv("LLMG_NO_TAIL")
    st1, its1, rrs1, sts1, xs1 = _solve(B, ms, cases)
    st2, its2, rrs2, sts2, xs2 = _solve(N, ms, cases)
    assert sts1 == sts2
    for k in range(len(cases)):
        assert abs(its1[k] - its2[k]) <= 1, (k, its1[k], its2[k])
        if sts1[k] == ll.LL_OK:
            assert np.linalg.norm(xs1[k] - xs2[k]) <= 1e-10 * np.linalg.norm(xs2[k]), k


def test_groups_with_different_coarsest_sizes_update_repeatedly():
    """Groups run on host threads of their own, and every instance's numeric
    setup ends with the coarsest inverse, whose shared memory depends on the
    coarsest size.  Groups of different coarsest sizes updated many times
    over must each succeed and leave the solves unchanged."""
    cases = [{"grid": (16 + 8 * (k % 3), 16, 1), "h": 1 / 16, "alpha": 0.1, "dt": 2e-3, "kind": "smooth"}
             for k in range(24)]
    sizes = [8, 24, 48, 84]  # coarsest cells: 24 to 252 unknowns
    per = [ll.Params(rtol=1e-10, coarsest_cells=sizes[k % 4], nu_pre=1 + (k // 4) % 2) for k in range(len(cases))]
    ms = [_field("smooth", c["grid"], k) for k, c in enumerate(cases)]
    mt = [_t(m) for m in ms]
    al, dts = [c["alpha"] for c in cases], [c["dt"] for c in cases]
    B = ll.Batch(mt, al, dts, [c["h"] for c in cases], [c["grid"] for c in cases], params=per)
    assert B.groups == 8
    st0, its0, _, _, xs0 = _solve(B, ms, cases)
    assert st0 == ll.LL_OK
    for _ in range(40):
        B.update(mt, al, dts)
    st, its, _, _, xs = _solve(B, ms, cases)
    assert st == ll.LL_OK and its == its0
    for a, b in zip(xs, xs0):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [ll.LL_FP64, ll.LL_MIXED_FP32])
def test_stagnation_stop_single_and_batch(precision):
    """The optional stagnation stop (stall_window 20, stall_ratio 0.99): two
    2-D instances whose V-cycle-preconditioned GCR makes no progress (large
    dt/h^2, small alpha) stop at the restart after 20 iterations, as the
    oracle's solve with the same stop does, in a single solve and in a batch
    next to converging instances; the converging instances still match the
    oracle within 1e-10 (float32 V-cycle: 1e-8, the mixed path's bound), and
    their iterations equal those of the same batch without the stop within
    one."""
    tol = 1e-10 if precision == ll.LL_FP64 else 1e-8
    # with the float32 V-cycle, GCR on the stagnating instances may also end
    # in a breakdown (a zero or non-finite image) before the stop's restart
    bad = (ll.LL_NOT_CONVERGED,) if precision == ll.LL_FP64 else (ll.LL_NOT_CONVERGED, ll.LL_BREAKDOWN)

    def stopped(st, it):
        return st in bad and it <= 20 and (st != ll.LL_NOT_CONVERGED or it == 20)
    stag = [{"grid": (64, 64, 1), "h": 1 / 64, "alpha": 0.01, "dt": 300 / 64 ** 2, "kind": "smooth"},
            {"grid": (48, 48, 1), "h": 1 / 48, "alpha": 0.02, "dt": 200 / 48 ** 2, "kind": "smooth"}]
    cases = stag + SMALL[:4]
    stall = dict(stall_window=20, stall_ratio=0.99)
    ms = [_field(c["kind"], c["grid"], 5 + k) for k, c in enumerate(cases)]
    oracle_out = [_oracle_solve(c, m, rtol=1e-10, maxit=200, coarsest_cells=CC, **stall) for c, m in zip(cases, ms)]
    for k in range(2):
        assert oracle_out[k][1] == oracle.NOT_CONVERGED and oracle_out[k][2] == 20
    for k in range(2, len(cases)):
        assert oracle_out[k][1] == oracle.OK
    # single solve
    c, m = stag[0], ms[0]
    H = ll.Hierarchy(_t(m), c["alpha"], c["dt"], c["h"], c["grid"],
                     ll.Params(rtol=1e-10, maxit=200, coarsest_cells=CC, precision=precision, **stall))
    x = torch.zeros(3 * int(np.prod(c["grid"])), dtype=torch.float64, device=DEV)
    st, it, rr = H.solve(_t(m / c["dt"]), x)
    assert stopped(st, it), (st, it)
    if st == ll.LL_NOT_CONVERGED:
        assert abs(rr - oracle_out[0][3]) <= 1e-3
    # batch, with and without the stop
    args = ([_t(m) for m in ms], [c["alpha"] for c in cases], [c["dt"] for c in cases], [c["h"] for c in cases],
            [c["grid"] for c in cases])
    out = {}
    for key, kw in (("stall", stall), ("plain", {})):
        B = ll.Batch(*args, ll.Params(rtol=1e-10, maxit=200, coarsest_cells=CC, precision=precision, **kw))
        out[key] = _solve(B, ms, cases)
    st, its, rrs, sts, xs = out["stall"]
    _, its_p, _, sts_p, _ = out["plain"]
    for k in range(2):
        assert stopped(sts[k], its[k]) and sts_p[k] in bad, (k, sts[k], its[k], sts_p[k])
        if sts_p[k] == ll.LL_NOT_CONVERGED:
            assert its_p[k] == 200
        if sts[k] == ll.LL_NOT_CONVERGED:
            assert abs(rrs[k] - oracle_out[k][3]) <= 1e-3
    for k in range(2, len(cases)):
        xo, sto, ito, rro = oracle_out[k]
        assert sts[k] == ll.LL_OK and abs(its[k] - its_p[k]) <= 1, (k, its[k], its_p[k])
        if precision == ll.LL_FP64:
            assert abs(its[k] - ito) <= 1, (k, its[k], ito)
        assert np.linalg.norm(xs[k] - xo) <= tol * np.linalg.norm(xo), k
