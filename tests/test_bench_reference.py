"""The benchmark's reference arm runs on the CPU alone: the FP64 oracle on
whole time steps of the bounded sample (the central 48^3 block of the 128^3
workload field), one JSON line with its measured step time, the all-core
replica throughput and the host's core count."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_line():
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "unknown-solves/s" and d["higher_is_better"] is True
    # value = unknowns of the sample per measured second of a whole step
    assert abs(d["value"] - 3 * 48 ** 3 / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["all_cores"]["cores"] >= 1 and d["nproc"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert 30 <= d["iterations_per_step"]["mean"] <= 45


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=120, env=env, cwd=ROOT)
    assert out.returncode == 0 and "{" not in out.stdout


def test_other_workloads_record_a_failing_leg(monkeypatch):
    """A workload of the list whose library call fails is recorded with the
    error (the status and the failing CUDA call) and the others still run,
    so that the bench line is printed."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_2608_09102_b300 as ll

    class _Cuda:
        @staticmethod
        def synchronize():
            pass

        @staticmethod
        def empty_cache():
            pass

    class _Torch:
        cuda = _Cuda

    ran = []

    def ok(name):
        def leg(ll_, torch, inputs, dev):
            ran.append(name)
            return {"ran": name}
        return leg

    def fails(ll_, torch, inputs, dev):
        ran.append("config4")
        raise ll.LLError(ll.LL_ECUDA, "ll_mg_batch_update")

    monkeypatch.setattr(bench, "_leg_config1", ok("config1"))
    monkeypatch.setattr(bench, "_leg_config3", ok("config3"))
    monkeypatch.setattr(bench, "_leg_config4", fails)
    monkeypatch.setattr(bench, "_leg_config5", ok("config5"))
    out = bench.other_workloads(ll, _Torch, None, None)
    assert ran == ["config1", "config3", "config4", "config5"]
    assert "ll_mg_batch_update failed: CUDA runtime error" in out["config4_batch512_mixed_autotuned"]["error"]
    assert out["config5_grad96_fp64"] == {"ran": "config5"}
