"""Host-side logic of the batch autotuner, no GPU needed: the class octave
of dt/h^2 and the reading of its plain-text cache (exact class match,
precision kept apart, malformed lines and invalid parameter sets ignored)."""
from __future__ import annotations

import math

import pytest

import paper_2608_09102_b300 as ll
from paper_2608_09102_b300 import build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return ll.load_library()


@pytest.mark.parametrize("dt,h", [(1e-3, 1 / 64), (5e-4, 1 / 128), (1e-5, 1 / 32), (1e-2, 1 / 256), (0.25, 0.5)])
def test_octave_is_floor_log2_of_dt_over_h2(dt, h):
    assert ll.tune_octave(dt, h) == math.floor(math.log2(dt / (h * h)))


def test_octave_rejects_bad_input():
    assert ll.tune_octave(0.0, 0.1) < -2 ** 30
    assert ll.tune_octave(1e-3, -1.0) < -2 ** 30


def test_cache_lookup(tmp_path):
    path = tmp_path / "tune.txt"
    o = ll.tune_octave(1e-3, 1 / 64)  # 2
    path.write_text(
        "# comment line\n"
        "llmg-tune-v1 0 64 64 1 %d 2 2 1 8 128 3.5\n" % o
        + "llmg-tune-v1 1 64 64 1 %d 1 1 0 0 0 2.0\n" % o  # float32 preconditioner class
        + "llmg-tune-v1 0 48 48 1 %d 9 9 0 0 0 1.0\n" % o  # nine sweeps: a valid choice
        + "llmg-tune-v1 0 32 32 1 %d 1 1 0 5 0 1.0\n" % o  # invalid lanes: ignored
        + "llmg-tune-v1 0 96 96 1\n"  # malformed: ignored
        + "other-tag 0 128 128 1 %d 2 2 0 0 0 1.0\n" % o)  # another tag: ignored
    base = ll.Params(rtol=1e-9, maxit=77)
    got = ll.tune_lookup(str(path), (64, 64, 1), 1e-3, 1 / 64, base)
    assert (got.nu_pre, got.nu_post, got.kcycle, got.coarse_lanes, got.coarse_block) == (2, 2, 1, 8, 128)
    assert (got.rtol, got.maxit) == (1e-9, 77)  # the rest of base is kept
    mixed = ll.tune_lookup(str(path), (64, 64, 1), 1e-3, 1 / 64, ll.Params(precision=ll.LL_MIXED_FP32))
    assert (mixed.nu_pre, mixed.kcycle) == (1, 0)
    assert ll.tune_lookup(str(path), (64, 64, 1), 4e-3, 1 / 64, base) is None  # another octave
    assert ll.tune_lookup(str(path), (64, 64, 2), 1e-3, 1 / 64, base) is None  # another grid
    assert ll.tune_lookup(str(path), (48, 48, 1), 1e-3, 1 / 64, base).nu_pre == 9
    assert ll.tune_lookup(str(path), (32, 32, 1), 1e-3, 1 / 64, base) is None
    assert ll.tune_lookup(str(path), (128, 128, 1), 1e-3, 1 / 64, base) is None
    assert ll.tune_lookup(str(tmp_path / "absent.txt"), (64, 64, 1), 1e-3, 1 / 64, base) is None
