"""Host-side accounting of the benchmark (CPU only): the ray-step count
behind the viewshed roofline, the greedy loop's byte count, and the rule that
recorded ncu counters are used only for the source they were measured on."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench


@pytest.mark.parametrize("R,lo,hi", [(50, 6.95, 6.99), (100, 6.99, 7.03), (200, 7.01, 7.05)])
def test_interior_ray_steps_about_7_R2(R, lo, hi):
    """Rays to the 8R ring cells cut at the disc take ~7.0 R^2 steps."""
    assert lo * R * R <= bench.interior_ray_steps(R) <= hi * R * R


def test_interior_ray_steps_brute_force():
    """Against a direct walk of every ring ray (R small)."""
    for R in (1, 2, 3, 7, 12):
        n = 0
        for ex, ey in ([(R, e) for e in range(-R + 1, R + 1)] + [(e, R) for e in range(-R, R)] +
                       [(-R, e) for e in range(-R, R)] + [(e, -R) for e in range(-R + 1, R + 1)]):
            dmin = ey if abs(ex) >= abs(ey) else ex
            for k in range(1, R + 1):
                a = (2 * abs(k * dmin) + R) // (2 * R)
                if k * k + a * a > R * R:
                    break
                n += 1
        assert bench.interior_ray_steps(R) == n


def test_site_loop_bytes_isolated_winners():
    """Winners far apart: each step moves its own window (V and C read, C
    written) and refreshes nobody."""
    W, R, PR = 10000, 10, 2
    cand = np.array([0 * W + 100, 5000 * W + 5000, 9000 * W + 200], np.int64)
    words = (2 * R + 1) * PR
    assert bench.site_loop_bytes(cand, cand[:2], W, R, PR) == 2 * 3 * words * 4


def test_recorded_counters_follow_the_source(tmp_path, monkeypatch):
    """Per-unit counters from the mid-workload capture are used only while
    the kernel's source file is the one they were measured on."""
    root = tmp_path
    (root / "profiles").mkdir()
    src = root / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()
    rec = {"kernels": {"viewshed": {"thread_inst_per_unit": 63.5, "dram_bytes_per_unit": 0.5,
                                    "issue_active_pct": 76.0, "source": "k.cu", "sha1": sha},
                       "vix": {"thread_inst_per_unit": 29.0, "dram_bytes_per_unit": 0.01,
                               "issue_active_pct": 68.0, "source": "k.cu", "sha1": "0" * 40}}}
    (root / "profiles" / "counters_mid_11600sq_R100.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "__file__", str(root / "bench.py"))
    got = bench.recorded_counters()
    assert got["viewshed"]["thread_inst_per_unit"] == 63.5
    assert "vix" not in got                       # another source than the one measured
    src.write_text("__global__ void k() { }\n")   # the kernel changed
    assert bench.recorded_counters() == {}


def test_committed_counters_record():
    """The committed capture's per-unit figures are consistent with its raw counts."""
    rec = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles",
                                      "counters_mid_11600sq_R100.json")))
    for k, r in rec["kernels"].items():
        assert r["units"] > 0
        assert abs(r["dram_bytes_per_unit"] - r["dram_bytes"] / r["units"]) < 1e-9 * max(r["dram_bytes_per_unit"], 1)
        if "thread_inst" in r:  # the instruction captures (the forward's entry records traffic only)
            assert abs(r["thread_inst_per_unit"] - r["thread_inst"] / r["units"]) < 1e-9 * r["thread_inst_per_unit"]
            assert 0 < r["issue_active_pct"] <= 100


def test_cnn_flops_match_the_oracle():
    """The bench's FLOP count per patch (used for the tensor roofline) is the
    oracle's: 2 * outputs * 9 * cin * 32 per convolution plus the fc layer."""
    from oracle import cnn_oracle as C
    assert bench.cnn_flops_per_patch() == C.flops_per_patch() == 8368768
