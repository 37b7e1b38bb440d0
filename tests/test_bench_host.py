"""Host-side parts of bench.py, on CPU: the workload shapes the bench line
names, the algorithmic byte and flop counts its roofline and paper-style
Gflop/s rest on (checked against values worked out by hand), launch-plan
parsing, and the reference arm's JSON line (the FP64 oracle on the host
cores, run here on the small raider-like workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("config,N,T,k,vlo,vhi", [
    (1, 16, 1000, 50, 20000, 60000),      # greeneyes-like
    (3, 8, 3500, 100, 600000, 600000),    # forrest-like
    (4, 1024, 500, 50, 20000, 60000),     # forrest-1024-like (the headline)
])
def test_workload_shapes(config, N, T, k, vlo, vhi):
    spec, vox = bench.workload(config, 0)
    assert (spec.n_subjects, spec.T, spec.k) == (N, T, k)
    assert len(vox) == N
    assert min(vox) >= vlo and max(vox) <= vhi
    # the same draw every time (the bench line and the parity tests name it)
    assert list(bench.workload(config, 0)[1]) == list(vox)


def test_workload_overrides():
    spec, vox = bench.workload(4, 0)
    s2, v2 = bench.workload(4, 0, subjects=64)
    assert s2.n_subjects == 64 and list(v2) == list(vox[:64]) and "first 64 subjects" in s2.name
    s3, v3 = bench.workload(4, 0, voxels_cap=25000)
    assert max(v3) == 25000 and all(a == min(b, 25000) for a, b in zip(v3, vox))
    s4, v4 = bench.workload(4, 0, k=100)
    assert s4.k == 100 and list(v4) == list(vox) and s4.T == spec.T


def test_headline_total_voxels():
    # the forrest-1024-like voxel total that the bench line and the profiles quote
    assert sum(bench.workload(4, 0)[1]) == 40640984


def test_algorithmic_bytes_by_hand():
    vox = [3, 5]
    # two passes: each reads X^ (8 voxels x T = 7 x 2 B) and moves A_i (8 x k = 2 x 4 B)
    e, m = bench.algorithmic_bytes(vox, 7, 2, 2, 4)
    assert e == m == 8 * 7 * 2 + 8 * 2 * 4
    # single pass: X^ once, A_i written once
    assert bench.single_pass_bytes(vox, 7, 2, 2, 4) == 8 * 7 * 2 + 8 * 2 * 4
    # the headline pass: 40,640,984 voxels x (500 x 2 + 50 x 2) bytes
    vox4 = bench.workload(4, 0)[1]
    assert bench.single_pass_bytes(vox4, 500, 50, 2, 2) == 44705082400.0


def test_paper_flops_by_hand():
    # Sec. V-A: 2 (2 v T k) + 2 v k^2 + (2 v k^2 - 2/3 k^3) per subject
    v, T, k = 10, 4, 3
    want = 2 * (2 * v * T * k) + 2 * v * k * k + (2 * v * k * k - 2.0 / 3.0 * k ** 3)
    assert bench.paper_flops([v], T, k) == pytest.approx(want, rel=0, abs=1e-9)
    assert bench.paper_flops([v, v], T, k) == pytest.approx(2 * want, rel=0, abs=1e-9)


def test_parse_plan():
    assert bench.parse_plan("single_pass=1, f_slots=9,f_first_stages=4") == {
        "single_pass": 1, "f_slots": 9, "f_first_stages": 4}
    assert bench.parse_plan("") == {}


def test_reference_arm_json_line():
    """`bench.py --impl reference` prints one JSON line for the oracle on the
    host cores, on our arm's metric and unit, with at least 3 warm-up steps
    whatever is asked, and an e2e block that moves no bytes."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "0",
                        "--steps", "2", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "EM iterations/s" and d["higher_is_better"] is True
    assert d["metric"].startswith("pSRM EM iterations/s")
    assert d["steps"] == 2 and d["warmup"] >= 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["dtype"] == "f64"
    assert d["config"]["N"] == 4 and d["config"]["T"] == 300 and d["config"]["k"] == 10
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
