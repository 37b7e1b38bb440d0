"""The committed ncu summaries that bench.py reads its `roofline.traffic`
from: every summary that carries DRAM traffic names an existing kernel
source and a 40-hex SHA-1, and the bench's lookups return that traffic while
the source is unchanged, or None with a note saying it is stale."""
import glob
import hashlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1608_04647_gb300", "csrc")
SUMMARIES = sorted(p for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))
                   if "traffic_bytes_per_launch" in open(p).read())


def _fields(path):
    text = open(path).read()
    mt = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    ms = re.search(r"source_sha1: ([0-9a-f]{40}) \(([\w.]+) when captured\)", text)
    return text, mt, ms


def test_there_are_traffic_summaries():
    names = [os.path.basename(p) for p in SUMMARIES]
    assert any(n.startswith("mstep_tc_") for n in names)
    assert any(n.startswith("htfa_residual_") for n in names)


@pytest.mark.parametrize("path", SUMMARIES, ids=lambda p: os.path.basename(p))
def test_summary_format(path):
    text, mt, ms = _fields(path)
    assert mt and int(mt.group(1)) > 0
    assert ms, "a traffic summary must record the SHA-1 of the kernel source it was captured from"
    assert os.path.exists(os.path.join(CSRC, ms.group(2)))
    assert "--clock-control none" in text, "every ncu command must leave the clocks alone"


def _current(ms):
    return hashlib.sha1(open(os.path.join(CSRC, ms.group(2)), "rb").read()).hexdigest() == ms.group(1)


def test_htfa_lookup_matches_the_summary():
    import bench
    path = os.path.join(ROOT, "profiles", "htfa_residual_greeneyes_subsampled_like_N40_T174_V6857_K100.md")
    _, mt, ms = _fields(path)
    traffic, src = bench.htfa_profiled_traffic("htfa_residual", "greeneyes-subsampled-like")
    if _current(ms):
        assert traffic == int(mt.group(1)) and src.endswith(os.path.basename(path))
        # DRAM traffic close to the algorithmic bytes 4 (nTV + nKV + nTK)
        n, T, V, K = 40, 174, 6857, 100
        assert 0.95 <= traffic / (4 * (n * T * V + n * K * V + n * T * K)) <= 1.2
    else:
        assert traffic is None and "stale" in src
    assert bench.htfa_profiled_traffic("htfa_residual", "no-such-workload") == (None, None)


def test_srm_lookup_matches_the_summary():
    import bench
    path = os.path.join(ROOT, "profiles", "mstep_tc_greeneyes_like_N16_T1000_k50.md")
    _, mt, ms = _fields(path)
    traffic, src = bench.profiled_traffic("mstep_tc", 1, 10 ** 6)
    if _current(ms):
        assert traffic is not None and src.startswith(os.path.join("profiles", "mstep_tc_"))
    else:
        assert traffic is None and "stale" in src
