"""The committed ncu summaries describe the kernels as they are.

Each kernel summary under profiles/ ends with the hash of the kernel's own sources (its
launcher and tile header) at the time of the capture, and bench.py reports the DRAM and
L2 figures of a summary only while that hash still matches.  This test fails as soon as
a kernel changes without a new capture, so that the figures beside the bench line never
describe an older kernel.
"""
import hashlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1002_3675_b300", "csrc")

# summary name prefix -> the sources its hash covers, in the order they are hashed
SOURCES = {
    "k_project": ["k_project.cu", "project_tile.cuh"],
    "k_backproject": ["k_backproject.cu", "bp_tile.cuh"],
    "k_tv_x": ["k_tv.cu", "tv_tile.cuh", "tv_xmarch.cuh"],
    "k_bp_eq2": ["k_bp_eq2.cu", "bp_eq2_tile.cuh"],
}


def _hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _summaries():
    out = []
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        for prefix in sorted(SOURCES, key=len, reverse=True):
            if name.startswith(prefix + "_") and name.endswith(".md"):
                out.append((name, prefix))
                break
    return out


def test_every_kernel_has_a_summary_per_workload():
    names = {n for n, _ in _summaries()}
    for prefix in SOURCES:
        for workload in ("large", "medium"):
            assert f"{prefix}_{workload}.md" in names, f"no ncu summary {prefix}_{workload}.md"


@pytest.mark.parametrize("name,prefix", _summaries())
def test_summary_matches_current_sources(name, prefix):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    assert m, f"{name} records no source hash"
    assert m.group(1) == _hash(SOURCES[prefix]), f"{name} was captured on other sources of {prefix}"


def test_bench_hashes_the_same_sources():
    # bench.py decides from the same file lists whether a summary's figures still apply
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for kernel, (name, files) in bench.KERNEL_SOURCES.items():
        assert SOURCES[name] == list(files), kernel
