"""Host logic of the 3D work lists, without a GPU: the library's setup code
(csrc/setup.cpp) is compiled with g++ together with host_geometry_check.cpp,
which builds the torus hierarchy and checks, level by level,

* the row segments (every inside node in exactly one segment of at most 64
  consecutive inside nodes of one row),
* the red band sweep's neighbour sources (the node, or the number of the
  ghost at that neighbour, in the order of the sweep's sum),
* the box form of the ghost stencils against the stored 27 nodes,
* the list of coarse nodes with a partly outside neighbourhood (Sec. 2.5
  partial transfer) and their FP64 / FP32 weights against the independent
  host routine,
* the junction zone's blocks (every zone node written back by exactly one
  block; each block updates every zone node within 4 mu nodes of its own).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1111_0983_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("hgc") / "host_geometry_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, os.path.join(ROOT, "tests", "host_geometry_check.cpp"),
                    os.path.join(CSRC, "setup.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("n", [65, 129])
def test_host_work_lists_match_their_definitions(checker, n):
    out = subprocess.run([checker, str(n)], capture_output=True, text=True, timeout=600)
    rows = [ln.split() for ln in out.stdout.splitlines()]
    checks = [(r[0], int(r[1]), int(r[2])) for r in rows if len(r) == 3]
    assert checks, out.stdout + out.stderr
    bad = [c for c in checks if c[1] != 0]
    assert not bad and out.returncode == 0, bad
    names = {c[0] for c in checks}
    assert {"segments", "red_sources", "box_stencils", "partial_transfer", "junction_blocks"} <= names
    # the finest level's lists are not empty, and its junction zone is split into blocks
    first = {c[0]: c[2] for c in checks[:5]}
    assert all(first[k] > 0 for k in first), first
    assert rows[[r[0] for r in rows].index("junction_blocked")][1] == "1"
