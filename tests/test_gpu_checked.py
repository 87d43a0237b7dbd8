"""The bounds-checked library (libarbx_checked.so, loaded when the environment
has ARBX_CHECKED=1).  Both tests run in a child process, so the library this
session loaded stays the regular one:

* the parity suites pass on it unchanged: every tree those tests build passes
  the device-side walk from its root (each record and leaf reached once, codes
  in range, float32 parent boxes holding their children) and no index check
  fires during their queries;
* a query order that is not a permutation of 0..m-1 (one entry past m, or a
  repeated entry) is refused with ARBX_ERR_BOUNDS by the permutation check that
  runs before any traversal reads the order, and the library keeps working.
The child process checks that the checked build is the one loaded before it
passes a bad order."""
from __future__ import annotations

import os
import subprocess
import sys
import textwrap
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
pytestmark = pytest.mark.gpu


def _run(cmd: list[str], timeout: int) -> subprocess.CompletedProcess:
    env = dict(os.environ, ARBX_CHECKED="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def test_parity_suites_on_the_checked_library():
    r = _run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
              "tests/test_gpu_parity.py", "tests/test_gpu_contained.py", "tests/test_gpu_visits.py",
              "tests/test_gpu_forest.py"], timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


BAD_ORDER = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    import paper_2507_23700_b300 as arbx
    import oracle
    if arbx.library_flags() != arbx.LIB_CHECKED:
        sys.exit(3)  # not the checked build: never hand a bad order to the regular one
    rng = np.random.default_rng(7)
    pts = rng.random((20000, 3), dtype=np.float32)
    qs = rng.random((5000, 3), dtype=np.float32)
    tree = arbx.Tree(torch.from_numpy(pts).cuda())
    qd = torch.from_numpy(qs).cuda()
    m = qs.shape[0]
    good = tree.query_order(arbx.SPHERE, qd, 0.05)
    for bad_kind in ("past_end", "repeat"):
        bad = good.clone()
        if bad_kind == "past_end":
            bad[1234] = m + 7
        else:
            bad[1234] = bad[4321]
        try:
            tree.callback(arbx.SPHERE, qd, arbx.CB_COUNT, radius=0.05, order=bad)
        except arbx.ArbxError as e:
            assert e.status == arbx.ERR_BOUNDS, e
        else:
            raise AssertionError("a bad order was accepted: " + bad_kind)
    # the library keeps working, and a valid caller order gives the oracle's counts
    cnt = tree.callback(arbx.SPHERE, qd, arbx.CB_COUNT, radius=0.05, order=good)
    assert np.array_equal(cnt.cpu().numpy(), oracle.radius_count(pts, qs, 0.05))
    arbx.stream_check()
    print("checked-ok")
""")


def test_bad_order_is_refused_by_the_checked_library():
    r = _run([sys.executable, "-c", BAD_ORDER], timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked-ok" in r.stdout
