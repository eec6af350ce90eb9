"""The bounds-checked build (libkpdhg_checked.so, -DKP_CHECKED): the stand-in for a device
memory checker.  Every instrumented kernel tests its computed global-memory indices; the test
runs the cases of tests/checked_cases.py through the checked library in a child process and
asserts that no access was out of range and that its results equal the release library's
(the checks only skip accesses, so the arithmetic is the same)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_release_build_reports_no_checks():
    need_gpu()
    from paper_1902_09657_gb300.api import bounds_report
    r = bounds_report()
    assert r == dict(checked=False, count=0, first_site=0, first_index=0)


def test_checked_build_records_no_out_of_range_access(tmp_path):
    need_gpu()
    from paper_1902_09657_gb300 import _build
    from tests import checked_cases
    _build.build(checked=True)
    rel_res = checked_cases.run_cases()                      # release library, this process
    out = tmp_path / "checked.npz"
    env = dict(os.environ, KPDHG_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    report = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert report["checked"] is True
    assert report["count"] == 0, f"out-of-range accesses recorded: {report}"
    chk = np.load(out)
    assert sorted(chk.files) == sorted(rel_res)
    for k, v in rel_res.items():
        assert rel(chk[k], v, f"checked vs release build: {k}") < 1e-6, k
