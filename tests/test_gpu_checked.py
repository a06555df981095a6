"""The range-checked build (CWTHF_CHECKED): every data-driven index is tested
before use, so a library bug or an inconsistent input shows up as
CWTHF_E_INDEX instead of an out-of-range access.  The same workload through
both libraries gives the same results, and the checked one reports no bad
index."""
import json
import os
import subprocess
import sys

import pytest

from tests import checked_run

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_agrees_and_reports_nothing():
    plain = checked_run.run()
    assert plain["checked"] == 0
    env = dict(os.environ, CWTHF_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "tests.checked_run"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    checked = json.loads(r.stdout.strip().splitlines()[-1])
    assert checked["checked"] == 1
    for k in ("find_status", "deposit_status", "ms_status"):
        assert plain[k] == 0 and checked[k] == 0, (k, plain[k], checked[k])
    for k in ("find_n_halo", "find_ids", "deposit", "ms_n_halo", "ms_ids"):
        assert plain[k] == checked[k], k
    assert plain["ms_n_halo"] > 0 and sum(plain["find_n_halo"]) > 0
