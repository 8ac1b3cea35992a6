"""The checked build (device bounds checks compiled in) on the parity cases of
tests/checked_cases.py: every kernel agrees with the oracle and no check
fails.  The checks replace a memory checker, which this GPU pool does not
offer; the release build compiles none of them."""
import json
import os
import subprocess
import sys

import pytest

from conftest import has_gpu
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import qpath

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_release_build_compiles_no_checks():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    enabled, first = qpath.qp_device_checks()
    assert not enabled and first == 0


def test_checked_build_parity_and_no_failed_check():
    if not has_gpu():
        pytest.skip("no CUDA device")
    path = qbuild.build(checked=True)
    env = dict(os.environ, QPATH_LIBRARY=path)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["enabled"] and line["first_failure"] == 0
    assert len(line["results"]) >= 20 and all(line["results"].values()), line["results"]
