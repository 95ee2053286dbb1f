"""The checked build (-DBCH_CHECKED): its kernels record invalid caller-supplied indices
(automorphisms, OSD list entries) in a device check word and neutralise them instead of
faulting.  The cases run in a child process (checked_case.py) so that the checked
library, not the ordinary one this process has loaded, is the one in use."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_records_invalid_indices():
    env = dict(os.environ, BCHDEC_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_case.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    print(r.stdout[-4000:])
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
