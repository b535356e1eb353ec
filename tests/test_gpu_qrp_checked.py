"""The cluster QRP's index arithmetic under the checked build (TUCKER_QRP_CHECKED): every
index of its shared, distributed-shared and global arrays is compared with the array's
length, an index outside is replaced by 0 and its site recorded.  The QRP, HOOI,
column-norm and no-allocation parity tests run in a child process against that build;
they must pass as on the normal build and leave no recorded site (tucker_check_site() == 0,
read in the child after its last test)."""
import os
import subprocess
import sys

import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cluster_qrp_checked_build(tmp_path):
    need_gpu()
    from paper_2010_10638_gb300 import build
    lib = build.build_checked()
    report = tmp_path / "check_site.txt"
    env = dict(os.environ, TUCKER_LIB_PATH=lib, TUCKER_CHECK_REPORT=str(report), TUCKER_QRP_FORM="cluster")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_qrp.py", "tests/test_zz_no_alloc.py", "tests/test_gpu_norms.py",
           "tests/test_gpu_hooi.py", "-k", "not multi and not persistent"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    site = int(report.read_text())
    assert site == 0, f"checked build: index outside its array at site {site}"
