"""Global-index checks (the checked build, -DAC_BOUNDS_CHECK): every kernel
path -- binary64 on integer sums and plain, binary32 tiled and direct, the
batched ensemble, the closure convolutions on all three paths -- runs on small
and ragged grids with every index compared with its array's extent, and none
may leave it.  The self-test shows that a violation is recorded and redirected
(an index of -5 against an extent of 10, only computed).  Runs in a process of
its own, since the checked library replaces the normal one."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_kernel_leaves_its_arrays():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_run.py")], cwd=ROOT,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(res)
    for group in ("fp64_integer_sums", "fp64_plain", "fp32", "batch", "closure"):
        assert res[group] == 0, (group, hex(res[group]))
    assert res["selftest_status"] == 0
    assert res["selftest_values"] == [0, 3]
    word = res["selftest_word"]
    assert word >> 63 == 1 and (word >> 48) & 0x7fff == 7
    assert word & 0xffffffffffff == (-5) & 0xffffffffffff
