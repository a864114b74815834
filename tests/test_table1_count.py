"""Table 1 of the paper (Sec. 2): the proposed 8-point transform costs 22 additions, no
multiplications and no shifts.  The butterflies the kernels use (c0_forward, and c0t_inverse
for the inverse) are compiled on the host with a value type that counts every operation, and
their responses to the unit vectors are compared with the C0 printed in Sec. 2."""
import os
import shutil
import subprocess

import pytest

from tests.conftest import GOLDEN, ROOT, load_golden


def test_butterflies_cost_what_table1_prints(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "table1_count"
    src = os.path.join(ROOT, "tests", "native", "table1_count.cu")
    inc = os.path.join(ROOT, "paper_1402_6034_gb300", "csrc")
    res = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", inc, src, "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = subprocess.run([str(exe), os.path.join(GOLDEN, "c0_matrix.txt")], capture_output=True, text=True,
                         timeout=60)
    assert out.returncode == 0, out.stderr
    lines = {l.split()[0]: l.split()[1:] for l in out.stdout.strip().splitlines()}
    adds, muls, shifts = (int(v) for v in load_golden("table1_additions.txt")[0])
    assert [int(v) for v in lines["forward"]] == [adds, muls, shifts]
    # the inverse butterfly (C0^T) has the same cost
    assert [int(v) for v in lines["inverse"]] == [adds, muls, shifts]
    assert lines["matrix"] == ["ok"]
