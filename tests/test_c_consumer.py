"""The boundary from plain C: tests/c_consumer.c includes include/rdct.h,
compiles as C11 with gcc, links against the in-tree librdct.so and makes the
calls that need no GPU."""
import os
import shutil
import subprocess

import pytest

from paper_1402_6034_gb300 import rdct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_links_and_calls_the_library(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    rdct.load()  # builds the library if needed
    libdir = os.path.dirname(rdct.lib_path())
    exe = tmp_path / "c_consumer"
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_consumer.c"), "-o", str(exe), "-L", libdir, "-lrdct",
           f"-Wl,-rpath,{libdir}"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    lines = dict(line.split(" ", 1) for line in out.stdout.strip().splitlines())
    assert int(lines["version"]) >= 10000
    assert lines["status2"] == "invalid shape"
    assert lines["forward"] == "2 detail-ok"
    assert lines["fused"] == "1"
    assert lines["plan"] == "2 null named"
