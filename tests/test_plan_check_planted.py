"""Planted mistakes for the schedule check, in C++ against the host analysis itself."""
import os
import shutil
import subprocess

import pytest

from tests.conftest import ROOT


def test_planted_schedule_mistakes_are_reported(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    csrc = os.path.join(ROOT, "paper_1005_0088_gb300", "csrc")
    exe = str(tmp_path / "planted")
    cmd = [gxx, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"), "-I" + csrc,
           os.path.join(ROOT, "tests", "plan_check_planted.cpp"), os.path.join(csrc, "analyze.cpp"),
           os.path.join(csrc, "plan_check.cpp"), os.path.join(csrc, "mu_search.cpp"), "-lpthread", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    print(out.stdout)
    assert out.returncode == 0, out.stdout
    assert out.stdout.count("rejected") == 5
