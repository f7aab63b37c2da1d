"""Admission policy of the serving loop (rd_server_policy.h): built with the
host compiler and run without a GPU."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_admission_policy(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "policy_check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1806_08901_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "server_policy_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "ok"
