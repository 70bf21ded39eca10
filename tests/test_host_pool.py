"""The host thread pool (csrc/host_pool.cpp) when tasks throw, on the CPU.

A small harness (tests/host/host_pool_check.cpp, compiled here with g++)
runs 200 jobs in which some tasks throw, on the pool's threads or the
caller's: every task still runs exactly once, the caller receives a task's
exception only after the job is over (no worker is left holding the job),
and the pool then runs a plain job correctly.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_2895_gb300", "csrc")


def test_pool_survives_throwing_tasks(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "host_pool_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, os.path.join(ROOT, "tests", "host", "host_pool_check.cpp"),
                    os.path.join(CSRC, "host_pool.cpp"), "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok")
