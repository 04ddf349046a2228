"""The factorization's host thread pool (paper_1905_10602_gb300/csrc/host_pool.h),
compiled on its own with g++ and run on the CPU: exactly-once indices,
exception propagation, reuse after an exception, and two concurrent callers,
also under ThreadSanitizer where the compiler offers it."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1905_10602_gb300", "csrc")
SRC = os.path.join(HERE, "host_pool_check.cpp")


def _build(tmp_path, extra):
    exe = str(tmp_path / ("pool" + ("_tsan" if extra else "")))
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-pthread", "-I", CSRC, SRC, "-o", exe] + extra
    p = subprocess.run(cmd, capture_output=True, text=True)
    return exe, p


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_host_pool(tmp_path):
    exe, p = _build(tmp_path, [])
    assert p.returncode == 0, p.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "host_pool ok" in r.stdout, r.stdout + r.stderr


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_host_pool_thread_sanitizer(tmp_path):
    exe, p = _build(tmp_path, ["-fsanitize=thread"])
    if p.returncode != 0:
        pytest.skip("no ThreadSanitizer in this toolchain")
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
    if r.returncode != 0 and "FATAL: ThreadSanitizer" in r.stderr and "WARNING" not in r.stderr:
        pytest.skip("ThreadSanitizer cannot run here: " + r.stderr.strip().splitlines()[0])
    assert r.returncode == 0 and "host_pool ok" in r.stdout, r.stdout + r.stderr[-3000:]
