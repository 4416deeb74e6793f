"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU): the oracle's pin
tests against a sanitized oracle build, and the library's host BVH build and host walk from a
small driver; the multi-threaded host build under ThreadSanitizer (data races). compute-sanitizer
is closed on the GPU pool; device code is covered by bounds checks that report through the status
word instead."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    path = subprocess.run(["g++", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.fixture(scope="module")
def runtimes():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("sanitizer runtimes not available")
    return asan, ubsan


def test_oracle_pins_under_sanitizers(runtimes):
    env = dict(os.environ, GSP_ORACLE_SANITIZE="1", LD_PRELOAD=" ".join(runtimes),
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    tests = ["tests/test_oracle_geometry.py", "tests/test_oracle_grid.py", "tests/test_oracle_sppm.py",
             "tests/test_oracle_grad.py", "tests/test_oracle_rng.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"] + tests,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:] + r.stderr[-3000:])


def test_host_bvh_build_under_sanitizers(runtimes, tmp_path):
    exe = str(tmp_path / "sanitize_bvh")
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
           "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1505_06022_gb300", "csrc"), "-I", "/usr/local/cuda/include",
           os.path.join(ROOT, "tests", "sanitize_bvh_main.cpp"),
           os.path.join(ROOT, "paper_1505_06022_gb300", "csrc", "bvh_build.cpp"), "-o", exe, "-ldl"]
    if not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("CUDA headers not available")
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="halt_on_error=1"))
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout + r.stderr)[-3000:]


def test_host_bvh_build_under_thread_sanitizer(tmp_path):
    if shutil.which("g++") is None or not _runtime("libtsan.so"):
        pytest.skip("ThreadSanitizer runtime not available")
    if not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("CUDA headers not available")
    exe = str(tmp_path / "tsan_bvh")
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-fno-omit-frame-pointer",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1505_06022_gb300", "csrc"),
           "-I", "/usr/local/cuda/include", os.path.join(ROOT, "tests", "sanitize_bvh_main.cpp"),
           os.path.join(ROOT, "paper_1505_06022_gb300", "csrc", "bvh_build.cpp"), "-o", exe, "-ldl", "-pthread"]
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, TSAN_OPTIONS="halt_on_error=1:second_deadlock_stack=1"))
    assert r.returncode == 0 and "ok" in r.stdout, (r.stdout + r.stderr)[-3000:]
