"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer:
its pins run in a child process against the sanitized build (any report
aborts the child).  CPU only; skipped where gcc has no sanitizer runtime."""
import os
import subprocess
import sys

import pytest

import oracle.build as ob

HERE = os.path.dirname(os.path.abspath(__file__))
PINS = ["test_oracle_build.py", "test_oracle_octa_bin.py", "test_oracle_cube.py", "test_oracle_roi.py",
        "test_oracle_render.py", "test_oracle_footprint.py", "test_oracle_sh.py", "test_oracle_beta.py"]


def _asan_runtime():
    try:
        path = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True,
                              check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_pins_under_asan_and_ubsan():
    rt = _asan_runtime()
    if rt is None:
        pytest.skip("no ASan runtime")
    try:
        ob.build(sanitize=True)
    except subprocess.CalledProcessError:
        pytest.skip("gcc cannot build the sanitized oracle")
    env = dict(os.environ, ORACLE_SANITIZED="1", LD_PRELOAD=rt,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        *[os.path.join(HERE, f) for f in PINS]],
                       env=env, capture_output=True, text=True, timeout=900)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert "passed" in r.stdout and "ERROR: AddressSanitizer" not in tail and "runtime error" not in tail
