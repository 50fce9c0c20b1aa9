"""Host-side AddressSanitizer and UndefinedBehaviorSanitizer runs of the oracle and the input
generators (CPU only): tests/native/sanitize_driver.c calls every entry point of both on seeded
graphs; gcc instruments all three sources and any finding aborts the run."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_and_generators_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc is not installed")
    exe = str(tmp_path / "sanitize_driver")
    cmd = [gcc, "-O1", "-g", "-std=c11", "-fopenmp", "-fno-omit-frame-pointer", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           os.path.join(ROOT, "tests", "native", "sanitize_driver.c"),
           os.path.join(ROOT, "oracle", "tc_oracle.c"), os.path.join(ROOT, "graphgen", "graphgen.c"),
           "-lm", "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "asan" in build.stderr.lower():
        pytest.skip("the sanitizer runtime is not installed: " + build.stderr.strip().splitlines()[-1])
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1",
               OMP_NUM_THREADS="4")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    for family in ("erdos_renyi", "barabasi_albert", "chung_lu", "empty"):
        assert family in r.stdout
