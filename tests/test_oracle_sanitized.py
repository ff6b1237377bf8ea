"""The FP64 oracle built with AddressSanitizer and UndefinedBehaviorSanitizer and driven through its
frame-level entry points (tests/oracle_sanitize_driver.c): out-of-bounds accesses, leaks, signed
overflow, misaligned or null accesses in the test infrastructure would abort the run. Skipped when
the C compiler has no sanitizer runtime."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_is_clean_under_address_and_undefined_sanitizers(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "oracle_sanitized")
    build = subprocess.run([cc, "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                            "-fno-sanitize-recover=all", os.path.join(HERE, "oracle_sanitize_driver.c"), "-lm",
                            "-o", exe], capture_output=True, text=True)
    if build.returncode != 0:
        if "sanitize" in build.stderr or "asan" in build.stderr.lower():
            pytest.skip("no sanitizer runtime: " + build.stderr.strip().splitlines()[-1])
        raise AssertionError(build.stderr)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0 and run.stdout.strip().endswith("ok"), run.stdout[-2000:] + run.stderr[-4000:]
    assert "runtime error" not in run.stderr, run.stderr[-4000:]
