"""The oracle built with AddressSanitizer and UndefinedBehaviorSanitizer:
every pin must pass with no sanitizer report (out-of-bounds access, use of
freed memory, signed overflow, misaligned access, ...).  Runs in a child
process that preloads the address-sanitizer runtime."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _runtime(name):
    try:
        path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True,
                              text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_pins_under_asan_and_ubsan(tmp_path):
    asan = _runtime("libasan.so")
    if asan is None or _runtime("libubsan.so") is None:
        pytest.skip("gcc sanitizer runtimes are not installed")
    lib = oracle.compile_oracle(
        oracle.SOURCE, str(tmp_path / "liboracle_san.so"), werror=False,
        extra_flags=["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                     "-fno-omit-frame-pointer"])
    code = (
        "import sys; sys.path[:0] = [%r, %r]\n"
        "import oracle, oracle_pins\n"
        "L = oracle.load_library(%r)\n"
        "for pin in oracle_pins.PINS:\n"
        "    pin(L)\n"
        "print('pins ok', len(oracle_pins.PINS))\n"
    ) % (os.path.dirname(HERE), HERE, lib)
    env = dict(os.environ, LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:exitcode=23",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1:exitcode=24")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    report = r.stdout[-2000:] + r.stderr[-4000:]
    assert r.returncode == 0, report
    assert "pins ok" in r.stdout, report
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, report
