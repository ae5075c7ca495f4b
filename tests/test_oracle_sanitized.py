"""The oracle is free of memory errors and undefined behaviour on the pin
suite: oracle/gj_oracle.c is compiled with AddressSanitizer and
UndefinedBehaviorSanitizer and the pin tests (tests/test_oracle.py,
tests/test_oracle_specialisations.py) run against that build. A positive
control compiles a copy whose triangle list is allocated one element short
and checks that the sanitizer reports it, so a clean run means the checks
were active. CPU only; the builds live in a temporary directory."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gj_oracle.c")
PINS = ["tests/test_oracle.py", "tests/test_oracle_specialisations.py"]
SHORT_ALLOC = ("uint32_t* tn = (uint32_t*)malloc(sizeof(uint32_t) * (to[g->m] ? to[g->m] : 1));",
               "uint32_t* tn = (uint32_t*)malloc(sizeof(uint32_t) * (to[g->m] > 1 ? to[g->m] - 1 : 1));")


def _runtime(name):
    p = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True)
    path = p.stdout.strip()
    return path if p.returncode == 0 and os.path.isabs(path) and os.path.exists(path) else None


@pytest.fixture(scope="module")
def sanitizers():
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not installed")
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("the sanitizer runtimes are not installed")
    return asan, ubsan


def _build(text, path):
    with open(path + ".c", "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                           "-fno-omit-frame-pointer", "-fPIC", "-shared", "-o", path, path + ".c"])


def _run(lib, sanitizers, tests):
    env = dict(os.environ, GJ_ORACLE_LIB=lib, LD_PRELOAD=" ".join(sanitizers),
               ASAN_OPTIONS="detect_leaks=0", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    # -s: a sanitizer report is written to file descriptor 2 as the process
    # stops, which pytest's own capture would swallow
    p = subprocess.run([sys.executable, "-m", "pytest", *tests, "-x", "-q", "-s", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout + p.stderr


def test_pins_run_clean_under_sanitizers(sanitizers, tmp_path):
    lib = str(tmp_path / "liboracle_san.so")
    _build(open(SRC).read(), lib)
    rc, out = _run(lib, sanitizers, PINS)
    assert rc == 0 and "runtime error" not in out and "AddressSanitizer" not in out, out[-3000:]


def test_sanitizer_reports_a_planted_overflow(sanitizers, tmp_path):
    src = open(SRC).read()
    assert src.count(SHORT_ALLOC[0]) == 1
    lib = str(tmp_path / "liboracle_short.so")
    _build(src.replace(*SHORT_ALLOC), lib)
    rc, out = _run(lib, sanitizers, ["tests/test_oracle_specialisations.py"])
    assert rc != 0 and "heap-buffer-overflow" in out, out[-3000:]
