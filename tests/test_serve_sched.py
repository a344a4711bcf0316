"""The serving scheduler (``csrc/dg_serve_sched.cpp``: FIFO queue, admission by
the device-memory budget, retirement, byte and cell-stage accounting) on the
CPU against a fake device engine, built with AddressSanitizer and
UndefinedBehaviorSanitizer (``tests/serve_sched_driver.cpp``).  Failures are
injected on the host, as error codes from the fake engine: a start that fails,
a poll that fails, a result copy that fails, a tick whose wait gives up, a
solve that turns non-admissible.  The scenarios check:
* first-come-first-served admission under the budget;
* a request larger than the whole budget fails with DG_ENOMEM and does not
  change the bytes in use;
* failed starts hold no memory and free their inputs;
* errors propagate without losing or double-freeing a running solve;
* after an error, the batch is rebuilt before the next steps;
* under random traffic, bytes in use equal the running requests' bytes,
  never exceed the budget, and every request is freed exactly once."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2409_09620_gb300", "csrc")


def test_serve_scheduler_scenarios(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "sched")
    cmd = ["g++", "-O1", "-g", "-std=c++17", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-Wall", "-Wextra", "-I", CSRC, os.path.join(HERE, "serve_sched_driver.cpp"),
           os.path.join(CSRC, "dg_serve_sched.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr or "ubsan" in r.stderr):
        pytest.skip("the sanitizer runtimes are not installed")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:exitcode=23", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
