"""Host pin of the FP64 helper exp_neg_small (csrc/dg_math.h), which the OE
damping uses on the GPU for exp(-x) at 0 <= x <= 2^-8: compiled as plain C++
and compared with exp(-x) to 50 significant digits (Python's decimal module)
on 0, subnormals, the interval end and 40,000 seeded arguments.  The
truncation error is below 2^-79, so the result should be within about half
an ulp (the Horner rounding); the test allows 0.75 ulp."""
import os
import random
import shutil
import subprocess
from decimal import Decimal, getcontext

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2409_09620_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "dg_math.h"
int main() {
  double x;
  while (std::scanf("%la", &x) == 1) std::printf("%a\n", dg::exp_neg_small(x));
  return 0;
}
"""


def _ulp(v):
    import math
    m, e = math.frexp(v)          # v = m 2^e, 0.5 <= m < 1
    return 2.0 ** (e - 53)


def test_exp_neg_small_within_one_ulp(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "t.cpp"
    src.write_text(PROG)
    exe = tmp_path / "t"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-I", HDR, str(src), "-o", str(exe)], check=True)
    rng = random.Random(11)
    xmax = 2.0 ** -8
    xs = [0.0, 5e-324, 2.0 ** -1074 * 3, 2.0 ** -60, 2.0 ** -30, xmax, xmax * (1 - 2 ** -52)]
    xs += [rng.uniform(0.0, xmax) for _ in range(20000)]
    xs += [2.0 ** rng.uniform(-60.0, -8.0) for _ in range(20000)]
    out = subprocess.run([str(exe)], input="\n".join(x.hex() for x in xs), capture_output=True, text=True,
                         check=True).stdout.split()
    assert len(out) == len(xs)
    getcontext().prec = 50
    worst = 0.0
    for x, r in zip(xs, out):
        y = float.fromhex(r)
        ref = (-Decimal(x)).exp()
        err = float(abs(Decimal(y) - ref)) / _ulp(y)
        worst = max(worst, err)
    assert worst <= 0.75, worst
    assert float.fromhex(out[0]) == 1.0
