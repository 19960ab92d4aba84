"""Host unit test of the double-float arithmetic used by the diagonal-block Cholesky kernel
(paper_1805_11169_gb300/csrc/df64.cuh): the header is compiled as plain C++ and checked against
exact rational arithmetic (Python fractions) on random inputs.  CPU only."""
import os
import random
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1805_11169_gb300", "csrc", "df64.cuh")

PROG = r'''
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include "df64.cuh"
using namespace icwf;
int main(int argc, char** argv) {
  // stdin: op a b (doubles); stdout: h l of the result (as %a hex floats)
  char op[16]; double a, b;
  while (scanf("%15s %la %la", op, &a, &b) == 3) {
    df x = df_from(a), y = df_from(b), r;
    if (op[0] == 'a') r = df_add(x, y);
    else if (op[0] == 's') r = df_sub(x, y);
    else if (op[0] == 'm') r = df_mul(x, y);
    else if (op[0] == 'r') r = df_rsqrt(x);
    else if (op[0] == 'q') r = df_rsqrt1(x);
    else if (op[0] == 'Q') r = df_rsqrt_refine(x, (float)(1.0 / sqrt((double)x.h)) * (float)b);
    else if (op[0] == 'p') r = df_add_sloppy(x, y);
    else r = x;   // 'c': conversion round trip
    printf("%a %a\n", (double)r.h, (double)r.l);
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("df64")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    return str(exe)


def run(exe, cases):
    inp = "".join(f"{op} {a.hex()} {b.hex()}\n" for op, a, b in cases)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    res = []
    for line in out.strip().split("\n"):
        h, l = line.split()
        res.append(Fraction(float.fromhex(h)) + Fraction(float.fromhex(l)))
    return res


def test_df64_operations_have_48_bit_accuracy(prog):
    rnd = random.Random(7)
    cases = []
    for _ in range(400):
        a = rnd.uniform(-1, 1) * 10 ** rnd.uniform(-6, 2)
        b = rnd.uniform(-1, 1) * 10 ** rnd.uniform(-6, 2)
        cases += [("a", a, b), ("s", a, b), ("m", a, b), ("r", abs(a), 0.0), ("c", a, 0.0),
                  ("q", abs(a), 0.0), ("p", a, b)]
        # the device's FP32 reciprocal square root is not correctly rounded: seeds off by up to
        # a few units in the last place must refine just as well
        cases.append(("Q", abs(a), 1.0 + rnd.choice([-4, -2, -1, 1, 2, 4]) * 2.0 ** -23))
    res = run(prog, cases)
    # exact value of the df inputs (each input is first rounded to a df, ~48 bits)
    def df_exact(x):
        import struct
        h = struct.unpack("f", struct.pack("f", x))[0]
        l = struct.unpack("f", struct.pack("f", x - h))[0]
        return Fraction(h) + Fraction(l)
    worst = 0.0
    for (op, a, b), r in zip(cases, res):
        x, y = df_exact(a), df_exact(b)
        if op == "s":
            ref = x - y
            scale = abs(x) + abs(y)
        elif op == "m":
            ref = x * y
            scale = abs(ref)
        elif op in ("a", "p"):
            ref = x + y
            scale = abs(x) + abs(y)
        elif op in ("r", "q", "Q"):
            ref = Fraction(1) / Fraction(float(x) ** 0.5)   # reference to double accuracy
            scale = abs(ref)
        else:
            ref, scale = Fraction(a), abs(Fraction(a))
        if scale == 0:
            continue
        err = float(abs(r - ref) / scale)
        tol = 2.0 ** -44 if op not in ("r", "q", "Q") else 2.0 ** -43
        worst = max(worst, err)
        assert err < tol, (op, a, b, err)
    assert worst > 0.0
