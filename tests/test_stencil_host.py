"""Host unit test of the device's 4-point Lagrange stencils (paper_1805_11169_gb300/csrc/stencil.cuh),
which interpolate the CWFs and their gradients at the trajectory positions (Eq. v1/v2) and the
potential at the pinned coordinates: the header is compiled as plain C++ and its FP64 stencil is
compared with the oracle's (same start index, weights and derivative weights to rounding), its FP32
stencil to FP32 accuracy, inside the grid and where the start index is clamped at either end.
CPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.icwf import lagrange4

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_11169_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include "stencil.cuh"
using namespace icwf;
int main() {
  double p, lo, d; int n;
  while (scanf("%la %la %la %d", &p, &lo, &d, &n) == 4) {
    const Stencil s = lagrange4(p, lo, d, n);
    const StencilF f = lagrange4f(p, lo, d, n);
    printf("%d", s.i0);
    for (int m = 0; m < 4; ++m) printf(" %a", s.w[m]);
    for (int m = 0; m < 4; ++m) printf(" %a", s.dw[m]);
    printf(" %d", f.i0);
    for (int m = 0; m < 4; ++m) printf(" %a", (double)f.w[m]);
    for (int m = 0; m < 4; ++m) printf(" %a", (double)f.dw[m]);
    printf("\n");
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cuda_inc = None
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.isfile(os.path.join(c, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(c, "include")
    if shutil.which("g++") is None or cuda_inc is None:
        pytest.skip("g++ or the CUDA headers not available")
    d = tmp_path_factory.mktemp("stencil")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", cuda_inc,
                    str(src), "-o", str(exe)], check=True)
    return str(exe)


def run(exe, cases):
    inp = "".join(f"{float(p).hex()} {float(lo).hex()} {float(d).hex()} {n}\n"
                  for p, lo, d, n in cases)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    rows = []
    for line in out.strip().split("\n"):
        t = line.split()
        rows.append((int(t[0]), np.array([float.fromhex(v) for v in t[1:5]]),
                     np.array([float.fromhex(v) for v in t[5:9]]), int(t[9]),
                     np.array([float.fromhex(v) for v in t[10:14]]),
                     np.array([float.fromhex(v) for v in t[14:18]])))
    return rows


def test_device_stencils_match_the_oracle(prog):
    rng = np.random.default_rng(3)
    cases = []
    for lo, hi, n in ((-50.0, 50.0, 128), (-9.5, 9.5, 512), (-80.0, 80.0, 2048), (-1.0, 1.0, 8)):
        d = (hi - lo) / n
        ps = list(rng.uniform(lo + 0.5 * d, hi - 0.5 * d, 60))
        ps += [lo + 0.5 * d, hi - 0.5 * d, lo + 1.3 * d, hi - 1.2 * d, lo - 3 * d, hi + 2 * d]
        cases += [(p, lo, d, n) for p in ps]
    for (p, lo, d, n), (i0, w, dw, i0f, wf, dwf) in zip(cases, run(prog, cases)):
        j0, wo, dwo = lagrange4(p, lo, d, n)
        assert i0 == j0, (p, lo, d, n)
        assert np.allclose(w, wo, rtol=0, atol=1e-12), (p, w, wo)
        assert np.allclose(dw, dwo, rtol=0, atol=1e-12 / d), (p, dw, dwo)
        # FP32: s is rounded once to FP32, so the local coordinate u = s - i0 is off by up to
        # ulp(s)/2 (6e-5 of a cell at s ~ 2000) plus its own rounding; the weights are cubics in u
        # with slopes below 3 and second derivatives below 4 on the stencil.
        s = (p - lo) / d - 0.5
        du = float(np.spacing(np.float32(abs(s)) + np.float32(4.0))) + 1e-6
        if abs(s - np.round(s)) > 4 * du:     # the rounding cannot move the start index
            assert i0f == j0, (p, lo, d, n)
            assert np.allclose(wf, wo, rtol=0, atol=3 * du + 1e-6), (p, wf, wo)
            assert np.allclose(dwf, dwo, rtol=0, atol=(4 * du + 1e-6) / d), (p, dwf, dwo)


def test_device_stencil_is_exact_on_cubics(prog):
    """Interpolating a cubic and its derivative with the device weights is exact (to rounding)
    anywhere on the grid, clamped ends included: the stencil's defining property."""
    lo, n = -3.0, 64
    d = 0.1
    x = lo + (np.arange(n) + 0.5) * d
    f = lambda t: 0.3 * t ** 3 - 1.1 * t ** 2 + 0.7 * t - 2.0
    df = lambda t: 0.9 * t ** 2 - 2.2 * t + 0.7
    ps = np.linspace(lo - 0.2, lo + n * d + 0.2, 97)
    for p, (i0, w, dw, *_f) in zip(ps, run(prog, [(p, lo, d, n) for p in ps])):
        vals = f(x[i0:i0 + 4])
        assert abs(w @ vals - f(p)) < 1e-11 * (1 + abs(f(p)))
        assert abs(dw @ vals - df(p)) < 1e-9 * (1 + abs(df(p)))
