"""Host unit test of the shared-memory FFT passes of the CWF propagator and the observables
(paper_1805_11169_gb300/csrc/fft_smem.cuh: radix-2 stages taken two at a time in radix-4 passes).

The header is compiled as plain C++ with a one-thread stand-in for the CTA (threadIdx.x = 0,
blockDim.x = 1, a no-op barrier): the groups of one pass touch disjoint elements, so running them
one after another is a valid execution of the parallel pass.  The forward transform (natural order
in, bit-reversed out) is checked against numpy's FFT, and the inverse transform (bit-reversed in,
natural order out, no 1/n) against the input, for every power of two from 2 to 4096 (odd and even
numbers of stages), in double and in single precision.  CPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_11169_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>
struct OneThread { unsigned x; };
static const OneThread threadIdx = {0}, blockDim = {1};
static inline void __syncthreads() {}
#include "fft_smem.cuh"
using namespace icwf;

template <typename R, typename Z>
static void run(int n, int logn) {
  std::vector<Z> tw(n / 2 > 0 ? n / 2 : 1), buf(n);
  for (int k = 0; k < n / 2; ++k) {
    double re, im;
    if (scanf("%la %la", &re, &im) != 2) return;
    tw[k].x = (R)re; tw[k].y = (R)im;
  }
  for (int i = 0; i < n; ++i) {
    double re, im;
    if (scanf("%la %la", &re, &im) != 2) return;
    buf[i].x = (R)re; buf[i].y = (R)im;
  }
  fft_dif(buf.data(), tw.data(), n, logn);
  for (int i = 0; i < n; ++i) printf("%a %a\n", (double)buf[i].x, (double)buf[i].y);
  ifft_dit(buf.data(), tw.data(), n, logn);
  for (int i = 0; i < n; ++i) printf("%a %a\n", (double)buf[i].x, (double)buf[i].y);
}

int main() {
  char t[8]; int n, logn;
  if (scanf("%7s %d %d", t, &n, &logn) != 3) return 1;
  if (t[0] == 'd') run<double, double2>(n, logn);
  else run<float, float2>(n, logn);
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
    d = tmp_path_factory.mktemp("fft")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", cuda_inc,
                    str(src), "-o", str(exe)], check=True)
    return str(exe)


def bitrev(n):
    logn = n.bit_length() - 1
    return np.array([int(format(i, f"0{logn}b")[::-1], 2) if logn else 0 for i in range(n)])


def transform(exe, kind, x):
    n = len(x)
    logn = n.bit_length() - 1
    tw = np.exp(-2j * np.pi * np.arange(n // 2) / n)
    lines = [f"{kind} {n} {logn}"]
    lines += [f"{float(z.real).hex()} {float(z.imag).hex()}" for z in tw]
    lines += [f"{float(z.real).hex()} {float(z.imag).hex()}" for z in x]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split()
    v = np.array([float.fromhex(s) for s in out]).reshape(-1, 2)
    z = v[:, 0] + 1j * v[:, 1]
    return z[:n], z[n:]


@pytest.mark.parametrize("kind,tol", [("d", 1e-13), ("f", 3e-6)])
def test_fft_passes_match_numpy_and_invert(prog, kind, tol):
    rng = np.random.default_rng(7)
    for logn in range(1, 13):
        n = 1 << logn
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        if kind == "f":
            x = x.astype(np.complex64).astype(np.complex128)
        fwd, back = transform(prog, kind, x)
        ref = np.fft.fft(x)
        scale = np.max(np.abs(ref))
        # bit-reversed output: slot m holds the coefficient of frequency bitrev(m)
        assert np.max(np.abs(fwd - ref[bitrev(n)])) < tol * scale * logn, (kind, n)
        assert np.max(np.abs(back / n - x)) < tol * np.max(np.abs(x)) * logn, (kind, n)


def test_fft_of_a_single_mode_is_a_spike(prog):
    """exp(2 pi i q j / n) transforms to n at frequency q (slot bitrev(q)) and zero elsewhere: a
    transposed operand, a wrong twiddle index or a dropped stage moves or spreads the spike."""
    for n, q in ((8, 3), (64, 5), (512, 17), (1024, 1000), (2048, 1)):
        j = np.arange(n)
        x = np.exp(2j * np.pi * q * j / n)
        fwd, _ = transform(prog, "d", x)
        expect = np.zeros(n, complex)
        expect[bitrev(n)[q]] = n        # bit reversal is its own inverse
        assert np.max(np.abs(fwd - expect)) < 1e-9 * n, (n, q)
