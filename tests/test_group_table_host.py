"""Host unit test of the job lookup of the serving pool's grouped kernels (group_find in
paper_1805_11169_gb300/csrc/icwf_internal.h): every trajectory item and every CWF item of a group
of jobs with ragged N maps to the job whose range holds it, at the range edges too.  The header is
compiled as plain C++; the expected job comes from numpy's searchsorted over the prefix sums.
CPU only."""
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
#include "icwf_internal.h"
using namespace icwf;
int main() {
  int njobs;
  while (scanf("%d", &njobs) == 1) {
    std::vector<GroupJob> g(njobs);
    int traj = 0, cwf = 0;
    for (int k = 0; k < njobs; ++k) {
      int N;
      if (scanf("%d", &N) != 1) return 1;
      g[k].traj0 = traj; g[k].cwf0 = cwf;
      traj += N; cwf += 2 * N;
    }
    for (int i = 0; i < traj; ++i) printf("%d ", group_find(g.data(), njobs, i, false));
    printf("\n");
    for (int i = 0; i < cwf; ++i) printf("%d ", group_find(g.data(), njobs, i, true));
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
    d = tmp_path_factory.mktemp("group")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(src), "-o",
                    str(exe)], check=True)
    return str(exe)


def test_every_item_finds_its_job(prog):
    rng = np.random.default_rng(11)
    groups = [[1], [5], [1, 1, 1], [64, 1, 2048, 3], [16, 96, 48, 40, 16]]
    groups += [list(rng.integers(1, 300, size=int(rng.integers(1, 40)))) for _ in range(20)]
    inp = "".join(f"{len(ns)} " + " ".join(str(n) for n in ns) + "\n" for ns in groups)
    out = subprocess.run([prog], input=inp, capture_output=True, text=True,
                         check=True).stdout.strip().split("\n")
    for k, ns in enumerate(groups):
        ns = np.array(ns)
        for scale, line in ((1, out[2 * k]), (2, out[2 * k + 1])):
            got = np.array([int(v) for v in line.split()])
            starts = np.concatenate([[0], np.cumsum(scale * ns)[:-1]])
            want = np.searchsorted(starts, np.arange(scale * ns.sum()), side="right") - 1
            assert np.array_equal(got, want), (ns, scale)
