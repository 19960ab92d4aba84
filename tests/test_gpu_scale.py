"""Parity at the sizes the bench runs, through the C ABI.

* FP64 on the paper-scale grids: Shin-Metiu 1024 x 512 and the cavity 2048 x 256 (FFT lengths
  1024 and 2048; the FP64 propagator's column of 2048 complex128 samples needs more than 48 KB of
  shared memory), N = 16, 5 steps: CWFs, S, Heff, C (S-norm) and positions element by element
  against the FP64 oracle, to 1e-10.
* Mixed TF32x3 and BF16x3 at N = 1024 on the 1024 x 512 grid (the bench's launch configuration:
  144 CTAs of the tensor-core kernel, K = 1024 / 512 per Gram): the whole S and Heff against the
  oracle's formulas evaluated in FP64 on the GPU's own complex64 CWFs and positions, within
  1e-5 relative Frobenius, after init and after two steps.
"""
import numpy as np
import pytest

from oracle.icwf import Icwf as Oracle, Params
from workloads import cavity, shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def s_norm_rel(C, Cref, S):
    d = C - Cref
    return float(np.sqrt(abs((d.conj() @ S @ d).real)) / np.sqrt(abs((Cref.conj() @ S @ Cref).real)))


def oracle_for(w):
    return Oracle(Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
                         w.n_traj, w.svd_rel_cutoff, w.s_reg_eps), w.V)


def sm_paper(**kw):
    d = dict(nx=1024, x_range=(-100.0, 100.0), nR=512, R_range=(-9.5, 9.5), dt=0.05,
             svd_rel_cutoff=1e-12)
    d.update(kw)
    return shin_metiu(**d)


@pytest.mark.parametrize("name", ["shin_metiu_1024x512", "cavity_2048x256"])
def test_fp64_paper_grids_element_by_element(name):
    if name.startswith("shin"):
        w = sm_paper(n_traj=16)
    else:
        w = cavity(n_traj=16, dt=0.05, svd_rel_cutoff=1e-12, lam=0.5)
    o = oracle_for(w)
    ost = o.init_from_density(w.psi0, 0)
    sim = g.Icwf(g.params_from(w), w.V)
    sim.init_from_density(w.psi0, 0)
    assert sim.info()["rank"] == len(o.fac.s)
    for _ in range(5):
        o.step(ost)
    sim.step(5)
    st = sim.state()
    m = sim.matrices()
    assert rel(st["psi"], ost.psi) < 1e-11 and rel(st["chi"], ost.chi) < 1e-11
    assert rel(m["S"], ost.S) < 1e-10
    assert rel(m["Heff"], ost.Heff) < 1e-10
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-10
    assert np.max(np.abs(st["x"] - ost.x)) < 1e-10 and np.max(np.abs(st["R"] - ost.R)) < 1e-10
    sim.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_mixed_assembly_at_bench_size(mode):
    w = sm_paper(n_traj=1024, svd_rel_cutoff=1e-8, s_reg_eps=1e-3)
    sim = g.Icwf(g.params_from(w, precision=mode), w.V)
    sim.init_from_density(w.psi0, 0)
    o = oracle_for(w)
    for n_steps in (0, 2):
        sim.step(n_steps)
        st = sim.state()
        m = sim.matrices()
        S = o.overlaps(st["psi"], st["chi"])[2]
        H = o.heff_factorised(st["psi"], st["chi"], st["x"], st["R"])
        eS, eH = rel(m["S"], S), rel(m["Heff"], H)
        assert eS < 1e-5 and eH < 1e-5, (n_steps, eS, eH)
    sim.close()
