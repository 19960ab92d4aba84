"""Overlap S = S1 o S2 of the mixed modes as exact Grams of fixed-point CWFs (tensor cores).

The library writes each complex64 CWF column as 2^e times four balanced base-2^beta digits
(beta = 6 for grids up to 2048 points) and sums all digit products exactly.  These tests rebuild
that representation here from the GPU's own CWFs (the digit recursion in float32 NumPy) and check:

* S equals the FP64 Gram of the represented CWFs to 1e-9 relative (split products with FP32
  accumulation are ~1e-7 away), and the FP64 Gram of the unrounded complex64 CWFs to 1e-7;
* S is positive semidefinite to rounding at N = 1024 on the bench grid (smallest eigenvalue
  >= -1e-10), where the split-product overlap (overlap_split = 1) has eigenvalues near -1e-5;
* a 1000-step N = 1024 run with eps = 1e-5 keeps S + eps I positive definite (the split-product
  overlap needed eps = 1e-3), and the mixed mode at eps = 1e-6 stays within 1e-3 L1 of the FP64
  oracle at eps = 1e-6 on the paper grid (N = 256, 100 steps).
"""
import numpy as np
import pytest

from oracle.icwf import Icwf as Oracle, Params
from workloads import shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def fixed_point(cwf):
    """The 4-digit fixed-point form of complex64 columns (n x N), as complex128."""
    n = cwf.shape[0]
    beta = 6 if n <= 2048 else 5
    re = cwf.real.astype(np.float32)
    im = cwf.imag.astype(np.float32)
    m = np.maximum(np.abs(re).max(axis=0), np.abs(im).max(axis=0))
    e = np.frexp(m)[1].astype(np.int32)                 # m < 2^e
    B = np.float32(2.0 ** beta)

    def digits(v):
        v = np.ldexp(v, (beta - e)[None, :]).astype(np.float32)
        out = np.zeros(v.shape, np.float64)
        for p in range(4):
            d = np.rint(v)
            out += d.astype(np.float64) * 2.0 ** (-beta * (p + 1))
            v = ((v - d) * B).astype(np.float32)
        return np.ldexp(out, e[None, :])

    return digits(re) + 1j * digits(im)


def grams(psi, chi, dx, dR):
    return (dx * (psi.conj().T @ psi)) * (dR * (chi.conj().T @ chi))


def sm_paper(**kw):
    d = dict(nx=1024, x_range=(-100.0, 100.0), nR=512, R_range=(-9.5, 9.5), dt=0.05,
             svd_rel_cutoff=1e-8)
    d.update(kw)
    return shin_metiu(**d)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode,N", [(2, 37), (1, 130), (2, 1024)])
def test_overlap_is_the_exact_gram_of_the_fixed_point_cwfs(mode, N):
    if N == 1024:
        w = sm_paper(n_traj=N, s_reg_eps=1e-5)
    else:
        w = shin_metiu(n_traj=N, svd_rel_cutoff=1e-8, s_reg_eps=1e-5)
    sim = g.Icwf(g.params_from(w, precision=mode), w.V)
    sim.init_from_density(w.psi0, 0)
    for n_steps in (0, 5):
        sim.step(n_steps)
        st = sim.state()
        S = sim.matrices()["S"]
        Sfp = grams(fixed_point(st["psi"]), fixed_point(st["chi"]), w.dx, w.dR)
        assert rel(S, Sfp) < 1e-9, rel(S, Sfp)
        assert rel(S, grams(st["psi"], st["chi"], w.dx, w.dR)) < 1e-7
        assert np.array_equal(S, S.conj().T)
    if N == 1024:
        lam = np.linalg.eigvalsh(S)
        assert lam[0] > -1e-10 * lam[-1], lam[0]
        sim.close()
        # the split-product overlap cannot be factorised with eps = 1e-5 (it has eigenvalues near
        # -1e-5), so it runs with the eps it needs
        split = g.Icwf(g.params_from(w.with_(s_reg_eps=1e-3), precision=mode, overlap_split=1),
                       w.V)
        split.init_from_density(w.psi0, 0)
        split.step(5)
        Ss = split.matrices()["S"]
        assert np.linalg.eigvalsh(0.5 * (Ss + Ss.conj().T))[0] < -1e-7
        split.close()
    else:
        sim.close()


def test_small_eps_long_run_at_bench_size():
    w = sm_paper(n_traj=1024, s_reg_eps=1e-5)
    sim = g.Icwf(g.params_from(w, precision=2), w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, 0)
    sim.step(1000)
    ob = sim.observables()
    assert abs(ob["norm"] - 1.0) < 1e-2
    sim.close()


def test_mixed_at_fp64_eps_against_the_fp64_oracle():
    w = sm_paper(n_traj=256, s_reg_eps=1e-6)
    o = Oracle(Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
                      w.n_traj, w.svd_rel_cutoff, w.s_reg_eps), w.V)
    ost = o.init_from_density(w.psi0, 0)
    for _ in range(100):
        o.step(ost)
    oo = o.observables(ost, w.phi)
    for mode in (1, 2):
        sim = g.Icwf(g.params_from(w, precision=mode), w.V)
        sim.set_projectors(w.phi)
        sim.init_from_density(w.psi0, 0)
        sim.step(100)
        ob = sim.observables()
        l1x = w.dx * np.sum(np.abs(ob["rho_x"] - oo["rho_x"]))
        l1R = w.dR * np.sum(np.abs(ob["rho_R"] - oo["rho_R"]))
        l1p = np.sum(np.abs(ob["pop"] - oo["pop"]))
        assert l1x < 1e-3 and l1R < 1e-3 and l1p < 1e-3, (mode, l1x, l1R, l1p)
        sim.close()
