"""FP64 solver with the factorisation's trailing updates in emulated FP64 on the tensor cores
(panel rows cut into exact BF16 digits, digit products summed exactly in TMEM, levels combined in
double-float) against the same solver with FP64 FMA updates and against the FP64 oracle.

Bars:
* the initial solve (S + eps I) C = b holds to 1e-11 relative with either update, S as stored and
  b = <psi_a chi_a | Psi0> recomputed by the oracle from the library's positions, at sizes that
  span one to nine 128-row tiles and ragged last tiles (N = 40 leaves an 8-row trailing matrix);
* the two updates give the same C to the rounding of the update (~2^-47 relative per element)
  amplified by the conditioning of S + eps I;
* FP64 mode dynamics with the emulated update follow the oracle within the FP64 parity bar (1e-9
  on C, x and R after 5 steps) and match the FMA update's dynamics to 1e-9 after 30 steps.
"""
import numpy as np
import pytest

from oracle.icwf import Icwf as Oracle, Params
from workloads import shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")

EPS = 1e-4


def oracle_for(w):
    return Oracle(Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
                         w.n_traj, w.svd_rel_cutoff, w.s_reg_eps), w.V)


def init_solve(w, precision, emulated, solve_fp64=0):
    sim = g.Icwf(g.params_from(w, precision=precision, solve_fp64=solve_fp64), w.V)
    sim.set_emulated_update(emulated)
    sim.init_from_density(w.psi0, 0)
    st = sim.state()
    S = sim.matrices()["S"]
    sim.close()
    o = oracle_for(w)
    ost = o.init_from_positions(w.psi0, st["x"], st["R"])
    Y = w.psi0 @ ost.chi.conj()                              # (nx, N)
    b = w.dx * w.dR * np.sum(ost.psi.conj() * Y, axis=0)
    r = (S + w.s_reg_eps * np.eye(w.n_traj)) @ st["C"] - b
    return float(np.linalg.norm(r) / np.linalg.norm(b)), st["C"]


@pytest.mark.parametrize("N", [40, 300, 1024, 1100])
def test_fp64_mode_initial_solve_residual(N):
    w = shin_metiu(n_traj=N, svd_rel_cutoff=1e-8, s_reg_eps=EPS)
    r_emu, c_emu = init_solve(w, g.ICWF_FP64, 1)
    r_fma, c_fma = init_solve(w, g.ICWF_FP64, 0)
    assert r_emu < 1e-11, r_emu
    assert r_fma < 1e-11, r_fma
    assert np.linalg.norm(c_emu - c_fma) / np.linalg.norm(c_fma) < 1e-9


@pytest.mark.parametrize("mode", [g.ICWF_MIXED_TF32X3, g.ICWF_MIXED_BF16X3])
def test_mixed_solve_fp64_residual_at_1024(mode):
    """solve_fp64 = 1 in the mixed modes takes the same FP64 solver (emulated updates by default)."""
    w = shin_metiu(n_traj=1024, svd_rel_cutoff=1e-8, s_reg_eps=EPS)
    r, _ = init_solve(w, mode, 1, solve_fp64=1)
    assert r < 1e-11, r


def test_emulated_update_dynamics_match_oracle_and_fma():
    w = shin_metiu(nx=256, nR=128, n_traj=130, dt=0.1, svd_rel_cutoff=1e-10, s_reg_eps=EPS)
    sim = g.Icwf(g.params_from(w, precision=g.ICWF_FP64), w.V)
    sim.init_from_density(w.psi0, 0)
    st0 = sim.state()
    sim.step(5)
    st = sim.state()
    o = oracle_for(w)
    ost = o.init_from_positions(w.psi0, st0["x"], st0["R"])
    for _ in range(5):
        o.step(ost)
    assert np.linalg.norm(st["C"] - ost.C) / np.linalg.norm(ost.C) < 1e-9
    assert np.max(np.abs(st["x"] - ost.x)) < 1e-9
    assert np.max(np.abs(st["R"] - ost.R)) < 1e-9
    sim.close()

    out = []
    for emulated in (1, 0):
        sim = g.Icwf(g.params_from(w, precision=g.ICWF_FP64), w.V)
        sim.set_emulated_update(emulated)
        sim.init_from_density(w.psi0, 0)
        sim.step(30)
        out.append(sim.state())
        sim.close()
    a, b = out
    assert np.linalg.norm(a["C"] - b["C"]) / np.linalg.norm(b["C"]) < 1e-9
    assert np.max(np.abs(a["x"] - b["x"])) < 1e-9


def test_switching_the_update_re_records_the_step_graphs():
    """icwf_set_emulated_update between steps takes effect in the captured step graphs: switching
    to the FMA update after 3 steps reproduces, bit for bit, a run that launches the same kernels
    directly, and differs from a run that keeps the emulated update."""
    w = shin_metiu(nx=256, nR=128, n_traj=96, dt=0.1, svd_rel_cutoff=1e-10, s_reg_eps=EPS)

    def run(graphs, switch):
        sim = g.Icwf(g.params_from(w, precision=g.ICWF_FP64), w.V)
        sim.set_step_graphs(graphs)
        sim.init_from_density(w.psi0, 0)
        sim.step(3)
        if switch:
            sim.set_emulated_update(0)
        sim.step(3)
        c = sim.state()["C"]
        sim.close()
        return c

    switched = run(True, True)
    direct = run(False, True)
    kept = run(True, False)
    assert np.array_equal(switched, direct)
    assert not np.array_equal(switched, kept)
