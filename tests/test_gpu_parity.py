"""GPU (CUDA library, via the C ABI) versus the FP64 oracle, element by element.

Tolerances.  The FP64 path must match the oracle to 1e-10 relative on S, Heff and H after 100
steps of the 128 x 64 Shin-Metiu case.  The coefficient vector C is compared in the S-norm,
||dC||_S = sqrt(dC^H S dC) relative to ||C||_S, which is the norm of the wavefunction difference
sum_a dC_a phi_a: S has condition numbers up to 1e12 here, and C's components along S's
near-null space are fixed only through the regulariser.  A rounding perturbation dS of S moves C
by up to |dS C| / (2 sqrt(eps)) in the S-norm, which with eps = 1e-6 stays far below 1e-10.
Positions, CWFs and observables are compared directly.
"""
import numpy as np
import pytest

from oracle.icwf import Icwf as Oracle, Params
from oracle.sampler import sample_positions
from workloads import cavity, shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def s_norm_rel(C, Cref, S):
    d = C - Cref
    return float(np.sqrt(abs((d.conj() @ S @ d).real)) / np.sqrt(abs((Cref.conj() @ S @ Cref).real)))


def oracle_for(w, coeff_scheme=0):
    p = Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
               w.n_traj, w.svd_rel_cutoff, w.s_reg_eps)
    return Oracle(p, w.V)


def small_sm(**kw):
    d = dict(nx=64, x_range=(-25.0, 25.0), nR=32, R_range=(-9.0, 9.0), n_traj=8, dt=0.1,
             n_steps=5)
    d.update(kw)
    return shin_metiu(**d)


@pytest.fixture(scope="module")
def sm_tiny():
    """Shin-Metiu, 128 x 64 grid on [-50,50] x [-9,9], N = 16, dt = 0.1, FP64, full rank."""
    return shin_metiu()


def run_gpu(w, n_steps, seed=0, positions=None, **over):
    sim = g.Icwf(g.params_from(w, **over), w.V)
    if w.phi is not None:
        sim.set_projectors(w.phi)
    if positions is None:
        sim.init_from_density(w.psi0, seed)
    else:
        sim.init_from_positions(w.psi0, *positions)
    states = [(sim.state(), sim.matrices())]
    if n_steps:
        sim.step(n_steps)
        states.append((sim.state(), sim.matrices()))
    return sim, states


def test_sampler_is_bitwise_identical(sm_tiny):
    w = sm_tiny
    sim, [(st, _)] = run_gpu(w, 0)
    x, R = sample_positions(w.psi0, w.n_traj, 0, w.x_min, w.x_max, w.R_min, w.R_max)
    assert np.array_equal(st["x"], x) and np.array_equal(st["R"], R)
    sim.close()
    w2 = w.with_(n_traj=300)
    sim, [(st, _)] = run_gpu(w2, 0, seed=12345)
    x, R = sample_positions(w2.psi0, 300, 12345, w.x_min, w.x_max, w.R_min, w.R_max)
    assert np.array_equal(st["x"], x) and np.array_equal(st["R"], R)
    sim.close()


def test_init_parity(sm_tiny):
    w = sm_tiny
    o = oracle_for(w)
    ost = o.init_from_density(w.psi0, 0)
    sim, [(st, m)] = run_gpu(w, 0)
    assert rel(st["psi"], ost.psi) < 1e-14 and rel(st["chi"], ost.chi) < 1e-14
    assert rel(m["S"], ost.S) < 1e-13
    assert rel(m["Heff"], ost.Heff) < 1e-12
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-10
    sim.close()


def test_one_step_parity(sm_tiny):
    w = sm_tiny
    o = oracle_for(w)
    ost = o.init_from_density(w.psi0, 0)
    o.step(ost)
    sim, [_, (st, m)] = run_gpu(w, 1)
    assert np.max(np.abs(st["x"] - ost.x)) < 1e-12 and np.max(np.abs(st["R"] - ost.R)) < 1e-12
    assert rel(st["psi"], ost.psi) < 1e-13 and rel(st["chi"], ost.chi) < 1e-13
    assert rel(m["S"], ost.S) < 1e-12
    assert rel(m["Heff"], ost.Heff) < 1e-12
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-10
    sim.close()


def test_fp64_100_steps_parity(sm_tiny):
    """The FP64 acceptance case: S, Heff, H and C to 1e-10 after 100 steps (dt = 0.1)."""
    w = sm_tiny
    o = oracle_for(w)
    ost = o.init_from_density(w.psi0, 0)
    for _ in range(100):
        o.step(ost)
    sim, [_, (st, m)] = run_gpu(w, 100)
    Hm = sim.matrices(want_H=True)["H"]
    assert rel(m["S"], ost.S) < 1e-10
    assert rel(m["Heff"], ost.Heff) < 1e-10
    assert rel(Hm, o.hamiltonian(ost.psi, ost.chi)) < 1e-10
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-10
    assert np.max(np.abs(st["x"] - ost.x)) < 1e-9 and np.max(np.abs(st["R"] - ost.R)) < 1e-10
    obs = sim.observables()
    oo = o.observables(ost, w.phi)
    assert abs(obs["norm"] - oo["norm"]) < 1e-10
    assert abs(obs["energy"] - oo["energy"]) < 1e-10
    assert np.max(np.abs(obs["pop"] - oo["pop"])) < 1e-10
    assert np.max(np.abs(obs["decoherence"] - oo["decoherence"])) < 1e-10
    assert rel(obs["rho_x"], oo["rho_x"]) < 1e-10 and rel(obs["rho_R"], oo["rho_R"]) < 1e-10
    sim.close()


@pytest.mark.parametrize("N,nx,nR", [(1, 16, 8), (37, 64, 32), (70, 128, 16)])
def test_ragged_and_degenerate_sizes(N, nx, nR):
    """Trajectory counts that leave partial 32-wide tiles, N = 1, and grids down to 8 points."""
    w = small_sm(n_traj=N, nx=nx, nR=nR, R_range=(-7.0, 7.0))
    o = oracle_for(w)
    ost = o.init_from_density(w.psi0, 3)
    C0 = ost.C.copy()
    for _ in range(4):
        o.step(ost)
    sim, [_, (st, m)] = run_gpu(w, 4, seed=3)
    assert rel(m["S"], ost.S) < 1e-11
    assert rel(m["Heff"], ost.Heff) < 1e-11
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-9
    if N == 1:
        # |C| is constant in continuous time (real 1 x 1 Heff); RK4 changes it by O((h dt)^6)
        assert abs(abs(st["C"][0]) - abs(C0[0])) < 1e-9
    sim.close()


def test_frozen_coefficient_scheme():
    w = small_sm()
    p = Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
               w.n_traj, w.svd_rel_cutoff, w.s_reg_eps)
    o = Oracle(p, w.V)
    ost = o.init_from_density(w.psi0, 0)
    for _ in range(5):
        o.step(ost, freeze_matrices=True)
    sim, [_, (st, m)] = run_gpu(w, 5, coeff_scheme=1)
    assert rel(m["S"], ost.S) < 1e-12
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-10
    sim.close()


def test_truncated_rank_and_cavity():
    """Rank-k truncation (cutoff 1e-6) on Shin-Metiu and the exactly rank-1 cavity coupling."""
    w = small_sm(svd_rel_cutoff=1e-6)
    o = oracle_for(w)
    ost = o.init_from_density(w.psi0, 1)
    for _ in range(3):
        o.step(ost)
    sim, [_, (st, m)] = run_gpu(w, 3, seed=1)
    assert sim.info()["rank"] == len(o.fac.s)
    assert rel(m["Heff"], ost.Heff) < 1e-11
    sim.close()
    wc = cavity(nx=128, x_range=(-30.0, 30.0), nq=32, q_range=(-10.0, 10.0), n_traj=12,
                svd_rel_cutoff=1e-12, dt=0.05)
    o = oracle_for(wc)
    ost = o.init_from_density(wc.psi0, 0)
    for _ in range(5):
        o.step(ost)
    sim, [_, (st, m)] = run_gpu(wc, 5)
    assert sim.info()["rank"] == 1
    assert rel(m["S"], ost.S) < 1e-11 and rel(m["Heff"], ost.Heff) < 1e-11
    assert s_norm_rel(st["C"], ost.C, ost.S) < 1e-9
    sim.close()


def test_paper_scale_sampled_matrix_elements():
    """1024 x 512 Shin-Metiu grid, N = 1024 (the bench's launch configuration, FP64): after one
    step, sampled entries of S and Heff equal the oracle's formulas evaluated one by one on the
    GPU's own CWFs and positions; positions equal the oracle's Eq. v1/v2 evaluation."""
    w = shin_metiu(nx=1024, x_range=(-100.0, 100.0), nR=512, R_range=(-9.5, 9.5), n_traj=1024,
                   dt=0.05, svd_rel_cutoff=1e-12)
    sim = g.Icwf(g.params_from(w), w.V)
    sim.init_from_density(w.psi0, 0)
    before = sim.state()
    sim.step(1)
    st = sim.state()
    m = sim.matrices()
    o = oracle_for(w)
    rng = np.random.default_rng(0)
    a_idx = rng.integers(0, 1024, 6)
    b_idx = rng.integers(0, 1024, 6)
    cols = np.unique(np.concatenate([a_idx, b_idx]))
    psi, chi = st["psi"][:, cols], st["chi"][:, cols]
    S_o = o.overlaps(psi, chi)[2]
    H_o = o.heff_factorised(psi, chi, st["x"][cols], st["R"][cols])
    pos = {c: k for k, c in enumerate(cols)}
    for a, b in zip(a_idx, b_idx):
        assert abs(m["S"][a, b] - S_o[pos[a], pos[b]]) < 1e-12
        assert abs(m["Heff"][a, b] - H_o[pos[a], pos[b]]) < 1e-10 * np.max(np.abs(H_o))
    # velocities of a few trajectories from the state before the step
    from oracle.icwf import State
    sb = State(psi=before["psi"], chi=before["chi"], C=before["C"], x=before["x"], R=before["R"],
               S=None, Heff=None)
    vx, vR = o.velocities(sb)
    for a in a_idx:
        assert abs(st["x"][a] - np.clip(before["x"][a] + w.dt * vx[a], o.x[0], o.x[-1])) < 1e-11
        assert abs(st["R"][a] - np.clip(before["R"][a] + w.dt * vR[a], o.R[0], o.R[-1])) < 1e-12
    sim.close()


def test_errors_and_call_order():
    w = small_sm()
    sim = g.Icwf(g.params_from(w), w.V)
    with pytest.raises(g.IcwfError) as e:
        sim.step(1)
    assert e.value.status == g.ICWF_ERR_STATE
    with pytest.raises(g.IcwfError):
        sim.init_from_density(np.zeros_like(w.psi0), 0)     # zero density cannot be sampled
    sim.init_from_density(w.psi0, 0)
    sim.step(0)
    sim.close()
