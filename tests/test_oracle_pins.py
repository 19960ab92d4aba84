"""Pins of the FP64 oracle to facts fixed by the paper and the mathematics (CPU only).

Each test fixes one part of ``oracle/`` against something other than the oracle itself:
closed forms of the Schroedinger equation, exact invariants of the method, brute-force sums on
tiny inputs, and published generator test vectors.  Chosen so that a dropped term, a wrong sign,
a swapped bra/ket or a missing mass factor fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle.exact2d import Exact2D
from oracle.icwf import Icwf, Params, State, factorise, lagrange4, wavenumbers
from oracle.sampler import SplitMix64, cell_centres, sample_positions
from workloads import WORKLOADS, cavity, shin_metiu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator and sampler

def test_splitmix64_published_vectors():
    seeds = {}
    cur = None
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("seed"):
            cur = int(line.split()[1])
            seeds[cur] = []
        else:
            seeds[cur].append(int(line))
    assert seeds
    for seed, outs in seeds.items():
        g = SplitMix64(seed)
        assert [g.next_u64() for _ in outs] == outs


def test_sampler_chi_square():
    """Sampled cells follow |Psi0|^2 (chi-square over coarse bins, 2e4 draws)."""
    nx, nR = 32, 16
    x, dx = cell_centres(nx, -4, 4)
    R, dR = cell_centres(nR, -2, 2)
    psi0 = np.exp(-0.5 * (x[:, None] - 0.7) ** 2 - (R[None, :] + 0.3) ** 2) * (1 + 0.5j * x[:, None])
    xs, Rs = sample_positions(psi0, 20000, 7, -4, 4, -2, 2)
    assert np.all(np.abs(xs - np.clip(xs, -4, 4)) == 0) and np.all((Rs >= -2) & (Rs <= 2))
    bx = np.clip(((xs + 4) / 8 * 4).astype(int), 0, 3)
    bR = np.clip(((Rs + 2) / 4 * 4).astype(int), 0, 3)
    obs = np.zeros((4, 4))
    np.add.at(obs, (bx, bR), 1)
    p = np.abs(psi0) ** 2
    exp = p.reshape(4, nx // 4, 4, nR // 4).sum(axis=(1, 3))
    exp = exp / exp.sum() * 20000
    keep = exp > 5
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    assert chi2 < 45.0          # 15 dof: P(chi2 > 45) < 1e-4


# ---------------------------------------------------------------- interpolation

def test_lagrange_exact_on_cubics_and_derivative():
    n, lo, hi = 40, -3.0, 5.0
    x, d = cell_centres(n, lo, hi)
    f = 0.3 * x ** 3 - 1.1 * x ** 2 + 2.0 * x - 0.5
    fp = 0.9 * x ** 2 - 2.2 * x + 2.0
    rng = np.random.default_rng(1)
    for p in np.concatenate([rng.uniform(x[0], x[-1], 50), [x[0], x[-1], x[1], x[-2]]]):
        i0, w, dw = lagrange4(p, lo, d, n)
        assert 0 <= i0 <= n - 4
        val = w @ f[i0:i0 + 4]
        der = dw @ f[i0:i0 + 4]
        assert abs(val - (0.3 * p ** 3 - 1.1 * p ** 2 + 2 * p - 0.5)) < 1e-11
        assert abs(der - (0.9 * p ** 2 - 2.2 * p + 2.0)) < 1e-10
    # on a node the stencil reproduces the sample exactly
    i0, w, dw = lagrange4(x[17], lo, d, n)
    assert np.allclose(w, [0, 1, 0, 0], atol=1e-15) and i0 == 16


# ---------------------------------------------------------------- 1D propagator (a2/a3)

def free_gaussian(x, t, x0, k0, sig, m):
    """Textbook free evolution of (2 pi sig^2)^(-1/4) exp(-(x-x0)^2/(4 sig^2) + i k0 (x-x0))."""
    a = 1.0 + 1j * t / (2.0 * m * sig ** 2)
    v = k0 / m
    return ((2 * math.pi * sig ** 2) ** -0.25 / np.sqrt(a)
            * np.exp(-((x - x0 - v * t) ** 2) / (4 * sig ** 2 * a) + 1j * k0 * (x - x0 - 0.5 * v * t)))


@pytest.mark.parametrize("m,k0,dt", [(1.0, 1.5, 0.1), (1836.0, 8.0, 5.0)])
def test_free_gaussian_closed_form(m, k0, dt):
    n, lo, hi = 512, -40.0, 40.0
    x, d = cell_centres(n, lo, hi)
    k = wavenumbers(n, d)
    n_steps = 40
    f = free_gaussian(x, 0.0, -5.0, k0, 1.3, m)
    for _ in range(n_steps):
        f = Icwf.strang(f, np.zeros(n), k, m, dt)
    ref = free_gaussian(x, n_steps * dt, -5.0, k0, 1.3, m)
    assert np.max(np.abs(f - ref)) < 1e-10


def test_harmonic_coherent_state():
    """|psi|^2 of a displaced ground state of m w^2 x^2/2 stays a Gaussian centred at
    x0 cos(w t) with the ground-state width; Strang error O(dt^2)."""
    n, lo, hi = 256, -12.0, 12.0
    x, d = cell_centres(n, lo, hi)
    k = wavenumbers(n, d)
    m, w, x0 = 2.0, 0.7, 2.5
    v = 0.5 * m * w * w * x * x
    T = 2 * math.pi / w
    errs = []
    for dt in (T / 200, T / 400):
        f = (m * w / math.pi) ** 0.25 * np.exp(-0.5 * m * w * (x - x0) ** 2) + 0j
        nst = int(round(0.37 * T / dt))
        for _ in range(nst):
            f = Icwf.strang(f, v, k, m, dt)
        t = nst * dt
        ref = math.sqrt(m * w / math.pi) * np.exp(-m * w * (x - x0 * math.cos(w * t)) ** 2)
        errs.append(np.max(np.abs(np.abs(f) ** 2 - ref)))
        assert abs(d * np.sum(x * np.abs(f) ** 2) - x0 * math.cos(w * t)) < 5e-3
    assert errs[0] < 5e-3 and 3.0 < errs[0] / errs[1] < 5.0      # second order in dt


def test_strang_unitary():
    rng = np.random.default_rng(3)
    n = 128
    x, d = cell_centres(n, -10, 10)
    k = wavenumbers(n, d)
    f = rng.normal(size=n) + 1j * rng.normal(size=n)
    n0 = np.sum(np.abs(f) ** 2)
    v = rng.uniform(-2, 5, n)
    for _ in range(200):
        f = Icwf.strang(f, v, k, 1.0, 0.05)
    assert abs(np.sum(np.abs(f) ** 2) / n0 - 1.0) < 1e-12


# ---------------------------------------------------------------- exact 2D solver

def _tiny_sm():
    return shin_metiu(nx=64, x_range=(-25.0, 25.0), nR=32, R_range=(-9.0, 9.0), n_traj=6,
                      n_steps=10, dt=0.1)


def test_exact2d_norm_and_energy():
    w = _tiny_sm()
    ex = Exact2D(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, 0.1, w.V)
    P = w.psi0.copy()
    o0 = ex.observables(P)
    es = []
    for _ in range(5):
        P = ex.run(P, 200)
        o = ex.observables(P)
        assert abs(o["norm"] - o0["norm"]) < 1e-12
        es.append(o["energy"])
    # Strang conserves a modified energy: fluctuation bounded, no drift
    assert max(abs(e - o0["energy"]) for e in es) < 2e-3


def test_exact2d_separable_equals_product():
    nx, nR = 64, 32
    x, dx = cell_centres(nx, -10, 10)
    R, dR = cell_centres(nR, -6, 6)
    v1 = 0.5 * 0.3 * x ** 2
    v2 = 0.5 * 4.0 * 0.05 * R ** 2 + 0.1 * R
    V = v1[:, None] + v2[None, :]
    f = np.exp(-0.5 * (x - 1) ** 2) + 0j
    g = np.exp(-0.5 * (R + 0.5) ** 2 / 0.5) * np.exp(0.3j * R)
    ex = Exact2D(nx, nR, -10, 10, -6, 6, 1.0, 4.0, 0.05, V)
    P = ex.run(np.outer(f, g), 50)
    kx, kR = wavenumbers(nx, dx), wavenumbers(nR, dR)
    for _ in range(50):
        f = Icwf.strang(f, v1, kx, 1.0, 0.05)
        g = Icwf.strang(g, v2, kR, 4.0, 0.05)
    assert np.max(np.abs(P - np.outer(f, g))) < 1e-12


# ---------------------------------------------------------------- matrix elements (a5)

def _params(w, **kw):
    d = dict(nx=w.nx, nR=w.nR, x_min=w.x_min, x_max=w.x_max, R_min=w.R_min, R_max=w.R_max,
             mass_x=w.mass_x, mass_R=w.mass_R, dt=w.dt, n_traj=w.n_traj,
             svd_rel_cutoff=w.svd_rel_cutoff, s_reg_eps=w.s_reg_eps)
    d.update(kw)
    return Params(**d)


def test_brute_force_matrix_elements():
    """Quadruple loops over the grid on tiny random CWFs, trajectories on grid nodes (where the
    pinned potential is a column / row of V exactly): S and Heff of the oracle agree."""
    rng = np.random.default_rng(5)
    nx, nR, N = 8, 6, 3
    V = rng.normal(size=(nx, nR))
    p = Params(nx, nR, -2.0, 2.0, -1.5, 1.5, 1.0, 3.0, 0.1, N, 0.0, 1e-10)
    o = Icwf(p, V)
    psi = rng.normal(size=(nx, N)) + 1j * rng.normal(size=(nx, N))
    chi = rng.normal(size=(nR, N)) + 1j * rng.normal(size=(nR, N))
    ix = [2, 5, 3]
    jR = [1, 4, 2]
    x = o.x[ix]
    R = o.R[jR]
    S_bf = np.zeros((N, N), complex)
    H_bf = np.zeros((N, N), complex)
    for a in range(N):
        for b in range(N):
            for i in range(nx):
                for j in range(nR):
                    bra = np.conj(psi[i, a] * chi[j, a])
                    ket = psi[i, b] * chi[j, b]
                    S_bf[a, b] += o.dx * o.dR * bra * ket
                    H_bf[a, b] += o.dx * o.dR * bra * (V[i, j] - V[i, jR[b]] - V[ix[b], j]) * ket
    S, H = o.matrices(psi, chi, x, R)
    assert np.max(np.abs(S - S_bf)) < 1e-13
    assert np.max(np.abs(H - H_bf)) < 1e-12
    assert np.max(np.abs(o.heff_direct(psi, chi, x, R) - H_bf)) < 1e-12
    # Hamiltonian matrix: W part brute force, kinetic parts via the dense FFT kinetic operator
    W_bf = np.zeros((N, N), complex)
    for a in range(N):
        for b in range(N):
            W_bf[a, b] = o.dx * o.dR * np.sum(np.conj(np.outer(psi[:, a], chi[:, a])) * V
                                              * np.outer(psi[:, b], chi[:, b]))
    S1, S2, _ = o.overlaps(psi, chi)
    Tx = np.fft.ifft((o.kx ** 2 / 2)[:, None] * np.fft.fft(np.eye(nx), axis=0), axis=0)
    TR = np.fft.ifft((o.kR ** 2 / 6)[:, None] * np.fft.fft(np.eye(nR), axis=0), axis=0)
    T1 = o.dx * psi.conj().T @ Tx @ psi
    T2 = o.dR * chi.conj().T @ TR @ chi
    assert np.max(np.abs(o.hamiltonian(psi, chi) - (T1 * S2 + S1 * T2 + W_bf))) < 1e-12


def test_factorised_equals_direct_and_hermiticity():
    w = _tiny_sm()
    o = Icwf(_params(w), w.V)
    st = o.init_from_density(w.psi0, 0)
    for _ in range(3):
        o.step(st)
    S, Hf = o.matrices(st.psi, st.chi, st.x, st.R)
    Hd = o.heff_direct(st.psi, st.chi, st.x, st.R)
    assert np.max(np.abs(Hf - Hd)) < 1e-12 * np.max(np.abs(Hd))
    assert np.max(np.abs(S - S.conj().T)) < 1e-15
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-12
    H = o.hamiltonian(st.psi, st.chi)
    assert np.max(np.abs(H - H.conj().T)) < 1e-12 * np.max(np.abs(H))
    # Heff = H - i tau with tau_ab = <phi_a| d phi_b/dt> = -i <phi_a| H_b^pin |phi_b>: the
    # anti-Hermitian part of Heff comes from the pinned Hamiltonians only
    N = w.n_traj
    Hpin = np.empty((N, N), complex)
    for b in range(N):
        ve = o.pinned_e(st.R[b])
        vn = o.pinned_n(st.x[b])
        hpsi = o.kinetic(st.psi[:, [b]], o.kx, w.mass_x)[:, 0] + ve * st.psi[:, b]
        hchi = o.kinetic(st.chi[:, [b]], o.kR, w.mass_R)[:, 0] + vn * st.chi[:, b]
        S1b = o.dx * st.psi.conj().T @ st.psi[:, b]
        S2b = o.dR * st.chi.conj().T @ st.chi[:, b]
        Hpin[:, b] = (o.dx * st.psi.conj().T @ hpsi) * S2b + S1b * (o.dR * st.chi.conj().T @ hchi)
    assert np.max(np.abs(Hd - (H - Hpin))) < 1e-11 * np.max(np.abs(H))


def test_cavity_interaction_is_rank_one():
    w = cavity(nx=256, x_range=(-40.0, 40.0), nq=64, q_range=(-15.0, 15.0), n_traj=4, lam=0.7)
    f = factorise(w.V, 1e-13)
    assert len(f.s) == 1 and f.tail_rel < 1e-13
    f0 = factorise(w.V, 0.0)
    assert f0.s[1] / f0.s[0] < 1e-13


def test_factorisation_truncation_rule():
    w = _tiny_sm()
    f = factorise(w.V, 1e-6)
    assert f.tail_rel <= 1e-6
    g = factorise(w.V, 0.0)
    k = len(f.s)
    # one fewer singular value would violate the cutoff
    assert np.sqrt(np.sum(g.s[k - 1:] ** 2)) / np.sqrt(np.sum(g.s ** 2)) > 1e-6
    rec = g.v1[:, None] + g.v2[None, :] + (g.u * g.s) @ g.w.T
    assert np.max(np.abs(rec - w.V)) < 1e-12 * np.max(np.abs(w.V))


# ---------------------------------------------------------------- velocities (a4)

def test_velocity_of_moving_gaussian():
    """One trajectory at the centre of a Gaussian packet with momenta (kx, kR) moves with
    (kx / m_x, kR / m_R) (Eq. v1/v2 with the 1/m factor and the Im sign)."""
    nx, nR = 256, 128
    p = Params(nx, nR, -20.0, 20.0, -10.0, 10.0, 1.0, 50.0, 0.01, 1, 0.0, 1e-10)
    o = Icwf(p, np.zeros((nx, nR)))
    k1, k2 = 0.8, -1.5
    xa, Ra = 1.234, -0.77
    psi = np.exp(-0.5 * (o.x - xa) ** 2 + 1j * k1 * o.x)[:, None]
    chi = np.exp(-0.5 * (o.R - Ra) ** 2 + 1j * k2 * o.R)[:, None]
    st = State(psi=psi, chi=chi, C=np.array([0.3 - 0.4j]), x=np.array([xa]), R=np.array([Ra]),
               S=None, Heff=None)
    vx, vR = o.velocities(st)
    # relative interpolation error of the cubic stencil on a resolved packet (k dx < 0.25)
    assert abs(vx[0] / (k1 / 1.0) - 1) < 1e-3 and abs(vR[0] / (k2 / 50.0) - 1) < 1e-3


# ---------------------------------------------------------------- coefficients (a6)

def test_rk4_matches_matrix_exponential():
    """Constant S, Heff: C(t) = exp(-i (S + eps I)^-1 Heff t) C0 to O(dt^4)."""
    import scipy.linalg
    rng = np.random.default_rng(2)
    N = 5
    A = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    S = A.conj().T @ A / N + np.eye(N)
    H = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    p = Params(8, 8, 0, 1, 0, 1, 1, 1, 0.01, N, 0.0, 1e-10)
    o = Icwf(p, np.zeros((8, 8)))
    C0 = rng.normal(size=N) + 1j * rng.normal(size=N)
    errs = []
    for dt in (0.02, 0.01):
        o.p.dt = dt
        C = C0.copy()
        n = int(round(0.4 / dt))
        for _ in range(n):
            C = o.rk4(C, S, H, S, H)
        ref = scipy.linalg.expm(-1j * np.linalg.solve(S + 1e-10 * np.eye(N), H) * 0.4) @ C0
        errs.append(np.max(np.abs(C - ref)))
    assert errs[0] < 1e-6 and 12 < errs[0] / errs[1] < 20      # fourth order


# ---------------------------------------------------------------- whole method

def test_norm_conserved_to_second_order():
    """C^H S C is conserved by the continuous ICWF equations; the discrete step keeps it to
    O(dt^2) (Strang CWFs, S and Heff linear over the step)."""
    w = _tiny_sm()
    devs = []
    for dt, n in ((0.1, 40), (0.05, 80)):
        o = Icwf(_params(w, dt=dt, s_reg_eps=1e-10), w.V)
        st = o.init_from_density(w.psi0, 0)
        n0 = (st.C.conj() @ st.S @ st.C).real
        for _ in range(n):
            o.step(st)
        devs.append(abs((st.C.conj() @ st.S @ st.C).real - n0))
    assert devs[0] < 1e-5 and 3.0 < devs[0] / devs[1] < 5.0


def test_separable_potential_product_state_is_exact():
    """V = v1(x) + v2(R) and Psi0 = f(x) g(R): every CWF stays proportional to the exact factor, so
    the ICWF wavefunction equals the exact 2D solution for any N (here N = 1 and N = 4), to
    integrator error."""
    nx, nR = 64, 32
    x, dx = cell_centres(nx, -12, 12)
    R, dR = cell_centres(nR, -6, 6)
    V = (0.5 * 0.4 * x ** 2 + 0.2 * x)[:, None] + (0.5 * 5.0 * 0.2 * R ** 2)[None, :]
    psi0 = np.outer(np.exp(-0.5 * (x - 1.0) ** 2), np.exp(-(R + 0.4) ** 2)).astype(complex)
    psi0 /= np.sqrt(dx * dR * np.sum(np.abs(psi0) ** 2))
    ex = Exact2D(nx, nR, -12, 12, -6, 6, 1.0, 5.0, 0.02, V)
    Pex = ex.run(psi0, 100)
    for N in (1, 4):
        p = Params(nx, nR, -12, 12, -6, 6, 1.0, 5.0, 0.02, N, 0.0, 1e-10)
        o = Icwf(p, V)
        st = o.init_from_density(psi0, 11)
        C0 = st.C.copy()
        for _ in range(100):
            o.step(st)
        P = o.wavefunction(st)
        assert np.max(np.abs(P - Pex)) < 2e-4 * np.max(np.abs(Pex))
        if N == 1:
            assert abs(abs(st.C[0]) - abs(C0[0])) < 1e-12


def test_observables_agree_with_matrix_forms():
    """Grid observables of the ansatz agree with the matrix forms: norm = C^H S C and
    energy = C^H H C / C^H S C; densities integrate to the norm; populations <= norm."""
    w = _tiny_sm()
    o = Icwf(_params(w), w.V)
    st = o.init_from_density(w.psi0, 0)
    for _ in range(5):
        o.step(st)
    ob = o.observables(st, w.phi)
    nS = (st.C.conj() @ st.S @ st.C).real
    H = o.hamiltonian(st.psi, st.chi)
    assert abs(ob["norm"] - nS) < 1e-12
    assert abs(ob["energy"] - (st.C.conj() @ H @ st.C).real / nS) < 1e-10
    assert abs(w.dx * ob["rho_x"].sum() - ob["norm"]) < 1e-12
    assert abs(w.dR * ob["rho_R"].sum() - ob["norm"]) < 1e-12
    assert np.all(ob["pop"] >= 0) and ob["pop"].sum() <= ob["norm"] + 1e-12
    D = ob["decoherence"]
    assert np.allclose(D, D.T) and np.all(D >= 0)


# ---------------------------------------------------------------- populations and decoherence

def _bo_superposition(w, a_of_R, b_of_R, n_lo=0, n_hi=2):
    """Psi(x, R) = a(R) phi_lo(x; R) + b(R) phi_hi(x; R) on the workload's grid."""
    return (a_of_R[None, :] * w.phi[n_lo].T + b_of_R[None, :] * w.phi[n_hi].T).astype(complex)


def _closed_form_pop(w, a_of_R, b_of_R, n_lo=0, n_hi=2):
    """The BO states are orthonormal on the x grid at every R_j, so chi^(lo) = a, chi^(hi) = b,
    the third projection vanishes, rho_R = |a|^2 + |b|^2, P_n = int dR |chi^(n)|^2 and
    D_nm = int dR |chi^(n)|^2 |chi^(m)|^2 (the Shin-Metiu discussion's indicator)."""
    ns = w.phi.shape[0]
    chin = np.zeros((ns, w.nR), complex)
    chin[n_lo] = a_of_R
    chin[n_hi] = b_of_R
    pn = np.abs(chin) ** 2
    return pn.sum(axis=1) * w.dR, w.dR * (pn[:, None, :] * pn[None, :, :]).sum(axis=2), \
        np.abs(a_of_R) ** 2 + np.abs(b_of_R) ** 2


def _assert_obs(ob, pop, D, rhoR):
    assert np.max(np.abs(ob["pop"] - pop)) < 1e-12
    assert np.max(np.abs(ob["decoherence"] - D)) < 1e-12 * max(1.0, np.max(D))
    assert np.max(np.abs(ob["rho_R"] - rhoR)) < 1e-12 * np.max(rhoR)


def test_initial_state_populations_and_decoherence_closed_form():
    """Psi0 = g(R) phi_1(x; R) (the Shin-Metiu initial state) has P = (0, 1, 0) and
    D_11 = int dR |g|^4 with g the normalised nuclear Gaussian, every other D_nm zero; checked
    through the exact solver's observables and through an ICWF state whose basis reproduces
    Psi0 (chi_a = grid delta at R_a, psi_a = g(R_a) phi_1(.; R_a))."""
    w = _tiny_sm()
    g = np.exp(-((w.R - w.model["R0"]) ** 2) / (2.0 * w.model["width"] ** 2))
    g = g / np.sqrt(w.dR * np.sum(g ** 2))
    pop, D, rhoR = _closed_form_pop(w, np.zeros(w.nR), g, n_lo=0, n_hi=1)
    assert abs(pop[1] - 1.0) < 1e-12 and abs(D[1, 1] - w.dR * np.sum(g ** 4)) < 1e-15
    ex = Exact2D(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt, w.V)
    _assert_obs(ex.observables(w.psi0, w.phi), pop, D, rhoR)
    o = Icwf(_params(w, n_traj=w.nR), w.V)
    theta = np.linspace(0.3, 2.9, w.nR)                        # complex C, compensated in psi
    psi = (w.phi[1].T * (g * np.exp(-1j * theta))[None, :])   # column a = g(R_a) phi_1(x; R_a)
    chi = np.eye(w.nR, dtype=complex)                          # chi_a(R_j) = delta_aj
    st = State(psi=psi, chi=chi, C=np.exp(1j * theta), x=np.zeros(w.nR), R=w.R.copy(),
               S=None, Heff=None)
    assert np.max(np.abs(o.wavefunction(st) - w.psi0)) < 1e-13 * np.max(np.abs(w.psi0))
    _assert_obs(o.observables(st, w.phi), pop, D, rhoR)


def test_superposition_populations_and_decoherence_closed_form():
    """Psi = a(R) phi_0 + b(R) phi_2 with unequal complex nuclear factors: P_0 = int |a|^2,
    P_1 = 0, P_2 = int |b|^2, D_02 = int |a|^2 |b|^2 dR (a dropped dx, a transposed projector or
    a wrong squared modulus fails)."""
    w = _tiny_sm()
    a = np.exp(-((w.R + 2.0) ** 2) / 2.0) * np.exp(0.7j * w.R)
    b = 0.6 * np.exp(-((w.R - 1.0) ** 2) / 3.0) * (1.0 - 0.4j * w.R)
    pop, D, rhoR = _closed_form_pop(w, a, b)
    assert pop[1] == 0.0 and D[0, 2] > 1e-3 and abs(pop[0] - pop[2]) > 0.1
    Psi = _bo_superposition(w, a, b)
    ex = Exact2D(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt, w.V)
    ob = ex.observables(Psi, w.phi)
    _assert_obs(ob, pop, D, rhoR)
    assert abs(ob["norm"] - (pop[0] + pop[2])) < 1e-12


# ---------------------------------------------------------------- velocities, several terms

def test_velocity_of_two_boosted_gaussians():
    """N = 2 basis functions psi_b chi_b (Gaussians with their own centres and momenta) and
    unequal complex C: Eq. v1/v2 at a trajectory's position equals the closed form
    Im(d_x Psi / Psi) / m_x, Im(d_R Psi / Psi) / m_R with
    d_x psi_b = (-(x - x_b) / s^2 + i k_b) psi_b.  C does not cancel, so using C_a for C_b, a
    conjugate, or a factor at the wrong point fails."""
    nx, nR = 1024, 1024       # cells of 0.02: the stencil's O(dx^3) derivative error ~1e-6
    mx, mR = 1.0, 40.0
    p = Params(nx, nR, -10.0, 10.0, -10.0, 10.0, mx, mR, 0.01, 2, 0.0, 1e-10)
    o = Icwf(p, np.zeros((nx, nR)))
    s = 1.3
    xc, kx = np.array([-0.8, 1.1]), np.array([0.9, -0.6])
    Rc, kR = np.array([0.5, -0.7]), np.array([-1.2, 0.8])
    C = np.array([0.9 - 0.3j, -0.4 + 0.7j])

    def g(z, zc, k):
        return np.exp(-((z - zc) ** 2) / (2 * s * s) + 1j * k * z)

    def dg(z, zc, k):
        return (-(z - zc) / (s * s) + 1j * k) * g(z, zc, k)

    psi = np.stack([g(o.x, xc[b], kx[b]) for b in range(2)], axis=1)
    chi = np.stack([g(o.R, Rc[b], kR[b]) for b in range(2)], axis=1)
    rng = np.random.default_rng(9)
    checked = 0
    for _ in range(6):
        xa = rng.uniform(-1.5, 1.5, 2)
        Ra = rng.uniform(-1.2, 1.2, 2)
        st = State(psi=psi, chi=chi, C=C, x=xa, R=Ra, S=None, Heff=None)
        vx, vR = o.velocities(st)
        for a in range(2):
            P = sum(C[b] * g(xa[a], xc[b], kx[b]) * g(Ra[a], Rc[b], kR[b]) for b in range(2))
            Px = sum(C[b] * dg(xa[a], xc[b], kx[b]) * g(Ra[a], Rc[b], kR[b]) for b in range(2))
            PR = sum(C[b] * g(xa[a], xc[b], kx[b]) * dg(Ra[a], Rc[b], kR[b]) for b in range(2))
            ex_vx, ex_vR = (Px / P).imag / mx, (PR / P).imag / mR
            assert abs(vx[a] - ex_vx) < 1e-5 * max(1.0, abs(ex_vx))
            assert abs(vR[a] - ex_vR) < 1e-5 * max(1.0 / mR, abs(ex_vR))
            checked += 1
    assert checked == 12


# ---------------------------------------------------------------- RK4 with moving matrices

def test_rk4_with_linear_matrices_matches_fine_integrator():
    """S(t), Heff(t) linear in t over the whole interval (so the per-step interpolation between
    the endpoint assemblies is exact): the RK4 of Eq. coeff converges at fourth order to an
    independent adaptive integrator (scipy DOP853, rtol 1e-12) of dC/dt = -i (S(t) + eps I)^-1
    Heff(t) C.  Freezing the matrices at t_n, or using the endpoint matrices at the half-step
    stages, drops the order and fails the ratio."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(4)
    N, T = 4, 0.6
    A0 = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    A1 = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    S0 = A0.conj().T @ A0 / N + np.eye(N)
    S1 = A1.conj().T @ A1 / N + np.eye(N)
    H0 = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    H1 = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    eps = 1e-10
    St = lambda t: S0 + (t / T) * (S1 - S0)
    Ht = lambda t: H0 + (t / T) * (H1 - H0)
    C0 = rng.normal(size=N) + 1j * rng.normal(size=N)

    def rhs(t, c):
        return -1j * np.linalg.solve(St(t) + eps * np.eye(N), Ht(t) @ c)

    ref = solve_ivp(rhs, (0.0, T), C0, method="DOP853", rtol=1e-12, atol=1e-14).y[:, -1]
    p = Params(8, 8, 0, 1, 0, 1, 1, 1, 0.01, N, 0.0, eps)
    o = Icwf(p, np.zeros((8, 8)))
    errs = []
    for n in (20, 40):
        dt = T / n
        o.p.dt = dt
        C = C0.copy()
        for k in range(n):
            C = o.rk4(C, St(k * dt), Ht(k * dt), St((k + 1) * dt), Ht((k + 1) * dt))
        errs.append(np.max(np.abs(C - ref)))
    assert errs[0] < 1e-5 and 12 < errs[0] / errs[1] < 20      # fourth order


def test_displaced_coherent_photon_follows_the_classical_oscillator():
    """The cavity's displaced coherent photon state at lambda = 0 (V separable: atom + w^2 q^2/2,
    photon mass 1): under the exact solver <q>(t) = q0 cos(w t) + (p0 / w) sin(w t) and the width
    stays that of the vacuum (a coherent state), to Strang O(dt^2)."""
    w = cavity(nx=256, x_range=(-40.0, 40.0), nq=128, q_range=(-25.0, 25.0), lam=0.0, n_traj=4,
               q0=3.0, p0=-0.4)
    om = w.model["omega"]
    dt = 0.02
    ex = Exact2D(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, dt, w.V)
    P = w.psi0.copy()
    q = w.R
    for n in range(4):
        rhoq = ex.observables(P)["rho_R"]
        t = n * 150 * dt
        mean = w.dR * np.sum(q * rhoq)
        var = w.dR * np.sum((q - mean) ** 2 * rhoq)
        assert abs(mean - (3.0 * np.cos(om * t) - 0.4 / om * np.sin(om * t))) < 2e-3
        assert abs(var - 0.5 / om) < 2e-3 * (0.5 / om)
        P = ex.run(P, 150)
