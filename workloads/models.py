"""Model Hamiltonians of the paper's two applications, tabulated as synthetic inputs.

* Shin-Metiu proton-coupled electron transfer: one electron (x) and one proton (R) on a line
  between two fixed ions at +-L/2 (the paper's first application; its parameters live in an
  appendix that is not part of the paper, so the standard set L = 19, R_f = 5, R_l = 3.1,
  R_r = 4, proton mass 1836 is used).  Initial state: the first excited BO state times a nuclear
  Gaussian (the paper's description of its initial condition).
* One electron in a single-mode cavity, photon displacement q in the role of R with unit mass
  (the paper's second application).  The atom is the soft-Coulomb well -1/sqrt(x^2 + 1); the
  cavity frequency is the atom's 0 -> 1 gap; coupling omega*lambda*q*x plus the dipole
  self-energy (lambda x)^2 / 2.  Initial state: first excited atomic state times the photon
  vacuum.

Grids are cell-centred, x_i = lo + (i + 1/2) dx, which keeps every node off the ion positions.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os
from dataclasses import dataclass, field, replace

import numpy as np
import scipy.linalg
from scipy.special import erf


def cell_grid(n: int, lo: float, hi: float):
    d = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * d, d


def _erf_over(d: np.ndarray, a: float) -> np.ndarray:
    """erf(d / a) / d with its finite d -> 0 limit 2 / (a sqrt(pi)) (1 - d^2 / (3 a^2))."""
    d = np.asarray(d, dtype=np.float64)
    out = np.empty_like(d)
    small = d < 1e-6
    out[~small] = erf(d[~small] / a) / d[~small]
    out[small] = 2.0 / (a * math.sqrt(math.pi)) * (1.0 - d[small] ** 2 / (3.0 * a * a))
    return out


def shin_metiu_potential(x, R, L=19.0, Rf=5.0, Rl=3.1, Rr=4.0):
    """V(x, R) = 1/|L/2 - R| + 1/|L/2 + R| - erf(|R - x|/Rf)/|R - x|
                 - erf(|x - L/2|/Rr)/|x - L/2| - erf(|x + L/2|/Rl)/|x + L/2|, table [i, j]."""
    X, RR = np.meshgrid(np.asarray(x, float), np.asarray(R, float), indexing="ij")
    return (1.0 / np.abs(L / 2 - RR) + 1.0 / np.abs(L / 2 + RR)
            - _erf_over(np.abs(RR - X), Rf)
            - _erf_over(np.abs(X - L / 2), Rr)
            - _erf_over(np.abs(X + L / 2), Rl))


def soft_coulomb(x):
    return -1.0 / np.sqrt(np.asarray(x, float) ** 2 + 1.0)


def cavity_potential(x, q, omega, lam):
    """V(x, q) = -1/sqrt(x^2+1) + omega^2 q^2 / 2 + omega lambda q x + (lambda x)^2 / 2."""
    X, Q = np.meshgrid(np.asarray(x, float), np.asarray(q, float), indexing="ij")
    return soft_coulomb(X) + 0.5 * omega ** 2 * Q ** 2 + omega * lam * Q * X + 0.5 * (lam * X) ** 2


def fourier_kinetic_matrix(n: int, d: float, mass: float) -> np.ndarray:
    """Dense real-symmetric matrix of -1/(2m) d^2/dx^2 on the periodic grid (FFT definition)."""
    m = np.arange(n)
    m = np.where(m < n // 2, m, m - n)
    k = 2.0 * np.pi * m / (n * d)
    T = np.fft.ifft((k * k / (2.0 * mass))[:, None] * np.fft.fft(np.eye(n), axis=0), axis=0)
    T = T.real
    return 0.5 * (T + T.T)


def _lowest(H: np.ndarray, n_states: int):
    return scipy.linalg.eigh(H, subset_by_index=[0, n_states - 1], driver="evr")


def bo_states(V: np.ndarray, dx: float, mass_x: float, n_states: int = 3, threads: int | None = None):
    """Lowest n_states eigenpairs of H_el(R_j) = T_x + V(., R_j) for every column j of V.

    Returns (E (nR x n_s), phi (n_s x nR x nx)), phi real and normalised with dx.  Sign gauge:
    the largest-|.| entry of phi_n(.; R_0) is positive; thereafter phi_n(.; R_j) is flipped when
    its overlap with phi_n(.; R_{j-1}) is negative (continuity in R).
    """
    nx, nR = V.shape
    T = fourier_kinetic_matrix(nx, dx, mass_x)
    threads = threads or min(16, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda j: _lowest(T + np.diag(V[:, j]), n_states), range(nR)))
    E = np.array([r[0] for r in res])
    phi = np.stack([r[1].T for r in res], axis=1) / math.sqrt(dx)      # n_s x nR x nx
    for n in range(n_states):
        i = int(np.argmax(np.abs(phi[n, 0])))
        if phi[n, 0, i] < 0:
            phi[n, 0] *= -1.0
        for j in range(1, nR):
            if np.dot(phi[n, j], phi[n, j - 1]) < 0:
                phi[n, j] *= -1.0
    return E, phi


@dataclass
class Workload:
    """A synthetic ICWF problem: grids, masses, dt, N, V table, Psi0, BO projectors."""
    name: str
    nx: int
    nR: int
    x_min: float
    x_max: float
    R_min: float
    R_max: float
    mass_x: float
    mass_R: float
    dt: float
    n_traj: int
    n_steps: int
    svd_rel_cutoff: float = 0.0
    s_reg_eps: float = 1e-6
    seed: int = 0
    model: dict = field(default_factory=dict)
    V: np.ndarray | None = None
    psi0: np.ndarray | None = None
    phi: np.ndarray | None = None
    bo_energies: np.ndarray | None = None

    @property
    def x(self):
        return cell_grid(self.nx, self.x_min, self.x_max)[0]

    @property
    def R(self):
        return cell_grid(self.nR, self.R_min, self.R_max)[0]

    @property
    def dx(self):
        return (self.x_max - self.x_min) / self.nx

    @property
    def dR(self):
        return (self.R_max - self.R_min) / self.nR

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _normalise(psi0, dx, dR):
    return psi0 / math.sqrt(dx * dR * float(np.sum(np.abs(psi0) ** 2)))


def shin_metiu(nx=128, x_range=(-50.0, 50.0), nR=64, R_range=(-9.0, 9.0), n_traj=16, dt=0.1,
               n_steps=100, R0=-4.0, width=1.0 / math.sqrt(2.85), Rf=5.0, Rl=3.1, Rr=4.0, L=19.0,
               mass_R=1836.0, n_states=3, svd_rel_cutoff=0.0, s_reg_eps=1e-6, seed=0,
               name="shin_metiu") -> Workload:
    """Shin-Metiu PCET: Psi0(x, R) = exp(-(R - R0)^2 / (2 width^2)) phi_1(x; R), normalised."""
    x, dx = cell_grid(nx, *x_range)
    R, dR = cell_grid(nR, *R_range)
    V = shin_metiu_potential(x, R, L=L, Rf=Rf, Rl=Rl, Rr=Rr)
    E, phi = bo_states(V, dx, 1.0, n_states=max(n_states, 2))
    g = np.exp(-((R - R0) ** 2) / (2.0 * width ** 2))
    psi0 = _normalise((phi[1].T * g[None, :]).astype(np.complex128), dx, dR)
    return Workload(name=name, nx=nx, nR=nR, x_min=x_range[0], x_max=x_range[1],
                    R_min=R_range[0], R_max=R_range[1], mass_x=1.0, mass_R=mass_R, dt=dt,
                    n_traj=n_traj, n_steps=n_steps, svd_rel_cutoff=svd_rel_cutoff,
                    s_reg_eps=s_reg_eps, seed=seed,
                    model=dict(kind="shin_metiu", R0=R0, width=width, Rf=Rf, Rl=Rl, Rr=Rr, L=L),
                    V=V, psi0=psi0, phi=phi[:n_states], bo_energies=E[:, :n_states])


def atom_levels(nx, x_range, n=3):
    x, dx = cell_grid(nx, *x_range)
    H = fourier_kinetic_matrix(nx, dx, 1.0) + np.diag(soft_coulomb(x))
    E, v = _lowest(H, n)
    return E, v.T / math.sqrt(dx)


def cavity(nx=2048, x_range=(-80.0, 80.0), nq=256, q_range=(-30.0, 30.0), lam=0.5,
           n_traj=1024, dt=0.01, n_steps=100, n_states=3, svd_rel_cutoff=1e-12,
           s_reg_eps=1e-4, seed=0, name="cavity", q0=0.0, p0=0.0) -> Workload:
    """Electron in a resonant single-mode cavity; Psi0 = phi_1^atom(x) times the photon state
    (w/pi)^(1/4) e^{-w (q - q0)^2 / 2 + i p0 q}: the vacuum for q0 = p0 = 0 (the default), else a
    coherent state displaced to <q> = q0, <p> = p0 (the displaced coherent photon state of the
    paper's cavity discussion).

    dt = 0.01 a.u.: the product initial state makes every CWF the same, so S starts with rank one
    while the trajectories' pinned potentials differ widely; the regularised coefficient equation
    is then stiff, and its RK4 step diverges at dt = 0.05 for every eps tried (1e-6 to 1e-3, FP64
    included) but stays stable at 0.01.  eps = 1e-4 keeps the stiffness moderate at that step."""
    x, dx = cell_grid(nx, *x_range)
    q, dq = cell_grid(nq, *q_range)
    Ea, va = atom_levels(nx, x_range, 2)
    omega = float(Ea[1] - Ea[0])
    V = cavity_potential(x, q, omega, lam)
    E, phi = bo_states(V, dx, 1.0, n_states=n_states)
    e1 = va[1] * (1.0 if va[1][np.argmax(np.abs(va[1]))] > 0 else -1.0)
    vac = (omega / math.pi) ** 0.25 * np.exp(-0.5 * omega * (q - q0) ** 2 + 1j * p0 * q)
    psi0 = _normalise(np.outer(e1, vac).astype(np.complex128), dx, dq)
    return Workload(name=name, nx=nx, nR=nq, x_min=x_range[0], x_max=x_range[1],
                    R_min=q_range[0], R_max=q_range[1], mass_x=1.0, mass_R=1.0, dt=dt,
                    n_traj=n_traj, n_steps=n_steps, svd_rel_cutoff=svd_rel_cutoff,
                    s_reg_eps=s_reg_eps, seed=seed,
                    model=dict(kind="cavity", omega=omega, lam=lam, q0=q0, p0=p0), V=V, psi0=psi0,
                    phi=phi, bo_energies=E)


# Named workloads.  Sizes follow the paper's two applications at the scales quoted with them.
WORKLOADS = {
    # Shin-Metiu, 128 x 64 grid, 16 trajectories, dt 0.1 a.u., 100 steps, FP64, full rank.
    "sm_tiny": lambda **kw: shin_metiu(**{**dict(name="sm_tiny"), **kw}),
    # Shin-Metiu at paper scale: 1024 x 512 grid on [-100,100] x [-9.5,9.5], dt 0.05 a.u.
    "sm_paper": lambda **kw: shin_metiu(**{**dict(name="sm_paper", nx=1024, x_range=(-100.0, 100.0),
                                                  nR=512, R_range=(-9.5, 9.5), n_traj=1024,
                                                  dt=0.05, n_steps=20000,
                                                  svd_rel_cutoff=1e-12), **kw}),
    # Cavity QED, 2048 x 256 grid on [-80,80] x [-30,30], lambda 0.5, dt 0.01 a.u.
    "cavity": lambda **kw: cavity(**{**dict(name="cavity"), **kw}),
}
