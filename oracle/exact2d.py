"""Exact solver of the full two-coordinate TDSE (Eq. TDSE, no vector potential), oracle part 2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Strang split-operator on the periodic (x, R) grid with the same V table, masses, grid and dt as
the ICWF run it is compared with:
Psi <- e^{-i V dt/2} F2^-1 e^{-i (kx^2/2m_x + kR^2/2m_R) dt} F2 e^{-i V dt/2} Psi.
It is the "exact results" curve of the paper's figures, recomputed here.
Parity pinned: norm conservation, energy conservation without drift, separable V with a product
state equals the product of two 1D Strang propagations (tests).
"""
import numpy as np

from .icwf import grid_observables, wavenumbers
from .sampler import cell_centres


class Exact2D:
    def __init__(self, nx, nR, x_min, x_max, R_min, R_max, mass_x, mass_R, dt, V):
        self.x, self.dx = cell_centres(nx, x_min, x_max)
        self.R, self.dR = cell_centres(nR, R_min, R_max)
        self.kx = wavenumbers(nx, self.dx)
        self.kR = wavenumbers(nR, self.dR)
        self.mass_x, self.mass_R, self.dt = mass_x, mass_R, dt
        self.V = np.asarray(V, dtype=np.float64)
        self.half = np.exp(-0.5j * dt * self.V)
        T = (self.kx ** 2 / (2 * mass_x))[:, None] + (self.kR ** 2 / (2 * mass_R))[None, :]
        self.kin = np.exp(-1j * dt * T)

    def step(self, Psi: np.ndarray) -> np.ndarray:
        g = self.half * Psi
        g = np.fft.ifft2(self.kin * np.fft.fft2(g))
        return self.half * g

    def run(self, Psi: np.ndarray, n_steps: int) -> np.ndarray:
        for _ in range(n_steps):
            Psi = self.step(Psi)
        return Psi

    def observables(self, Psi, phi=None) -> dict:
        return grid_observables(Psi, self.V, self.dx, self.dR, self.kx, self.kR, self.mass_x,
                                self.mass_R, phi)
