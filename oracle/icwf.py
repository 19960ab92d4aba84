"""Plain FP64 oracle of one Interacting-CWF (ICWF) time step, arXiv 1805.11169.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): only tests, the smoke check and the bench's
CPU baseline may import this module.

Notation (paper -> here).  Electron coordinate r -> x (grid of nx cells), nuclear or photon
coordinate R -> R (nR cells), trajectory count M -> N.  psi_1^a(r) -> psi[:, a] (column a of an
nx x N array), psi_2^a(R) -> chi[:, a] (nR x N).  The ansatz (Eq. ansatz) is
Psi(x, R) = sum_a C_a psi_a(x) chi_a(R).  Overlap matrix (Eq. M) -> S, the interaction matrices
(Eq. W, W1, W2) combine into Heff = W - W1 - W2, and the coefficient law (Eq. coeff) reads
S dC/dt = -i Heff C.

Readings of the paper used throughout (the paper leaves these to an appendix that is not part
of it):

* matrix orientation: row = bra a, column = ket b, S_ab = <phi_a|phi_b>, phi_a = psi_a chi_a;
  in W1 and W2 the pinned coordinate is the ket's.  Projecting the TDSE (Eq. TDSE) with the
  ansatz on <phi_a| while each psi_b, chi_b obeys its Hermitian-CWF equation (Eq. conditional_e /
  conditional_n with the eta terms dropped) cancels the kinetic terms and gives exactly this
  orientation: sum_b S_ab i dC_b/dt = sum_b <phi_a| V - V(x, R_b) - V(x_b, R) |phi_b> C_b.
* velocities (Eq. v1/v2): the sums run over the basis index b at the trajectory a's position,
  and carry the factor hbar/m_j (hbar = 1).
* grids: cell-centred periodic grids, x_i = x_min + (i + 1/2) dx; FFT kinetic energy.
* off-grid values (pinned potentials, CWFs and their gradients at trajectory positions): the
  4-point cubic Lagrange interpolant on the uniform grid, stencil start clamped to [0, n-4],
  derivative = exact derivative of that interpolant.
* time step n -> n+1: velocities at t_n, explicit Euler positions clamped to [first cell centre,
  last cell centre]; CWFs advanced by one Strang split-operator step with the potential pinned at
  the midpoint position; matrices assembled at t_{n+1}; RK4 for C over [t_n, t_{n+1}] with S and
  Heff linear in t between the two assemblies.
* regularisation: (S + eps I), eps absolute (S_aa = 1 for normalised CWFs, so relative to
  trace(S)/N = 1); Cholesky solves.  Default eps = 1e-6: on the Shin-Metiu test problem it gives
  the smallest population and nuclear-density errors against the exact 2D solution among
  eps in {1e-10, 1e-8, 1e-6, 1e-4}, and it bounds the sensitivity of C to rounding in S.
* initial state: CWFs are slices of Psi0 at the sampled positions (Eq. CWF1/CWF2), each
  normalised to 1; C_0 = (S_0 + eps I)^-1 b with b_a = <phi_a|Psi0> (least-squares projection).
* rank-k factorised interaction: V = v1(x) + v2(R) + V_c with v1 = row mean and v2 = column mean
  minus grand mean (exact identity); V_c = sum_k s_k u_k(x) w_k(R) by SVD, truncated where the
  Frobenius tail falls to the relative cutoff (cutoff 0 keeps every singular value).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .sampler import cell_centres, sample_positions


# --------------------------------------------------------------------------------------------
# grids and interpolation
# --------------------------------------------------------------------------------------------

def wavenumbers(n: int, d: float) -> np.ndarray:
    """FFT-ordered angular wavenumbers k_m = 2 pi m / (n d), m = 0..n/2-1, -n/2..-1."""
    m = np.arange(n)
    m = np.where(m < n // 2, m, m - n)
    return 2.0 * np.pi * m / (n * d)


def lagrange4(p: float, lo: float, d: float, n: int):
    """4-point cubic Lagrange stencil at coordinate p on the cell-centred grid (lo, d, n).

    Returns (i0, w, dw): f(p) ~ sum_m w[m] f[i0 + m] and f'(p) ~ sum_m dw[m] f[i0 + m].
    The stencil start i0 = floor(s) - 1 (s = fractional cell index) is clamped to [0, n - 4].
    Parity pinned: exact on cubic polynomials (test).
    """
    s = (p - lo) / d - 0.5
    i0 = int(np.floor(s)) - 1
    i0 = min(max(i0, 0), n - 4)
    u = s - i0                                    # local coordinate; nodes at u = 0, 1, 2, 3
    w = np.array([
        -(u - 1.0) * (u - 2.0) * (u - 3.0) / 6.0,
        u * (u - 2.0) * (u - 3.0) / 2.0,
        -u * (u - 1.0) * (u - 3.0) / 2.0,
        u * (u - 1.0) * (u - 2.0) / 6.0,
    ])
    dw = np.array([
        -((u - 2.0) * (u - 3.0) + (u - 1.0) * (u - 3.0) + (u - 1.0) * (u - 2.0)) / 6.0,
        ((u - 2.0) * (u - 3.0) + u * (u - 3.0) + u * (u - 2.0)) / 2.0,
        -((u - 1.0) * (u - 3.0) + u * (u - 3.0) + u * (u - 1.0)) / 2.0,
        ((u - 1.0) * (u - 2.0) + u * (u - 2.0) + u * (u - 1.0)) / 6.0,
    ]) / d
    return i0, w, dw


def interp(f: np.ndarray, p: float, lo: float, d: float, axis: int = 0, deriv: bool = False):
    """Value (or derivative) at coordinate p of grid samples f along `axis`."""
    n = f.shape[axis]
    i0, w, dw = lagrange4(p, lo, d, n)
    c = dw if deriv else w
    sl = np.take(f, np.arange(i0, i0 + 4), axis=axis)
    return np.tensordot(c, sl, axes=([0], [axis]))


# --------------------------------------------------------------------------------------------
# problem definition
# --------------------------------------------------------------------------------------------

@dataclass
class Params:
    """The paper's statement of the problem (Eq. TDSE with 1D x and R): grids, masses, dt, N."""
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
    svd_rel_cutoff: float = 0.0
    s_reg_eps: float = 1e-6


@dataclass
class Factors:
    """Rank-k factorisation V = v1(x) + v2(R) + sum_k s_k u_k(x) w_k(R)."""
    v1: np.ndarray
    v2: np.ndarray
    s: np.ndarray
    u: np.ndarray        # nx x k
    w: np.ndarray        # nR x k
    tail_rel: float      # Frobenius norm of the dropped part of V_c over ||V_c||_F
    next_rel: float      # first dropped singular value over the largest


def factorise(V: np.ndarray, cutoff: float) -> Factors:
    """Double-centre V and truncate the SVD of the remainder (interaction factorisation used to
    evaluate Eq. W, whose cost the paper flags for large ensembles).

    v1(x) = mean_j V(x, R_j); v2(R) = mean_i V(x_i, R) - mean_ij V; V_c = V - v1 - v2 exactly.
    Keeps the smallest k with sqrt(sum_{j >= k} s_j^2) <= cutoff * ||V_c||_F (cutoff 0: all).
    Parity pinned: the cavity V_c is rank 1; factorised Heff equals the direct double sum at
    cutoff 0 (tests).
    """
    v1 = V.mean(axis=1)
    v2 = V.mean(axis=0) - V.mean()
    Vc = V - v1[:, None] - v2[None, :]
    U, s, Wt = np.linalg.svd(Vc, full_matrices=False)
    fro = np.sqrt(np.sum(s * s))
    if cutoff <= 0.0 or fro == 0.0:
        k = len(s)
    else:
        tails = np.sqrt(np.cumsum((s * s)[::-1])[::-1])   # tails[j] = ||s_j..s_end||
        k = len(s)
        for j in range(len(s)):
            if tails[j] <= cutoff * fro:
                k = j
                break
    tail = float(np.sqrt(np.sum(s[k:] ** 2)) / fro) if fro > 0 else 0.0
    nxt = float(s[k] / s[0]) if (k < len(s) and s[0] > 0) else 0.0
    return Factors(v1, v2, s[:k].copy(), U[:, :k].copy(), Wt[:k, :].T.copy(), tail, nxt)


# --------------------------------------------------------------------------------------------
# state
# --------------------------------------------------------------------------------------------

@dataclass
class State:
    psi: np.ndarray          # nx x N complex128, column a = psi_a(x)
    chi: np.ndarray          # nR x N complex128, column a = chi_a(R)
    C: np.ndarray            # N complex128
    x: np.ndarray            # N float64
    R: np.ndarray            # N float64
    S: np.ndarray            # N x N at the current time
    Heff: np.ndarray         # N x N at the current time
    t: float = 0.0
    n_steps: int = 0
    n_clamped: int = 0
    extra: dict = field(default_factory=dict)


class Icwf:
    """The ICWF method of the paper for one electron coordinate and one nuclear/photon coordinate.

    Construct with the problem (Params) and the potential table V[i, j] = V(x_i, R_j).
    """

    def __init__(self, p: Params, V: np.ndarray, factorised: bool = True):
        self.p = p
        self.V = np.asarray(V, dtype=np.float64)
        assert self.V.shape == (p.nx, p.nR)
        self.x, self.dx = cell_centres(p.nx, p.x_min, p.x_max)
        self.R, self.dR = cell_centres(p.nR, p.R_min, p.R_max)
        self.kx = wavenumbers(p.nx, self.dx)
        self.kR = wavenumbers(p.nR, self.dR)
        self.factorised = factorised
        self.fac = factorise(self.V, p.svd_rel_cutoff)

    # ---- off-grid helpers -------------------------------------------------------------------

    def at_x(self, f, xa, deriv=False):
        return interp(f, xa, self.p.x_min, self.dx, axis=0, deriv=deriv)

    def at_R(self, f, Ra, deriv=False):
        return interp(f, Ra, self.p.R_min, self.dR, axis=0, deriv=deriv)

    def pinned_e(self, Ra: float) -> np.ndarray:
        """V(x, R_a) on the x grid: the electronic CWF's potential (Eq. conditional_e)."""
        return interp(self.V, Ra, self.p.R_min, self.dR, axis=1)

    def pinned_n(self, xa: float) -> np.ndarray:
        """V(x_a, R) on the R grid: the nuclear CWF's potential (Eq. conditional_n)."""
        return interp(self.V, xa, self.p.x_min, self.dx, axis=0)

    # ---- a2/a3: Hermitian-CWF propagation ---------------------------------------------------

    @staticmethod
    def strang(f: np.ndarray, v: np.ndarray, k: np.ndarray, mass: float, dt: float):
        """One Strang split-operator step of i df/dt = (-1/(2m) d^2/dx^2 + v) f:
        f <- e^{-i v dt/2} F^-1 e^{-i k^2 dt/(2m)} F e^{-i v dt/2} f.
        Parity pinned: free-Gaussian and harmonic coherent-state closed forms, unitarity (tests).
        """
        half = np.exp(-0.5j * dt * v)
        g = half * f
        g = np.fft.ifft(np.exp(-0.5j * dt * k * k / mass) * np.fft.fft(g))
        return half * g

    def propagate(self, st: State, xbar: np.ndarray, Rbar: np.ndarray):
        """Advance every psi_a with V(x, Rbar_a) and every chi_a with V(xbar_a, R) by dt
        (Hermitian-CWF equations: Eq. conditional_e/n with eta dropped)."""
        p = self.p
        for a in range(p.n_traj):
            st.psi[:, a] = self.strang(st.psi[:, a], self.pinned_e(Rbar[a]), self.kx,
                                       p.mass_x, p.dt)
            st.chi[:, a] = self.strang(st.chi[:, a], self.pinned_n(xbar[a]), self.kR,
                                       p.mass_R, p.dt)

    # ---- a4: Bohmian velocities -------------------------------------------------------------

    def velocities(self, st: State):
        """Eq. v1/v2: xdot_a = Im[sum_b C_b chi_b(R_a) psi_b'(x_a) / Psi(x_a, R_a)] / m_x and
        Rdot_a = Im[sum_b C_b psi_b(x_a) chi_b'(R_a) / Psi(x_a, R_a)] / m_R, with
        Psi(x_a, R_a) = sum_b C_b psi_b(x_a) chi_b(R_a).
        Parity pinned: a moving Gaussian (1/m and the sign of Im) and two boosted Gaussians with
        unequal complex C against the closed-form Im(grad Psi / Psi) / m (tests)."""
        p = self.p
        vx = np.empty(p.n_traj)
        vR = np.empty(p.n_traj)
        for a in range(p.n_traj):
            E1 = self.at_x(st.psi, st.x[a])
            G1 = self.at_x(st.psi, st.x[a], deriv=True)
            E2 = self.at_R(st.chi, st.R[a])
            G2 = self.at_R(st.chi, st.R[a], deriv=True)
            den = np.sum(st.C * E1 * E2)
            vx[a] = (np.sum(st.C * G1 * E2) / den).imag / p.mass_x
            vR[a] = (np.sum(st.C * E1 * G2) / den).imag / p.mass_R
        return vx, vR

    # ---- a5: matrix elements ----------------------------------------------------------------

    def overlaps(self, psi, chi):
        """S1 = <psi_a|psi_b>, S2 = <chi_a|chi_b>, S = S1 o S2 (Eq. M)."""
        S1 = self.dx * (psi.conj().T @ psi)
        S2 = self.dR * (chi.conj().T @ chi)
        return S1, S2, S1 * S2

    def heff_direct(self, psi, chi, x, R):
        """Heff_ab = <phi_a| V(x,R) - V(x,R_b) - V(x_b,R) |phi_b> as the literal double sum over
        the grid (Eq. W - W1 - W2, pinned at the ket b).  O(N^2 nx nR): small cases only."""
        N = psi.shape[1]
        H = np.empty((N, N), dtype=np.complex128)
        for b in range(N):
            Ve = self.pinned_e(R[b])                       # V(x_i, R_b)
            Vn = self.pinned_n(x[b])                       # V(x_b, R_j)
            D = self.V - Ve[:, None] - Vn[None, :]
            ket = np.outer(psi[:, b], chi[:, b])
            for a in range(N):
                bra = np.outer(psi[:, a], chi[:, a]).conj()
                H[a, b] = self.dx * self.dR * np.sum(bra * D * ket)
        return H

    def heff_factorised(self, psi, chi, x, R):
        """Heff from the rank-k factorisation (same quantity as heff_direct, up to truncation):

        V - V(x,R_b) - V(x_b,R) = -d_b + sum_k s_k (u_k(x) - u_k(x_b)) (w_k(R) - w_k(R_b)),
        d_b = v1(x_b) + v2(R_b) + sum_k s_k u_k(x_b) w_k(R_b), so
        Heff = sum_k s_k At_k o Bt_k - S diag(d), At_k = A_k - S1 diag(u_k(x_b)),
        Bt_k = B_k - S2 diag(w_k(R_b)), A_k = <psi_a|u_k|psi_b>, B_k = <chi_a|w_k|chi_b>.
        """
        f = self.fac
        S1, S2, S = self.overlaps(psi, chi)
        N = psi.shape[1]
        ux = np.array([self.at_x(f.u, x[b]) for b in range(N)]).reshape(N, -1)   # N x k
        wR = np.array([self.at_R(f.w, R[b]) for b in range(N)]).reshape(N, -1)
        v1x = np.array([self.at_x(f.v1, x[b]) for b in range(N)])
        v2R = np.array([self.at_R(f.v2, R[b]) for b in range(N)])
        d = v1x + v2R + (ux * wR) @ f.s
        H = -S * d[None, :]
        for k in range(len(f.s)):
            A = self.dx * (psi.conj().T @ (f.u[:, k][:, None] * psi))
            B = self.dR * (chi.conj().T @ (f.w[:, k][:, None] * chi))
            At = A - S1 * ux[:, k][None, :]
            Bt = B - S2 * wR[:, k][None, :]
            H += f.s[k] * At * Bt
        return H

    def matrices(self, psi, chi, x, R):
        S = self.overlaps(psi, chi)[2]
        if self.factorised:
            return S, self.heff_factorised(psi, chi, x, R)
        return S, self.heff_direct(psi, chi, x, R)

    def kinetic(self, f: np.ndarray, k: np.ndarray, mass: float):
        """T f = F^-1 (k^2 / 2m) F f, column by column."""
        return np.fft.ifft((k * k / (2.0 * mass))[:, None] * np.fft.fft(f, axis=0), axis=0)

    def hamiltonian(self, psi, chi):
        """H_ab = <phi_a| T_x + T_R + V |phi_b> = T1 o S2 + S1 o T2 + W (energy / reporting).
        W by the literal double sum over the grid."""
        S1, S2, _ = self.overlaps(psi, chi)
        T1 = self.dx * (psi.conj().T @ self.kinetic(psi, self.kx, self.p.mass_x))
        T2 = self.dR * (chi.conj().T @ self.kinetic(chi, self.kR, self.p.mass_R))
        W = self.dx * self.dR * np.einsum("ia,ib,ij,ja,jb->ab", psi.conj(), psi, self.V,
                                          chi.conj(), chi, optimize=True)
        return T1 * S2 + S1 * T2 + W

    # ---- a6: coefficients -------------------------------------------------------------------

    def solve(self, S, y):
        """(S + eps I)^-1 y by Cholesky (regularised overlap)."""
        A = S + self.p.s_reg_eps * np.eye(S.shape[0])
        c, low = scipy.linalg.cho_factor(A, lower=True)
        return scipy.linalg.cho_solve((c, low), y)

    def rk4(self, C, S0, H0, S1, H1):
        """Classical RK4 on dC/dt = -i (S(t) + eps I)^-1 Heff(t) C (Eq. coeff) over one dt, with
        S and Heff linear in t between their values at t_n (S0, H0) and t_{n+1} (S1, H1).
        Parity pinned: constant matrices against the matrix exponential, and matrices linear in t
        against an independent adaptive integrator, both at fourth order (tests)."""
        dt = self.p.dt
        Sh = 0.5 * (S0 + S1)
        Hh = 0.5 * (H0 + H1)
        f = lambda S, H, c: -1j * self.solve(S, H @ c)
        k1 = f(S0, H0, C)
        k2 = f(Sh, Hh, C + 0.5 * dt * k1)
        k3 = f(Sh, Hh, C + 0.5 * dt * k2)
        k4 = f(S1, H1, C + dt * k3)
        return C + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    # ---- initialisation ---------------------------------------------------------------------

    def init_from_positions(self, psi0: np.ndarray, x: np.ndarray, R: np.ndarray) -> State:
        """CWFs as slices of Psi0 at (x_a, R_a) (Eq. CWF1/CWF2), each normalised to 1, and C_0 by
        least-squares projection of Psi0 on the product basis."""
        p = self.p
        N = p.n_traj
        psi0 = np.asarray(psi0, dtype=np.complex128)
        psi = np.empty((p.nx, N), dtype=np.complex128)
        chi = np.empty((p.nR, N), dtype=np.complex128)
        for a in range(N):
            psi[:, a] = interp(psi0, R[a], p.R_min, self.dR, axis=1)
            chi[:, a] = interp(psi0, x[a], p.x_min, self.dx, axis=0)
            psi[:, a] /= np.sqrt(self.dx * np.sum(np.abs(psi[:, a]) ** 2))
            chi[:, a] /= np.sqrt(self.dR * np.sum(np.abs(chi[:, a]) ** 2))
        b = self.dx * self.dR * np.einsum("ia,ja,ij->a", psi.conj(), chi.conj(), psi0)
        S, H = self.matrices(psi, chi, x, R)
        C = self.solve(S, b)
        return State(psi=psi, chi=chi, C=C, x=np.array(x, dtype=np.float64),
                     R=np.array(R, dtype=np.float64), S=S, Heff=H)

    def init_from_density(self, psi0: np.ndarray, seed: int) -> State:
        p = self.p
        x, R = sample_positions(psi0, p.n_traj, seed, p.x_min, p.x_max, p.R_min, p.R_max)
        return self.init_from_positions(psi0, x, R)

    # ---- one step ---------------------------------------------------------------------------

    def step(self, st: State, freeze_coefficients: bool = False,
             freeze_matrices: bool = False) -> State:
        """t_n -> t_{n+1}: velocities (Eq. v1/v2) -> Euler positions -> Hermitian-CWF propagation
        pinned at the midpoints -> matrices at t_{n+1} (Eq. Matrices) -> RK4 on C (Eq. coeff).
        `freeze_coefficients` keeps C fixed (the plain Hermitian-CWF scheme).  `freeze_matrices`
        holds S and Heff at their t_n values over the step (one factorisation per step)."""
        p = self.p
        vx, vR = self.velocities(st)
        xlo, xhi = self.x[0], self.x[-1]
        Rlo, Rhi = self.R[0], self.R[-1]
        xn = st.x + p.dt * vx
        Rn = st.R + p.dt * vR
        n_cl = int(np.sum((xn < xlo) | (xn > xhi)) + np.sum((Rn < Rlo) | (Rn > Rhi)))
        xn = np.clip(xn, xlo, xhi)
        Rn = np.clip(Rn, Rlo, Rhi)
        xbar = 0.5 * (st.x + xn)
        Rbar = 0.5 * (st.R + Rn)
        self.propagate(st, xbar, Rbar)
        S1, H1 = self.matrices(st.psi, st.chi, xn, Rn)
        if freeze_matrices:
            st.C = self.rk4(st.C, st.S, st.Heff, st.S, st.Heff)
        elif not freeze_coefficients:
            st.C = self.rk4(st.C, st.S, st.Heff, S1, H1)
        st.S, st.Heff = S1, H1
        st.x, st.R = xn, Rn
        st.t += p.dt
        st.n_steps += 1
        st.n_clamped += n_cl
        return st

    # ---- a7: observables --------------------------------------------------------------------

    def wavefunction(self, st: State) -> np.ndarray:
        """Eq. ansatz on the grid: Psi[i, j] = sum_a C_a psi_a(x_i) chi_a(R_j)."""
        return (st.psi * st.C[None, :]) @ st.chi.T

    def observables(self, st: State, phi: np.ndarray | None = None) -> dict:
        return grid_observables(self.wavefunction(st), self.V, self.dx, self.dR, self.kx,
                                self.kR, self.p.mass_x, self.p.mass_R, phi)


def grid_observables(Psi, V, dx, dR, kx, kR, mass_x, mass_R, phi=None) -> dict:
    """Observables of a wavefunction tabulated on the (x, R) grid.

    rho_x(x) = int dR |Psi|^2, rho_R(R) = int dx |Psi|^2 (reduced densities), norm = <Psi|Psi>,
    energy = <Psi|T_x + T_R + V|Psi> / <Psi|Psi> (kinetic parts by Parseval on the FFT),
    chi^(n)(R) = int dx phi_n(x; R) Psi(x, R) for real BO states phi (n_s x nR x nx),
    P_n = int dR |chi^(n)|^2 (BO populations), D_nm = int dR |chi^(n)|^2 |chi^(m)|^2 (decoherence
    indicator defined in the paper's discussion of the Shin-Metiu results).
    Parity pinned: norm and energy against the matrix forms C^H S C and C^H H C; populations,
    D_nm and rho_R against the closed forms of g(R) phi_1 and of a two-state superposition a(R)
    phi_0 + b(R) phi_2 (BO states orthonormal at every R) (tests).
    """
    nx, nR = Psi.shape
    dens = Psi.real ** 2 + Psi.imag ** 2
    out = {
        "rho_x": dR * dens.sum(axis=1),
        "rho_R": dx * dens.sum(axis=0),
        "norm": dx * dR * dens.sum(),
    }
    Fx = np.fft.fft(Psi, axis=0)
    FR = np.fft.fft(Psi, axis=1)
    ekx = dR * (dx / nx) * np.sum((np.abs(Fx) ** 2) * (kx * kx / (2.0 * mass_x))[:, None])
    ekR = dx * (dR / nR) * np.sum((np.abs(FR) ** 2) * (kR * kR / (2.0 * mass_R))[None, :])
    epot = dx * dR * np.sum(dens * V)
    out["energy"] = (ekx + ekR + epot) / out["norm"]
    if phi is not None:
        chin = dx * np.einsum("nji,ij->nj", phi, Psi)        # n_s x nR
        pn = np.abs(chin) ** 2
        out["pop"] = dR * pn.sum(axis=1)
        out["decoherence"] = dR * np.einsum("nj,mj->nm", pn, pn)
    return out
