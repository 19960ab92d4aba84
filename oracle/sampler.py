"""Seeded sampling of the initial trajectory positions from |Psi0|^2 (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper samples the trajectories stochastically from the initial density (Eq. ansatz and the
text after it; the sentence on ensembles that explore the support of |Psi|^2 before it) but does
not say how.  Reading used here, implemented independently in the CUDA library's host code:

* generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the state advances by the golden-gamma constant and each output is
  the new state through Stafford's variant-13 finaliser (xorshift 30, multiply, xorshift 27,
  multiply, xorshift 31);
* uniform double in [0, 1): the top 53 bits of one output times 2^-53;
* per trajectory, in this order: the grid cell (i, j) by inverse CDF over p_ij = |Psi0_ij|^2
  flattened row-major (i over x, j over R; first index whose running sum exceeds u * total),
  then an x jitter x_i + (u' - 1/2) dx, then an R jitter R_j + (u'' - 1/2) dR.

Pinned by: the published first outputs of SplitMix64 for seed 0, a chi-square test of the
sampled cells against |Psi0|^2, and bitwise equality with the library's sampler (GPU test).
"""
import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


class SplitMix64:
    """SplitMix64 as published (state += gamma; xor-shift-multiply mixing of the new state)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Top 53 bits scaled to [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def cell_centres(n: int, lo: float, hi: float):
    """x_i = lo + (i + 1/2) dx with dx = (hi - lo) / n (cell-centred periodic grid)."""
    d = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * d, d


def sample_positions(psi0: np.ndarray, n_traj: int, seed: int,
                     x_lo: float, x_hi: float, R_lo: float, R_hi: float):
    """Draw n_traj positions (x_a, R_a) from |psi0|^2 on the (x, R) grid.

    psi0: (nx, nR) complex128, psi0[i, j] = Psi0(x_i, R_j).
    Returns float64 arrays x (n_traj,), R (n_traj,).
    """
    nx, nR = psi0.shape
    x, dx = cell_centres(nx, x_lo, x_hi)
    R, dR = cell_centres(nR, R_lo, R_hi)
    re = psi0.real.ravel()
    im = psi0.imag.ravel()
    p = re * re + im * im                 # |Psi0|^2, one rounding per product and one per sum
    cum = np.add.accumulate(p)            # sequential running sum, left to right
    total = cum[-1]
    rng = SplitMix64(seed)
    xs = np.empty(n_traj)
    Rs = np.empty(n_traj)
    for a in range(n_traj):
        target = rng.uniform() * total
        idx = int(np.searchsorted(cum, target, side="right"))   # first cum[idx] > target
        idx = min(idx, nx * nR - 1)
        i, j = divmod(idx, nR)
        xs[a] = x[i] + (rng.uniform() - 0.5) * dx
        Rs[a] = R[j] + (rng.uniform() - 0.5) * dR
    return xs, Rs
