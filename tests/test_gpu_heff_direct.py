"""icwf_heff_direct: Heff columns by the full double sum over the grid (no rank-k factorisation),
the reference for the factorised assembly's error report.

Checked against the oracle's literal double sum (heff_direct) on the GPU's own CWFs and positions
to 1e-12 relative, for FP64 and complex64 storage, with ragged grid and trajectory tiles; and the
factorised Heff of the step differs from it by the truncation level of the kept rank.
"""
import numpy as np
import pytest

from oracle.icwf import Icwf as Oracle, Params
from workloads import shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def oracle_for(w):
    return Oracle(Params(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
                         w.n_traj, w.svd_rel_cutoff, w.s_reg_eps), w.V)


@pytest.mark.parametrize("precision,N,nx,nR", [(0, 16, 128, 64), (2, 37, 64, 64), (0, 70, 16, 8),
                                               (1, 5, 256, 64)])
def test_direct_columns_match_the_oracle_double_sum(precision, N, nx, nR):
    w = shin_metiu(nx=nx, x_range=(-30.0, 30.0), nR=nR, R_range=(-7.0, 7.0), n_traj=N, dt=0.1,
                   svd_rel_cutoff=1e-4, s_reg_eps=1e-6 if precision == 0 else 1e-4)
    sim = g.Icwf(g.params_from(w, precision=precision), w.V)
    sim.init_from_density(w.psi0, 2)
    sim.step(2)
    st = sim.state()
    cols = np.array(sorted({0, N // 2, N - 1}), dtype=np.int32)
    Hd = sim.heff_direct(cols)
    o = oracle_for(w)
    Ho = o.heff_direct(st["psi"], st["chi"], st["x"], st["R"])[:, cols]
    assert np.linalg.norm(Hd - Ho) < 1e-12 * np.linalg.norm(Ho)
    # the factorised Heff of the step carries the truncation of the kept rank (cutoff 1e-4);
    # a grid whose dropped singular values vanish (double-centring leaves V_c rank-deficient)
    # is factorised exactly
    Hf = sim.matrices()["Heff"][:, cols]
    err = np.linalg.norm(Hf - Hd) / np.linalg.norm(Hd)
    if sim.info()["tail_rel"] > 1e-8:       # something of size was dropped
        assert 1e-9 < err < 1e-2, err
    else:
        assert err < (1e-12 if precision == 0 else 1e-5), err
    sim.close()


def test_full_rank_factorisation_equals_the_direct_sum():
    """At cutoff 0 (every singular value kept) the factorised FP64 assembly equals the direct sum
    to rounding."""
    w = shin_metiu(n_traj=16, svd_rel_cutoff=0.0)
    sim = g.Icwf(g.params_from(w), w.V)
    sim.init_from_density(w.psi0, 0)
    sim.step(3)
    cols = np.arange(16, dtype=np.int32)
    Hd = sim.heff_direct(cols)
    Hf = sim.matrices()["Heff"]
    assert np.linalg.norm(Hf - Hd) < 1e-11 * np.linalg.norm(Hd)
    with pytest.raises(g.IcwfError) as e:
        sim.heff_direct(np.array([16], dtype=np.int32))
    assert e.value.status == g.ICWF_ERR_ARG
    sim.close()
