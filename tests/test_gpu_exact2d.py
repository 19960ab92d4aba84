"""Exact 2D propagation on the GPU (include/icwf_exact2d.h) against the FP64 oracle's Strang
solver (oracle/exact2d.py, numpy fft2): the same arithmetic in a different order, so the state
and the observables agree to rounding.  Also: norm conservation at the bench grid."""
import numpy as np
import pytest

from oracle.exact2d import Exact2D as OracleExact2D
from workloads import cavity, shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def _oracle(w):
    return OracleExact2D(w.nx, w.nR, w.x_min, w.x_max, w.R_min, w.R_max, w.mass_x, w.mass_R, w.dt,
                         w.V)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("name", ["shin_metiu", "cavity"])
def test_state_and_observables_match_the_oracle(name):
    if name == "shin_metiu":
        w = shin_metiu()                                 # 128 x 64, dt = 0.1
        steps = 50
    else:
        w = cavity(nx=256, x_range=(-40.0, 40.0), nq=64, q_range=(-15.0, 15.0), n_traj=8,
                   lam=0.5, dt=0.05)
        steps = 40
    o = _oracle(w)
    ref = o.run(w.psi0, steps)
    oo = o.observables(ref, w.phi)
    e = g.Exact2D(g.params_from(w), w.V)
    e.set_projectors(w.phi)
    e.set_state(w.psi0)
    for _ in range(2):                                  # two calls: the state carries over
        e.step(steps // 2)
    psi = e.state()
    assert _rel(psi, ref) < 1e-11
    ob = e.observables()
    assert abs(ob["t"] - steps * w.dt) < 1e-12
    assert abs(ob["norm"] - oo["norm"]) < 1e-12
    assert abs(ob["energy"] - oo["energy"]) < 1e-10 * max(1.0, abs(oo["energy"]))
    assert _rel(ob["rho_x"], oo["rho_x"]) < 1e-10
    assert _rel(ob["rho_R"], oo["rho_R"]) < 1e-10
    assert np.max(np.abs(ob["pop"] - oo["pop"])) < 1e-11
    assert np.max(np.abs(ob["decoherence"] - oo["decoherence"])) < 1e-11
    e.close()


def test_bench_grid_parity_and_norm():
    """Shin-Metiu at the paper's scale (1024 x 512, dt = 0.05): 20 steps against the oracle, then
    the norm after 200 more (the split is unitary) and the energy (conserved up to the splitting
    error, which stays bounded)."""
    from workloads.models import WORKLOADS
    w = WORKLOADS["sm_paper"](n_traj=8)
    o = _oracle(w)
    ref = o.run(w.psi0, 20)
    e = g.Exact2D(g.params_from(w), w.V)
    e.set_state(w.psi0)
    ob0 = e.observables()
    e.step(20)
    assert _rel(e.state(), ref) < 1e-11
    e.step(200)
    ob = e.observables()
    assert abs(ob["norm"] - ob0["norm"]) < 1e-11
    assert abs(ob["energy"] - ob0["energy"]) < 1e-4 * abs(ob0["energy"])
    e.close()


def test_call_order_and_sizes():
    w = shin_metiu()
    e = g.Exact2D(g.params_from(w), w.V)
    with pytest.raises(g.IcwfError) as ex:
        e.step(1)
    assert ex.value.status == g.ICWF_ERR_STATE
    with pytest.raises(g.IcwfError) as ex:
        e.set_projectors(np.zeros((9, w.nR, w.nx)))
    assert ex.value.status == g.ICWF_ERR_ARG
    e.close()


def test_handles_of_different_sizes_coexist():
    """A small handle created after a large one must not break the large one's launches."""
    from workloads.models import WORKLOADS
    big = WORKLOADS["sm_paper"](n_traj=8)
    small = shin_metiu()
    eb = g.Exact2D(g.params_from(big), big.V)
    eb.set_state(big.psi0)
    es = g.Exact2D(g.params_from(small), small.V)
    es.set_state(small.psi0)
    eb.step(2)
    es.step(2)
    ref = _oracle(big).run(big.psi0, 2)
    assert _rel(eb.state(), ref) < 1e-11
    eb.close()
    es.close()

