"""Checkpoint / resume through the C ABI (icwf_state_bytes, icwf_save_state, icwf_load_state).

A handle saved after some steps and restored into a fresh handle with the same parameters must
continue bit for bit like the original: the saved state holds everything the next step reads
(CWFs, positions, C, S, Heff and the Cholesky factor at the current time, the counters).
Mismatched parameters and foreign buffers are rejected with ICWF_ERR_ARG.
"""
import numpy as np
import pytest

from workloads import shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def _w(N):
    return shin_metiu(n_traj=N, svd_rel_cutoff=1e-8, s_reg_eps=1e-6)


@pytest.mark.parametrize("precision,coeff_scheme", [(0, 0), (2, 0), (1, 1)])
def test_restored_handle_continues_bit_for_bit(precision, coeff_scheme):
    w = _w(40)
    a = g.Icwf(g.params_from(w, precision=precision, coeff_scheme=coeff_scheme), w.V)
    a.set_projectors(w.phi)
    a.init_from_density(w.psi0, 3)
    a.step(5)
    blob = a.save_state()
    a.step(7)
    sa, oa = a.state(), a.observables()
    b = g.Icwf(g.params_from(w, precision=precision, coeff_scheme=coeff_scheme), w.V)
    b.set_projectors(w.phi)
    b.load_state(blob)
    assert b.info()["steps_done"] == 5
    b.step(7)
    sb, ob = b.state(), b.observables()
    for k in ("C", "x", "R", "psi", "chi"):
        assert np.array_equal(sa[k], sb[k]), k
    for k in ("rho_x", "rho_R", "pop"):
        assert np.array_equal(oa[k], ob[k]), k
    assert oa["t"] == ob["t"] and oa["n_clamped"] == ob["n_clamped"]
    a.close()
    b.close()


def test_mismatched_state_is_rejected():
    w = _w(16)
    a = g.Icwf(g.params_from(w, precision=2), w.V)
    with pytest.raises(g.IcwfError) as e:
        a.save_state()
    assert e.value.status == g.ICWF_ERR_STATE
    a.init_from_density(w.psi0, 0)
    blob = a.save_state()
    other = g.Icwf(g.params_from(w.with_(n_traj=17), precision=2), w.V)
    with pytest.raises(g.IcwfError) as e:
        other.load_state(blob)
    assert e.value.status == g.ICWF_ERR_ARG
    with pytest.raises(g.IcwfError) as e:
        a.load_state(b"not a state" * 10)
    assert e.value.status == g.ICWF_ERR_ARG
    with pytest.raises(g.IcwfError) as e:
        a.load_state(blob[: len(blob) // 2])
    assert e.value.status == g.ICWF_ERR_ARG
    a.close()
    other.close()
