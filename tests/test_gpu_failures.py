"""Failure detection through the C ABI, in forms that fault, trap or hang no GPU.

* ICWF_ERR_NUMERIC: the host makes S + eps I indefinite by setting a negative eps
  (icwf_set_regularisation); the next step's Cholesky meets a pivot <= 0, the kernel raises the
  status flag and the call returns the status (FP64 and mixed solvers).
* ICWF_ERR_TIMEOUT: a zero poll budget for the spin waits on global flags
  (icwf_set_wait_limit(0)) makes every such wait give up at once; the kernels set the timeout flag
  and finish without their inputs, the call returns the status, and the GPU context stays usable
  (a fresh handle afterwards gives the same results as before).
* A pool job that fails mid-stream (its eps turned negative after two steps) ends in state 3
  while the other jobs of the mix finish with the same results as when they run alone.
"""
import numpy as np
import pytest

from workloads import shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def _sm(N, **kw):
    d = dict(nx=128, x_range=(-50.0, 50.0), nR=64, R_range=(-9.0, 9.0), n_traj=N, dt=0.1,
             svd_rel_cutoff=1e-8)
    d.update(kw)
    return shin_metiu(**d)


def _make(w, precision=0, seed=0):
    sim = g.Icwf(g.params_from(w, precision=precision), w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, seed)
    return sim


def _same(a, b, tol=1e-12):
    assert abs(a["norm"] - b["norm"]) < tol
    assert np.max(np.abs(a["rho_x"] - b["rho_x"])) < tol
    assert np.max(np.abs(a["rho_R"] - b["rho_R"])) < tol
    assert np.max(np.abs(a["pop"] - b["pop"])) < tol


def _reference_run():
    sim = _make(_sm(24), 0, 5)
    sim.step(3)
    out = sim.observables()
    sim.close()
    return out


@pytest.mark.parametrize("precision,N", [(0, 40), (2, 300), (1, 64)])
def test_indefinite_overlap_returns_numeric(precision, N):
    w = _sm(N, s_reg_eps=1e-6 if precision == 0 else 1e-4)
    sim = _make(w, precision)
    sim.step(1)
    sim.set_regularisation(-0.5)          # S - 0.5 I: S has eigenvalues near 0 and near N
    with pytest.raises(g.IcwfError) as e:
        sim.step(1)
    assert e.value.status == g.ICWF_ERR_NUMERIC
    assert "Cholesky" in str(e.value)
    sim.close()
    with pytest.raises(g.IcwfError) as e:
        sim2 = _make(w, precision)
        sim2.set_regularisation(float("nan"))
    assert e.value.status == g.ICWF_ERR_ARG
    sim2.close()


@pytest.mark.parametrize("precision,N", [(0, 100), (2, 300)])
def test_exhausted_wait_returns_timeout_and_context_survives(precision, N):
    before = _reference_run()
    w = _sm(N, s_reg_eps=1e-6 if precision == 0 else 1e-4)
    sim = _make(w, precision)
    sim.step(1)
    sim.set_wait_limit(0)
    with pytest.raises(g.IcwfError) as e:
        sim.step(1)
    assert e.value.status == g.ICWF_ERR_TIMEOUT
    assert "timed out" in str(e.value)
    sim.close()
    # a handle whose budget is restored runs normally
    sim = _make(w, precision)
    sim.set_wait_limit(0)
    sim.set_wait_limit(-1)
    sim.step(2)
    sim.close()
    _same(_reference_run(), before)


def test_pool_job_failing_mid_stream_leaves_the_others_unchanged():
    specs = [(_sm(16), 0, 0, 8), (_sm(40, R0=-4.5), 0, 1, 8), (_sm(96, s_reg_eps=1e-4), 2, 2, 6)]
    alone = []
    for w, prec, seed, n in specs:
        sim = _make(w, prec, seed)
        sim.step(n)
        alone.append(sim.observables())
        sim.close()
    pool = g.icwf_pool_create(1 << 34, 3)
    sims = [_make(w, prec, seed) for w, prec, seed, _ in specs]
    ids = [g.icwf_pool_submit(pool, s.h, n) for s, (_, _, _, n) in zip(sims, specs)]
    for _ in range(2):
        g.icwf_pool_tick(pool)
    # the middle job's overlap turns indefinite from its third step on
    sims[1].set_regularisation(-0.5)
    for s in sims:
        s.release()
    states = None
    for _ in range(50):
        g.icwf_pool_tick(pool)
        states = [g.icwf_pool_poll(pool, i, w.nx, w.nR)[0] for i, (w, *_r) in zip(ids, specs)]
        if all(st in (2, 3) for st in states):
            break
    assert states == [2, 3, 2], states
    for k in (0, 2):
        st, obs = g.icwf_pool_poll(pool, ids[k], specs[k][0].nx, specs[k][0].nR)
        assert st == 2
        _same(obs, alone[k])
    g.icwf_pool_destroy(pool)
