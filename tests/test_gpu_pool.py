"""Serving pool (icwf_pool_*): continuous batching of independent ICWF jobs of different sizes.

Jobs arrive while others run, are admitted in arrival order as slots and the device-memory budget
allow, and advance one step per tick together (each job on its own stream, so their kernels
overlap on the device).  Every job's result must be the same alone and in the mix: the jobs share
no state, and each job's kernels are deterministic, so the comparison is to rounding (1e-12).
"""
import numpy as np
import pytest

from workloads import cavity, shin_metiu

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1805_11169_gb300")


def _jobs():
    """Mixed sizes and both models, FP64 and mixed precision."""
    sm_a = shin_metiu(nx=128, x_range=(-50.0, 50.0), nR=64, R_range=(-9.0, 9.0), n_traj=16,
                      dt=0.1, svd_rel_cutoff=1e-8)
    sm_b = shin_metiu(nx=256, x_range=(-60.0, 60.0), nR=128, R_range=(-9.0, 9.0), n_traj=96,
                      dt=0.05, R0=-3.5, Rf=4.5, svd_rel_cutoff=1e-8, s_reg_eps=1e-4)
    cav = cavity(nx=256, x_range=(-40.0, 40.0), nq=64, q_range=(-15.0, 15.0), n_traj=48,
                 lam=0.3, dt=0.05, svd_rel_cutoff=1e-8)
    sm_c = shin_metiu(nx=128, x_range=(-50.0, 50.0), nR=64, R_range=(-9.0, 9.0), n_traj=40,
                      dt=0.1, R0=-4.5, svd_rel_cutoff=1e-8)
    # (workload, precision, seed, steps)
    return [(sm_a, 0, 0, 12), (sm_b, 2, 1, 9), (cav, 0, 2, 15), (sm_c, 0, 3, 6),
            (sm_a.with_(s_reg_eps=1e-4), 2, 4, 10)]


def _make(w, precision, seed):
    sim = g.Icwf(g.params_from(w, precision=precision), w.V)
    sim.set_projectors(w.phi)
    sim.init_from_density(w.psi0, seed)
    return sim


def _same(a, b):
    assert abs(a["norm"] - b["norm"]) < 1e-12
    assert abs(a["energy"] - b["energy"]) < 1e-12
    assert np.max(np.abs(a["rho_x"] - b["rho_x"])) < 1e-12
    assert np.max(np.abs(a["rho_R"] - b["rho_R"])) < 1e-12
    assert np.max(np.abs(a["pop"] - b["pop"])) < 1e-12
    assert abs(a["t"] - b["t"]) < 1e-12


def _group_nodes(jobs):
    """Grouped kernels a graph-ticked run of `jobs` (all admitted at the first tick) executes:
    at tick t, two for each CWF precision (FP64 or complex64) among the jobs still stepping."""
    total = 0
    for t in range(1, max(n for *_r, n in jobs) + 1):
        total += 2 * len({prec == 0 for _w, prec, _s, n in jobs if n >= t})
    return total


def _run_pool(jobs, max_live, graphs=True, grouping=None):
    pool = g.icwf_pool_create(1 << 34, max_live)
    g.icwf_pool_set_graphs(pool, graphs)
    if grouping is not None:
        g.icwf_pool_set_grouping(pool, *grouping)
    ids = [g.icwf_pool_submit(pool, _make(w, prec, seed).release(), n) for w, prec, seed, n in jobs]
    for _ in range(200):
        live, _ = g.icwf_pool_tick(pool)
        if live == 0 and all(g.icwf_pool_poll(pool, i, w.nx, w.nR)[0] == 2
                             for i, (w, *_r) in zip(ids, jobs)):
            break
    out = [g.icwf_pool_poll(pool, i, w.nx, w.nR) for i, (w, *_r) in zip(ids, jobs)]
    st = g.icwf_pool_get_stats(pool)
    g.icwf_pool_destroy(pool)
    assert all(s == 2 for s, _o in out), [s for s, _o in out]
    return [o for _s, o in out], st


def test_grouped_kernels_loop_over_all_jobs():
    """The grouped velocity and propagation kernels stride over the work items of every live job:
    capped at 3 CTAs each (every CTA then handles CWFs and trajectories of several jobs, with
    ragged N and grids), with no cap, and with grouping off, the results equal direct launches."""
    jobs = _jobs()
    ref, st = _run_pool(jobs, 5, graphs=False)
    assert st["group_nodes"] == 0
    for grouping in ((True, 3), (True, 0), (False, 0)):
        res, st = _run_pool(jobs, 5, graphs=True, grouping=grouping)
        assert st["eager_job_steps"] == 0
        assert st["group_nodes"] == (_group_nodes(jobs) if grouping[0] else 0)
        for a, b in zip(res, ref):
            _same(a, b)


def test_each_job_is_the_same_alone_and_in_the_mix():
    jobs = _jobs()
    alone = []
    for w, prec, seed, n in jobs:
        sim = _make(w, prec, seed)
        sim.step(n)
        alone.append(sim.observables())
        sim.close()

    pool = g.icwf_pool_create(1 << 34, 3)          # at most 3 live jobs
    ids = []
    # staggered arrivals: two jobs, a few ticks, then the rest while those still run
    for k, (w, prec, seed, n) in enumerate(jobs):
        sim = _make(w, prec, seed)
        ids.append(g.icwf_pool_submit(pool, sim.release(), n))
        if k == 1:
            for _ in range(4):
                live, _ = g.icwf_pool_tick(pool)
                assert live <= 3
    states = None
    for _ in range(200):
        live, _ = g.icwf_pool_tick(pool)
        assert live <= 3
        states = [g.icwf_pool_poll(pool, i, w.nx, w.nR)[0] for i, (w, *_r) in zip(ids, jobs)]
        if all(s == 2 for s in states):
            break
    assert states is not None and all(s == 2 for s in states), states
    for i, (w, *_r), ref in zip(ids, jobs, alone):
        st, obs = g.icwf_pool_poll(pool, i, w.nx, w.nR)
        assert st == 2
        _same(obs, ref)
    g.icwf_pool_destroy(pool)


def test_admission_by_device_memory_budget():
    """A budget that fits one job at a time serialises the jobs (arrival order kept)."""
    w = shin_metiu(nx=128, x_range=(-50.0, 50.0), nR=64, R_range=(-9.0, 9.0), n_traj=32,
                   dt=0.1, svd_rel_cutoff=1e-8)
    sims = [_make(w, 0, s) for s in range(3)]
    need = sims[0].info()["device_bytes"]
    pool = g.icwf_pool_create(int(need * 1.5), 8)
    ids = [g.icwf_pool_submit(pool, s.release(), 3) for s in sims]
    order = []
    for _ in range(50):
        live, fin = g.icwf_pool_tick(pool)
        assert live <= 1
        for i in ids:
            st, _ = g.icwf_pool_poll(pool, i, w.nx, w.nR)
            if st == 2 and i not in order:
                order.append(i)
        if len(order) == 3:
            break
    assert order == ids
    # a job larger than the whole budget is refused at submission
    big = _make(w.with_(n_traj=64), 0, 9)
    small_pool = g.icwf_pool_create(1024, 2)
    with pytest.raises(g.IcwfError) as e:
        g.icwf_pool_submit(small_pool, big.h, 1)
    assert e.value.status == g.ICWF_ERR_OOM
    big.close()
    g.icwf_pool_destroy(small_pool)
    g.icwf_pool_destroy(pool)


def test_graph_ticks_equal_eager_ticks_and_launch_once_per_tick():
    """The same mixed stream with captured tick graphs and with direct launches gives the same
    results to rounding; with graphs every tick that steps jobs is one graph launch (no job step
    launched directly), whatever the number of live jobs."""
    jobs = _jobs()[:4]
    results = {}
    for graphs in (True, False):
        pool = g.icwf_pool_create(1 << 34, 4)
        g.icwf_pool_set_graphs(pool, graphs)
        ids = [g.icwf_pool_submit(pool, _make(w, prec, seed).release(), n)
               for w, prec, seed, n in jobs]
        for _ in range(100):
            live, _ = g.icwf_pool_tick(pool)
            if live == 0 and all(g.icwf_pool_poll(pool, i, w.nx, w.nR)[0] == 2
                                 for i, (w, *_r) in zip(ids, jobs)):
                break
        results[graphs] = [g.icwf_pool_poll(pool, i, w.nx, w.nR)[1] for i, (w, *_r) in zip(ids, jobs)]
        st = g.icwf_pool_get_stats(pool)
        if graphs:
            assert st["eager_job_steps"] == 0
            assert st["graph_job_steps"] == sum(n for *_r, n in jobs)
            stepping_ticks = max(n for *_r, n in jobs)
            assert st["graph_launches"] == stepping_ticks
            assert st["kernel_nodes"] > 10 * st["graph_job_steps"]
            assert st["graph_builds"] <= 2 * len(jobs)
            # two grouped kernels (velocities, propagation) per CWF precision live in the tick,
            # however many jobs of that precision there are
            assert st["group_nodes"] == _group_nodes(jobs)
        else:
            assert st["graph_launches"] == 0 and st["eager_job_steps"] == sum(n for *_r, n in jobs)
            assert st["group_nodes"] == 0
        g.icwf_pool_destroy(pool)
    for a, b in zip(results[True], results[False]):
        _same(a, b)
