"""ctypes binding of the C ABI in include/icwf.h (argument marshalling only).

Every call goes straight to ``libicwf.so``; there is no Python or CPU implementation of any step
behind these functions.  A missing or unloadable library raises at import time.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libicwf.so")

ICWF_OK, ICWF_ERR_ARG, ICWF_ERR_STATE, ICWF_ERR_OOM, ICWF_ERR_CUDA, ICWF_ERR_NUMERIC, \
    ICWF_ERR_TIMEOUT = range(7)
ICWF_FP64, ICWF_MIXED_BF16X3, ICWF_MIXED_TF32X3 = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_OOM", 4: "ERR_CUDA",
                5: "ERR_NUMERIC", 6: "ERR_TIMEOUT"}


class IcwfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class icwf_params(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("nR", ct.c_int32),
                ("x_min", ct.c_double), ("x_max", ct.c_double),
                ("R_min", ct.c_double), ("R_max", ct.c_double),
                ("mass_x", ct.c_double), ("mass_R", ct.c_double),
                ("dt", ct.c_double), ("n_traj", ct.c_int32), ("precision", ct.c_int32),
                ("svd_rel_cutoff", ct.c_double), ("s_reg_eps", ct.c_double),
                ("coeff_scheme", ct.c_int32), ("max_rank", ct.c_int32),
                ("solve_fp64", ct.c_int32), ("overlap_split", ct.c_int32)]


class icwf_info(ct.Structure):
    _fields_ = [("rank", ct.c_int32), ("tail_rel", ct.c_double), ("next_rel", ct.c_double),
                ("sigma_max", ct.c_double), ("device_bytes", ct.c_size_t),
                ("steps_done", ct.c_int64), ("t", ct.c_double),
                ("kernel_launches", ct.c_int64), ("obs_bytes", ct.c_size_t),
                ("prop_threads", ct.c_int32)]


class icwf_pool_stats(ct.Structure):
    _fields_ = [("ticks", ct.c_int64), ("graph_launches", ct.c_int64),
                ("graph_builds", ct.c_int64), ("kernel_nodes", ct.c_int64),
                ("graph_job_steps", ct.c_int64), ("eager_job_steps", ct.c_int64),
                ("group_nodes", ct.c_int64)]


class icwf_obs(ct.Structure):
    _fields_ = [("t", ct.c_double), ("norm", ct.c_double), ("energy", ct.c_double),
                ("rho_x", ct.POINTER(ct.c_double)), ("rho_R", ct.POINTER(ct.c_double)),
                ("pop", ct.POINTER(ct.c_double)), ("decoh", ct.POINTER(ct.c_double)),
                ("n_states", ct.c_int32), ("n_clamped", ct.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (the CUDA library "
                          "is the only implementation)")
    lib = ct.CDLL(LIB_PATH)
    H = ct.c_void_p
    P = ct.POINTER
    d = P(ct.c_double)
    sig = {
        "icwf_create": [P(icwf_params), d, P(H)],
        "icwf_set_projectors": [H, ct.c_int32, d],
        "icwf_init_from_density": [H, d, ct.c_uint64],
        "icwf_init_from_positions": [H, d, d, d],
        "icwf_step": [H, ct.c_int32],
        "icwf_observables": [H, P(icwf_obs)],
        "icwf_observables_static": [H, P(icwf_obs)],
        "icwf_destroy": [H],
        "icwf_get_state": [H, d, d, d, d, d],
        "icwf_get_matrices": [H, d, d, d],
        "icwf_get_info": [H, P(icwf_info)],
        "icwf_heff_direct": [H, ct.c_int32, P(ct.c_int32), d],
        "icwf_state_bytes": [H, P(ct.c_size_t)],
        "icwf_save_state": [H, ct.c_void_p, ct.c_size_t],
        "icwf_load_state": [H, ct.c_void_p, ct.c_size_t],
        "icwf_get_stream": [H, P(ct.c_void_p)],
        "icwf_set_regularisation": [H, ct.c_double],
        "icwf_set_wait_limit": [H, ct.c_int64],
        "icwf_set_step_graphs": [H, ct.c_int32],
        "icwf_set_emulated_update": [H, ct.c_int32],
        "icwf_profile_enable": [H, ct.c_int32],
        "icwf_profile_reset": [H],
        "icwf_profile_read": [H, ct.c_int32, P(ct.c_char_p), d, P(ct.c_int64), P(ct.c_int32)],
        "icwf_pool_create": [ct.c_size_t, ct.c_int32, P(H)],
        "icwf_pool_submit": [H, H, ct.c_int64, P(ct.c_int32)],
        "icwf_pool_tick": [H, P(ct.c_int32), P(ct.c_int32)],
        "icwf_pool_poll": [H, ct.c_int32, P(icwf_obs), P(ct.c_int32)],
        "icwf_pool_destroy": [H],
        "icwf_pool_get_stats": [H, P(icwf_pool_stats)],
        "icwf_pool_set_graphs": [H, ct.c_int32],
        "icwf_pool_set_grouping": [H, ct.c_int32, ct.c_int32],
        "icwf_exact2d_create": [P(icwf_params), d, P(H)],
        "icwf_exact2d_set_state": [H, d],
        "icwf_exact2d_set_projectors": [H, ct.c_int32, d],
        "icwf_exact2d_step": [H, ct.c_int32],
        "icwf_exact2d_get_state": [H, d],
        "icwf_exact2d_observables": [H, P(icwf_obs)],
        "icwf_exact2d_destroy": [H],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ct.c_int
    lib.icwf_last_error.argtypes = [H]
    lib.icwf_last_error.restype = ct.c_char_p
    lib.icwf_exact2d_last_error.argtypes = [H]
    lib.icwf_exact2d_last_error.restype = ct.c_char_p
    return lib


LIB = _load()


def _dp(a):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))


def _check(st, h=None):
    if st != ICWF_OK:
        raise IcwfError(st, LIB.icwf_last_error(h).decode())


def _c128(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.shape == shape, (a.shape, shape)
    return a


# ---- functions with the C names ---------------------------------------------------------------

def icwf_create(params: icwf_params, V: np.ndarray):
    V = np.ascontiguousarray(V, dtype=np.float64)
    assert V.shape == (params.nx, params.nR)
    h = ct.c_void_p()
    _check(LIB.icwf_create(ct.byref(params), _dp(V), ct.byref(h)))
    return h


def icwf_set_projectors(h, phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    _check(LIB.icwf_set_projectors(h, phi.shape[0], _dp(phi)), h)


def icwf_init_from_density(h, psi0: np.ndarray, seed: int):
    psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    _check(LIB.icwf_init_from_density(h, psi0.ctypes.data_as(ct.POINTER(ct.c_double)),
                                      ct.c_uint64(seed)), h)


def icwf_init_from_positions(h, psi0: np.ndarray, x: np.ndarray, R: np.ndarray):
    psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    _check(LIB.icwf_init_from_positions(h, psi0.ctypes.data_as(ct.POINTER(ct.c_double)),
                                        _dp(x), _dp(R)), h)


def icwf_step(h, n_steps: int):
    _check(LIB.icwf_step(h, int(n_steps)), h)


def icwf_observables(h, nx: int, nR: int, n_states: int = 8) -> dict:
    rho_x = np.zeros(nx)
    rho_R = np.zeros(nR)
    pop = np.zeros(8)
    decoh = np.zeros(64)
    o = icwf_obs()
    o.rho_x, o.rho_R, o.pop, o.decoh = _dp(rho_x), _dp(rho_R), _dp(pop), _dp(decoh)
    _check(LIB.icwf_observables(h, ct.byref(o)), h)
    ns = o.n_states
    return {"t": o.t, "norm": o.norm, "energy": o.energy, "rho_x": rho_x, "rho_R": rho_R,
            "pop": pop[:ns].copy(), "decoherence": decoh[:ns * ns].reshape(ns, ns).copy(),
            "n_clamped": o.n_clamped}


def icwf_observables_static(h, nx: int, nR: int) -> dict:
    """icwf_observables without device allocation (fixed library work area; see icwf.h)."""
    rho_x = np.zeros(nx)
    rho_R = np.zeros(nR)
    pop = np.zeros(8)
    decoh = np.zeros(64)
    o = icwf_obs()
    o.rho_x, o.rho_R, o.pop, o.decoh = _dp(rho_x), _dp(rho_R), _dp(pop), _dp(decoh)
    _check(LIB.icwf_observables_static(h, ct.byref(o)), h)
    ns = o.n_states
    return {"t": o.t, "norm": o.norm, "energy": o.energy, "rho_x": rho_x, "rho_R": rho_R,
            "pop": pop[:ns].copy(), "decoherence": decoh[:ns * ns].reshape(ns, ns).copy(),
            "n_clamped": o.n_clamped}


def icwf_destroy(h):
    if h is not None and h.value:
        _check(LIB.icwf_destroy(h))


def icwf_get_state(h, N: int, nx: int, nR: int, cwfs: bool = True) -> dict:
    C = np.zeros(N, dtype=np.complex128)
    x = np.zeros(N)
    R = np.zeros(N)
    psi = np.zeros((N, nx), dtype=np.complex128) if cwfs else None
    chi = np.zeros((N, nR), dtype=np.complex128) if cwfs else None
    cp = lambda a: None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))
    _check(LIB.icwf_get_state(h, cp(C), _dp(x), _dp(R), cp(psi), cp(chi)), h)
    out = {"C": C, "x": x, "R": R}
    if cwfs:
        out["psi"] = psi.T.copy()       # nx x N, column a = psi_a
        out["chi"] = chi.T.copy()
    return out


def icwf_get_matrices(h, N: int, want_H: bool = False) -> dict:
    S = np.zeros((N, N), dtype=np.complex128)
    He = np.zeros((N, N), dtype=np.complex128)
    Hm = np.zeros((N, N), dtype=np.complex128) if want_H else None
    cp = lambda a: None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))
    _check(LIB.icwf_get_matrices(h, cp(S), cp(Hm), cp(He)), h)
    out = {"S": S, "Heff": He}
    if want_H:
        out["H"] = Hm
    return out


def icwf_get_info(h) -> dict:
    i = icwf_info()
    _check(LIB.icwf_get_info(h, ct.byref(i)), h)
    return {k: getattr(i, k) for k, _ in icwf_info._fields_}


def icwf_set_regularisation(h, eps: float):
    _check(LIB.icwf_set_regularisation(h, ct.c_double(eps)), h)


def icwf_set_wait_limit(h, polls: int):
    _check(LIB.icwf_set_wait_limit(h, ct.c_int64(polls)), h)


def icwf_heff_direct(h, N: int, cols) -> np.ndarray:
    """Heff[:, cols] by the full double sum over the grid (N x len(cols) complex128)."""
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros((len(cols), N), dtype=np.complex128)
    _check(LIB.icwf_heff_direct(h, len(cols), cols.ctypes.data_as(ct.POINTER(ct.c_int32)),
                                out.ctypes.data_as(ct.POINTER(ct.c_double))), h)
    return out.T.copy()


def icwf_save_state(h) -> bytes:
    n = ct.c_size_t()
    _check(LIB.icwf_state_bytes(h, ct.byref(n)), h)
    buf = ct.create_string_buffer(n.value)
    _check(LIB.icwf_save_state(h, buf, n.value), h)
    return buf.raw


def icwf_load_state(h, blob: bytes):
    buf = ct.create_string_buffer(blob, len(blob))
    _check(LIB.icwf_load_state(h, buf, len(blob)), h)


def icwf_get_stream(h) -> int:
    s = ct.c_void_p()
    _check(LIB.icwf_get_stream(h, ct.byref(s)), h)
    return s.value or 0


def icwf_profile_enable(h, on: bool = True):
    _check(LIB.icwf_profile_enable(h, 1 if on else 0), h)


def icwf_profile_reset(h):
    _check(LIB.icwf_profile_reset(h), h)


def icwf_profile_read(h) -> dict:
    n = 32
    names = (ct.c_char_p * n)()
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    nout = ct.c_int32()
    _check(LIB.icwf_profile_read(h, n, names, _dp(ms), cnt.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                 ct.byref(nout)), h)
    return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(nout.value)}


def icwf_pool_create(hbm_budget_bytes: int, max_jobs: int):
    p = ct.c_void_p()
    _check(LIB.icwf_pool_create(ct.c_size_t(hbm_budget_bytes), max_jobs, ct.byref(p)))
    return p


def icwf_pool_submit(pool, job, n_steps: int) -> int:
    jid = ct.c_int32()
    _check(LIB.icwf_pool_submit(pool, job, ct.c_int64(n_steps), ct.byref(jid)))
    return jid.value


def icwf_pool_tick(pool):
    nl = ct.c_int32()
    nf = ct.c_int32()
    _check(LIB.icwf_pool_tick(pool, ct.byref(nl), ct.byref(nf)))
    return nl.value, nf.value


def icwf_pool_poll(pool, job_id: int, nx: int, nR: int):
    rho_x = np.zeros(nx)
    rho_R = np.zeros(nR)
    pop = np.zeros(8)
    decoh = np.zeros(64)
    o = icwf_obs()
    o.rho_x, o.rho_R, o.pop, o.decoh = _dp(rho_x), _dp(rho_R), _dp(pop), _dp(decoh)
    state = ct.c_int32()
    _check(LIB.icwf_pool_poll(pool, job_id, ct.byref(o), ct.byref(state)))
    if state.value != 2:
        return state.value, None
    ns = o.n_states
    return state.value, {"t": o.t, "norm": o.norm, "energy": o.energy, "rho_x": rho_x,
                         "rho_R": rho_R, "pop": pop[:ns].copy(),
                         "decoherence": decoh[:ns * ns].reshape(ns, ns).copy(),
                         "n_clamped": o.n_clamped}


def icwf_pool_get_stats(pool) -> dict:
    st = icwf_pool_stats()
    _check(LIB.icwf_pool_get_stats(pool, ct.byref(st)))
    return {k: getattr(st, k) for k, _ in icwf_pool_stats._fields_}


def icwf_pool_set_graphs(pool, on: bool):
    _check(LIB.icwf_pool_set_graphs(pool, 1 if on else 0))


def icwf_pool_set_grouping(pool, on: bool, max_ctas: int = 0):
    _check(LIB.icwf_pool_set_grouping(pool, 1 if on else 0, max_ctas))


def icwf_pool_destroy(pool):
    _check(LIB.icwf_pool_destroy(pool))


# ---- convenience wrapper (marshalling only) ---------------------------------------------------

def params_from(w, precision: int = ICWF_FP64, coeff_scheme: int = 0, **over) -> icwf_params:
    """icwf_params from any object with the workload attributes (nx, nR, extents, masses, dt,
    n_traj, svd_rel_cutoff, s_reg_eps)."""
    d = dict(nx=w.nx, nR=w.nR, x_min=w.x_min, x_max=w.x_max, R_min=w.R_min, R_max=w.R_max,
             mass_x=w.mass_x, mass_R=w.mass_R, dt=w.dt, n_traj=w.n_traj, precision=precision,
             svd_rel_cutoff=w.svd_rel_cutoff, s_reg_eps=w.s_reg_eps, coeff_scheme=coeff_scheme,
             max_rank=0, solve_fp64=0, overlap_split=0)
    d.update(over)
    return icwf_params(**d)


class Icwf:
    """Owns one handle.  Methods map one-to-one onto the C calls."""

    def __init__(self, params: icwf_params, V: np.ndarray):
        self.p = params
        self.h = icwf_create(params, V)

    def close(self):
        if self.h is not None:
            icwf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_projectors(self, phi):
        icwf_set_projectors(self.h, phi)

    def init_from_density(self, psi0, seed):
        icwf_init_from_density(self.h, psi0, seed)

    def init_from_positions(self, psi0, x, R):
        icwf_init_from_positions(self.h, psi0, x, R)

    def step(self, n=1):
        icwf_step(self.h, n)

    def observables(self):
        return icwf_observables(self.h, self.p.nx, self.p.nR)

    def state(self, cwfs=True):
        return icwf_get_state(self.h, self.p.n_traj, self.p.nx, self.p.nR, cwfs)

    def matrices(self, want_H=False):
        return icwf_get_matrices(self.h, self.p.n_traj, want_H)

    def info(self):
        return icwf_get_info(self.h)

    def save_state(self) -> bytes:
        return icwf_save_state(self.h)

    def load_state(self, blob: bytes):
        icwf_load_state(self.h, blob)

    def heff_direct(self, cols):
        return icwf_heff_direct(self.h, self.p.n_traj, cols)

    def stream(self):
        return icwf_get_stream(self.h)

    def set_regularisation(self, eps):
        icwf_set_regularisation(self.h, eps)

    def set_wait_limit(self, polls):
        icwf_set_wait_limit(self.h, polls)

    def set_step_graphs(self, on):
        _check(LIB.icwf_set_step_graphs(self.h, 1 if on else 0), self.h)

    def set_emulated_update(self, on):
        """FP64 solver: trailing updates of the factorisation on the tensor cores in emulated FP64
        (default) or with FP64 FMAs."""
        _check(LIB.icwf_set_emulated_update(self.h, 1 if on else 0), self.h)

    def release(self):
        """Give up ownership (after icwf_pool_submit the pool owns the handle)."""
        h, self.h = self.h, None
        return h


# ---- exact 2D propagation (include/icwf_exact2d.h) ---------------------------------------------

def _check2(st, h=None):
    if st != ICWF_OK:
        raise IcwfError(st, LIB.icwf_exact2d_last_error(h).decode())


def icwf_exact2d_create(params: icwf_params, V: np.ndarray):
    V = np.ascontiguousarray(V, dtype=np.float64)
    assert V.shape == (params.nx, params.nR)
    h = ct.c_void_p()
    _check2(LIB.icwf_exact2d_create(ct.byref(params), _dp(V), ct.byref(h)))
    return h


class Exact2D:
    """The exact Strang-split propagation of Psi(x, R) on the GPU (FP64), same grid, masses, V
    and dt as an ICWF parameter set."""

    def __init__(self, params: icwf_params, V: np.ndarray):
        self.nx, self.nR = params.nx, params.nR
        self.h = icwf_exact2d_create(params, V)
        self.n_states = 0

    def set_state(self, psi: np.ndarray):
        psi = _c128(psi, (self.nx, self.nR))
        _check2(LIB.icwf_exact2d_set_state(self.h, psi.ctypes.data_as(ct.POINTER(ct.c_double))),
                self.h)

    def set_projectors(self, phi: np.ndarray):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        _check2(LIB.icwf_exact2d_set_projectors(self.h, phi.shape[0], _dp(phi)), self.h)
        self.n_states = phi.shape[0]

    def step(self, n: int = 1):
        _check2(LIB.icwf_exact2d_step(self.h, n), self.h)

    def state(self) -> np.ndarray:
        out = np.empty((self.nx, self.nR), dtype=np.complex128)
        _check2(LIB.icwf_exact2d_get_state(self.h, out.ctypes.data_as(ct.POINTER(ct.c_double))),
                self.h)
        return out

    def observables(self) -> dict:
        rx, rR = np.empty(self.nx), np.empty(self.nR)
        ns = max(self.n_states, 1)
        pop, dec = np.zeros(ns), np.zeros(ns * ns)
        o = icwf_obs(rho_x=_dp(rx), rho_R=_dp(rR), pop=_dp(pop), decoh=_dp(dec))
        _check2(LIB.icwf_exact2d_observables(self.h, ct.byref(o)), self.h)
        out = dict(t=o.t, norm=o.norm, energy=o.energy, rho_x=rx, rho_R=rR)
        if self.n_states:
            out["pop"] = pop[:self.n_states]
            out["decoherence"] = dec.reshape(ns, ns)[:self.n_states, :self.n_states]
        return out

    def close(self):
        if self.h is not None:
            LIB.icwf_exact2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
