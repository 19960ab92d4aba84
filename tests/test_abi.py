"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/*.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(icwf_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["icwf_create", "icwf_init_from_density", "icwf_step", "icwf_observables",
              "icwf_destroy", "icwf_pool_create", "icwf_pool_tick"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    """Argument validation happens on the host before any device call."""
    import numpy as np
    import paper_1805_11169_gb300 as g
    p = g.icwf_params(nx=100, nR=64, x_min=-1, x_max=1, R_min=-1, R_max=1, mass_x=1, mass_R=1,
                      dt=0.1, n_traj=4, precision=0, svd_rel_cutoff=0, s_reg_eps=1e-10,
                      coeff_scheme=0, max_rank=0)
    with pytest.raises(g.IcwfError) as e:
        g.icwf_create(p, np.zeros((100, 64)))
    assert e.value.status == g.ICWF_ERR_ARG and "powers of two" in str(e.value)
    p.nx = 64
    p.dt = -1.0
    with pytest.raises(g.IcwfError):
        g.icwf_create(p, np.zeros((64, 64)))
    p.dt = 0.1
    V = np.zeros((64, 64))
    V[3, 3] = np.nan
    with pytest.raises(g.IcwfError) as e:
        g.icwf_create(p, V)
    assert "non-finite" in str(e.value)


def test_null_handle_calls_are_rejected(lib):
    import paper_1805_11169_gb300 as g
    assert g.LIB.icwf_step(None, 1) == g.ICWF_ERR_ARG
    assert g.LIB.icwf_destroy(None) == g.ICWF_OK
    assert g.LIB.icwf_pool_destroy(None) == g.ICWF_OK
    assert g.LIB.icwf_pool_set_grouping(None, 1, 0) == g.ICWF_ERR_ARG
    assert g.LIB.icwf_pool_set_graphs(None, 1) == g.ICWF_ERR_ARG


def test_exact2d_rejects_bad_arguments_without_a_gpu(lib):
    import numpy as np
    import paper_1805_11169_gb300 as g
    p = g.icwf_params(nx=100, nR=64, x_min=-1, x_max=1, R_min=-1, R_max=1, mass_x=1, mass_R=1,
                      dt=0.1)
    with pytest.raises(g.IcwfError) as e:
        g.icwf_exact2d_create(p, np.zeros((100, 64)))
    assert e.value.status == g.ICWF_ERR_ARG and "powers of two" in str(e.value)
    p.nx = 64
    p.mass_R = 0.0
    with pytest.raises(g.IcwfError) as e:
        g.icwf_exact2d_create(p, np.zeros((64, 64)))
    assert e.value.status == g.ICWF_ERR_ARG
    assert g.LIB.icwf_exact2d_step(None, 1) == g.ICWF_ERR_ARG
    assert g.LIB.icwf_exact2d_destroy(None) == g.ICWF_OK
