"""CPU checks of the C ABI: the library loads, exports every symbol include/vlb.h declares, and the
host-only calls (parameter validation, workspace size, stable-dt estimate) behave as documented.
No call here touches a GPU."""
import math
import os
import re

import pytest

from paper_1904_10070_gb300 import vlb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(vlb_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(vlb.LIB_PATH):
        from paper_1904_10070_gb300 import build
        build.build()
    return vlb.lib()


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(vlb.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def _p(**kw):
    base = dict(R=2.5, r=1.0, n_theta=32, n_phi=64, dt=5e-3, tau=0.8, M=0.1, A=0.04, kappa=0.04)
    base.update(kw)
    return vlb.make_params(**base)


def test_workspace_size_and_validation(L):
    n64 = vlb.vlb_workspace_bytes(_p())
    n32 = vlb.vlb_workspace_bytes(_p(precision=vlb.FP32))
    N = 32 * 64
    assert n64 >= 3 * 17 * N * 8 + 17 * N * 8
    assert n32 >= 3 * 17 * N * 4 + 17 * N * 8
    assert n32 < n64
    for bad in (dict(R=1.0, r=2.0), dict(n_theta=3), dict(n_phi=0), dict(dt=0.0), dict(tau=-1.0),
                dict(M=-1.0), dict(precision=7), dict(advection=2), dict(ch_mode=3), dict(geometry=5),
                dict(n_theta=5, advection=vlb.WENO5), dict(dt=math.nan)):
        assert vlb.vlb_workspace_bytes(_p(**bad)) == 0, bad
        assert L.vlb_last_error(None).decode() != ""
    # flat geometry allows R <= r
    assert vlb.vlb_workspace_bytes(_p(R=1.0, r=2.0, geometry=vlb.FLAT)) > 0


def test_create_rejects_missing_or_small_workspace(L):
    import ctypes
    h = ctypes.c_void_p()
    p = _p()
    assert L.vlb_create(ctypes.byref(p), None, 0, None, ctypes.byref(h)) == vlb.VLB_ERR_WORKSPACE
    assert L.vlb_create(ctypes.byref(p), ctypes.c_void_p(256), 16, None, ctypes.byref(h)) == vlb.VLB_ERR_WORKSPACE
    assert L.vlb_create(ctypes.byref(p), ctypes.c_void_p(258), 1 << 30, None, ctypes.byref(h)) == vlb.VLB_ERR_WORKSPACE
    assert L.vlb_step(None, 1) == vlb.VLB_ERR_ARG
    assert L.vlb_destroy(None) == vlb.VLB_OK


def test_max_stable_dt_limits(L):
    # BGK limit 2.5 tau dominates with a tiny tau
    p = _p(tau=1e-4, M=0.0)
    assert abs(vlb.vlb_max_stable_dt(p) - 2.5e-4) < 1e-15
    # advection limit: 1 / (v_max (1/h_theta + 1/h_phi)), h_phi on the inner equator
    p = _p(tau=10.0, M=0.0)
    vmax = math.sqrt(3 + math.sqrt(6))
    ht, hp = 1.0 * 2 * math.pi / 32, (2.5 - 1.0) * 2 * math.pi / 64
    assert abs(vlb.vlb_max_stable_dt(p) - 1.0 / (vmax * (1 / ht + 1 / hp))) < 1e-15
    # Cahn-Hilliard limit on the 1024 x 2048 coarsening grid
    p = _p(R=2.0, n_theta=1024, n_phi=2048, tau=0.6, M=2.5e-3, A=0.5, kappa=5e-4)
    ht, hp = 2 * math.pi / 1024, 2 * math.pi / 2048
    lam = 4 / ht ** 2 + 4 / hp ** 2
    assert abs(vlb.vlb_max_stable_dt(p) - 2.5 / (2.5e-3 * lam * (5e-4 * lam + 1.0))) < 1e-18
