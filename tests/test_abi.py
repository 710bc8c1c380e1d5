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


UW3_STENCIL = ([-2, -1, 0, 1], [1.0, -6.0, 3.0, 2.0], 6.0)
# the fifth-order upwind difference that WENO5 reduces to with its linear weights
WENO5_STENCIL = ([-3, -2, -1, 0, 1, 2], [-2.0, 15.0, -60.0, 20.0, 30.0, -3.0], 60.0)


def _rk3_amplification(dt, ht, hp, tau, n=128, stencil=UW3_STENCIL):
    """max |1 + z + z^2/2 + z^3/6| over n x n Fourier modes and |v| pairs for an upwind difference
    (stencil offsets, weights, divisor) with relaxation 1/tau."""
    import numpy as np
    k = -np.pi + 2 * np.pi * np.arange(n) / n
    offsets, weights = np.array(stencil[0]), np.array(stencil[1]) / stencil[2]
    assert abs(weights.sum()) < 1e-15 and abs((weights * offsets).sum() - 1.0) < 1e-15  # consistent first derivative
    D = (weights[None, :] * np.exp(1j * k[:, None] * offsets[None, :])).sum(axis=1)
    worst = 0.0
    for vi in (math.sqrt(3 - math.sqrt(6)), math.sqrt(3 + math.sqrt(6))):
        for vj in (math.sqrt(3 - math.sqrt(6)), math.sqrt(3 + math.sqrt(6))):
            z = dt * (-vi / ht * D[:, None] - vj / hp * D[None, :] - 1.0 / tau)
            worst = max(worst, float(np.abs(1 + z + z * z / 2 + z ** 3 / 6).max()))
    return worst


def test_max_stable_dt_relaxation_and_advection_together(L):
    # stripe regime: dt / tau near 2 with advection in both directions; the separate limits give
    # 2.5 tau = 6.25e-3, at which RK3 amplifies some modes; the combined limit is the largest
    # stable dt of the linear model, checked here on a finer mode grid
    p = _p(R=3.0, r=1.0, n_theta=128, n_phi=384, tau=2.5e-3, M=2.5e-3, A=0.5, kappa=1.25e-3)
    dt = vlb.vlb_max_stable_dt(p)
    ht, hp = 2 * math.pi / 128, 2.0 * 2 * math.pi / 384
    assert dt < 2.5 * 2.5e-3
    assert _rk3_amplification(0.995 * dt, ht, hp, 2.5e-3) <= 1.0 + 1e-9
    assert _rk3_amplification(1.02 * dt, ht, hp, 2.5e-3) > 1.0
    assert _rk3_amplification(2.5 * 2.5e-3, ht, hp, 2.5e-3) > 1.3


@pytest.mark.parametrize("geometry,adv", [(vlb.TORUS, vlb.WENO5), (vlb.FLAT, vlb.UW3)])
def test_max_stable_dt_combined_bound_other_scheme_and_geometry(L, geometry, adv):
    p = _p(R=3.0, r=1.0, n_theta=128, n_phi=384, tau=2.5e-3, M=2.5e-3, A=0.5, kappa=1.25e-3)
    p.geometry, p.advection = geometry, adv
    dt = vlb.vlb_max_stable_dt(p)
    ht = 2 * math.pi / 128
    hp = (2.0 if geometry == vlb.TORUS else 3.0) * 2 * math.pi / 384  # inner equator, or R dvarphi flat
    stencil = WENO5_STENCIL if adv == vlb.WENO5 else UW3_STENCIL
    assert dt < 2.5 * 2.5e-3
    assert _rk3_amplification(0.995 * dt, ht, hp, 2.5e-3, stencil=stencil) <= 1.0 + 1e-9
    assert _rk3_amplification(1.02 * dt, ht, hp, 2.5e-3, stencil=stencil) > 1.0


def test_named_workloads_step_below_the_stable_limit(L):
    from paper_1904_10070_gb300 import inputs
    for name in ("drop_torus_32x64", "stripe_torus_128x384", "coarsen_torus_1024x2048", "coarsen_flat_1024x2048"):
        w = inputs.workload(name)["params"]
        assert w["dt"] <= vlb.vlb_max_stable_dt(vlb.make_params(**w)), name


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


def test_noalloc_rejects_a_stride_whose_size_would_wrap_around(L):
    """A stride of 2^60 elements makes the scratch size wrap around 2^64; it must be rejected before
    any size arithmetic (no device is touched: the call fails on its arguments)."""
    p = _p(precision=vlb.FP32)
    for stride in (1 << 60, (1 << 62) + 64 * 5, vlb.NOALLOC_SCRATCH_BYTES):
        with pytest.raises(vlb.VlbError) as exc:
            vlb.vlb_step_noalloc(p, 256, stride, 1.0, 1, 0)
        assert exc.value.status == vlb.VLB_ERR_ARG
        assert "stride" in str(exc.value)


def test_stabilised_cahn_hilliard_parameters(L):
    """ch_stab = 1 needs power-of-two grids (its Fourier solve); it lifts the Cahn-Hilliard limit of
    vlb_max_stable_dt, and ensembles and the no-allocation step refuse it."""
    assert vlb.vlb_workspace_bytes(_p(n_theta=48, n_phi=64, ch_stab=1)) == 0
    assert "powers of two" in L.vlb_last_error(None).decode()
    assert vlb.vlb_workspace_bytes(_p(ch_stab=2)) == 0
    base = dict(n_theta=1024, n_phi=2048, R=2.0, M=2.5e-3, A=0.5, kappa=5e-4, tau=0.6)
    n_exp = vlb.vlb_workspace_bytes(_p(**base))
    n_stab = vlb.vlb_workspace_bytes(_p(**base, ch_stab=1))
    assert n_stab >= n_exp + 1024 * 2048 * 8 * 3  # dt L_phi and the complex spectrum
    dt_exp = vlb.vlb_max_stable_dt(_p(**base))
    dt_stab = vlb.vlb_max_stable_dt(_p(**base, ch_stab=1))
    assert dt_stab > 50 * dt_exp  # the explicit Cahn-Hilliard limit (7e-6 here) no longer binds
    with pytest.raises(vlb.VlbError) as exc:
        vlb.vlb_step_noalloc(_p(precision=vlb.FP32, ch_stab=1), 256, 2048, 1.0, 1, 0)
    assert exc.value.status == vlb.VLB_ERR_ARG
    assert vlb.vlb_ensemble_workspace_bytes([_p(precision=vlb.FP32, ch_stab=1)]) == 0
