"""Failure detection through the C ABI, without faulting, trapping or hanging the GPU.

* A blow-up is made on the host side of the physics: a NaN in the initial order parameter, or a time
  step ten times the stable one; the in-step diagnostics must return VLB_ERR_UNSTABLE.
* A device wait that gives up is represented by the test hook vlb_test_raise_flag, which writes the
  value a timed-out kernel would write into the handle's device flag (or the convolutions' flag);
  the synchronous calls must then return VLB_ERR_TIMEOUT until the state is reset.
"""
import math

import numpy as np
import pytest

from paper_1904_10070_gb300 import inputs, vlb

pytestmark = pytest.mark.gpu


def _params(precision=vlb.FP32, diag_every=0, dt_factor=0.5, nt=32, ns=64):
    p = dict(R=2.5, r=1.0, n_theta=nt, n_phi=ns, dt=1.0, tau=0.5, M=0.05, A=0.3, kappa=0.01)
    p["dt"] = dt_factor * vlb.vlb_max_stable_dt(vlb.make_params(**p))
    return vlb.make_params(**p, precision=precision, diag_every=diag_every)


def _fields(nt=32, ns=64):
    phi = np.tanh(3.0 * inputs.noise(3, nt, ns, 1.0))
    return np.ones((nt, ns)), np.zeros((nt, ns)), np.zeros((nt, ns)), phi


@pytest.mark.parametrize("precision", [vlb.FP32, vlb.FP64])
def test_nan_in_the_initial_state_is_reported_unstable(precision):
    s = vlb.Solver(_params(precision, diag_every=5))
    rho, ut, up, phi = _fields()
    phi[7, 11] = math.nan
    s.set_fields(rho, ut, up, phi)
    with pytest.raises(vlb.VlbError) as exc:
        s.step(10)
    assert exc.value.status == vlb.VLB_ERR_UNSTABLE
    assert "unstable" in str(exc.value)
    s.close()


def test_nan_density_is_rejected_at_set_time():
    s = vlb.Solver(_params())
    rho, ut, up, phi = _fields()
    rho[0, 0] = math.nan
    with pytest.raises(vlb.VlbError) as exc:
        s.set_fields(rho, ut, up, phi)
    assert exc.value.status == vlb.VLB_ERR_ARG
    s.close()


@pytest.mark.parametrize("precision", [vlb.FP32, vlb.FP64])
def test_ten_times_the_stable_step_is_reported_unstable(precision):
    s = vlb.Solver(_params(precision, diag_every=10, dt_factor=10.0))
    s.set_fields(*_fields())
    with pytest.raises(vlb.VlbError) as exc:
        for _ in range(20):
            s.step(10)
    assert exc.value.status == vlb.VLB_ERR_UNSTABLE
    assert vlb.vlb_steps_done(s.h) <= 200
    s.close()


def test_stable_step_with_diagnostics_returns_ok():
    s = vlb.Solver(_params(diag_every=7))
    s.set_fields(*_fields())
    s.step(50)
    assert np.all(np.isfinite(s.totals()))
    s.close()


@pytest.mark.parametrize("nphi", [64, 1])
def test_a_skipped_tile_is_reported_as_timeout_until_reset(nphi):
    s = vlb.Solver(_params(nt=32, ns=nphi))
    fields = _fields(32, nphi)
    s.set_fields(*fields)
    s.step(3)
    vlb.vlb_test_raise_flag(s.h, 2)  # what a stage kernel writes when a bulk-copy wait gives up
    s.step(1)  # asynchronous and without diagnostics: nothing is read yet
    for call in (s.fields, s.totals, s.get_state, s.interface_length):
        with pytest.raises(vlb.VlbError) as exc:
            call()
        assert exc.value.status == vlb.VLB_ERR_TIMEOUT, call
        assert "gave up" in str(exc.value)
    s.set_fields(*fields)  # a new state clears the flag
    s.step(2)
    assert np.all(np.isfinite(s.totals()))
    s.close()


def test_timeout_takes_precedence_in_a_diagnosed_step():
    s = vlb.Solver(_params(diag_every=2))
    s.set_fields(*_fields())
    vlb.vlb_test_raise_flag(s.h, 2)
    with pytest.raises(vlb.VlbError) as exc:
        s.step(4)
    assert exc.value.status == vlb.VLB_ERR_TIMEOUT
    vlb.vlb_test_raise_flag(s.h, 1)
    with pytest.raises(vlb.VlbError) as exc:
        s.step(2)
    assert exc.value.status == vlb.VLB_ERR_UNSTABLE
    vlb.vlb_test_raise_flag(s.h, 0)
    s.step(2)
    s.close()


def test_ensemble_member_reports_the_ensembles_timeout():
    members = []
    for R, (nt, ns) in ((2.0, (32, 64)), (3.0, (48, 128))):
        p = dict(R=R, r=1.0, n_theta=nt, n_phi=ns, dt=1.0, tau=0.6, M=2.5e-3, A=0.5, kappa=5e-4)
        p["dt"] = 0.5 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
        members.append(vlb.make_params(**p, precision=vlb.FP32))
    ens = vlb.Ensemble(members)
    for v, m in zip(ens.views, members):
        vlb.vlb_set_fields(v, *_fields(m.n_theta, m.n_phi))
    ens.step(3)
    assert all(np.all(np.isfinite(vlb.vlb_get_totals(v))) for v in ens.views)
    vlb.vlb_test_raise_flag(ens.h, 2)
    ens.step(2)
    for v in ens.views:
        with pytest.raises(vlb.VlbError) as exc:
            vlb.vlb_get_totals(v)
        assert exc.value.status == vlb.VLB_ERR_TIMEOUT
    ens.close()


def test_convolution_status_reports_and_clears_the_tensor_core_flag():
    import torch
    st = torch.cuda.current_stream().cuda_stream
    vlb.vlb_conv_status(st, clear=True)  # nothing raised so far
    vlb.vlb_test_raise_flag(None, 1)      # what a convolution kernel writes when a wait gives up
    with pytest.raises(vlb.VlbError) as exc:
        vlb.vlb_conv_status(st, clear=False)
    assert exc.value.status == vlb.VLB_ERR_TIMEOUT
    with pytest.raises(vlb.VlbError):
        vlb.vlb_conv_status(st, clear=True)  # still raised; cleared now
    vlb.vlb_conv_status(st, clear=True)
