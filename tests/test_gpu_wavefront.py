"""The wavefront schedule of vlb_step (whole SSP-RK3 steps in one persistent launch, intermediate stages
read back from L2) against the per-stage launches and the oracle.

The two schedules run the same tile code on the same inputs, so the states must agree bit for bit:
at the smallest grid the schedule accepts (11 bands), at the coarsening grid, on the flat domain, in the
diffusive mode, and with the steps cut into launches by the in-step diagnostics.  The oracle gate is
the FP32 parity gate.  A CTA that never reports its tiles (the test hook) makes the dependency waits
give up after their budget: the launch ends with VLB_ERR_TIMEOUT and the handle steps normally after a
reset."""
import numpy as np
import pytest

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import inputs, vlb
from tests.gpu_helpers import max_err, oracle_params

pytestmark = pytest.mark.gpu


def _params(nt, ns, geometry=0, ch_mode=0, diag_every=0):
    p = dict(geometry=geometry, R=2.0, r=1.0, n_theta=nt, n_phi=ns, dt=1.0, tau=0.6, M=2.5e-3, A=0.5,
             kappa=5e-4, advection=0, ch_mode=ch_mode)
    p["dt"] = 0.8 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
    return p, vlb.make_params(**p, precision=vlb.FP32, diag_every=diag_every)


def _fields(nt, ns, seed):
    phi = inputs.quenched_noise(seed, nt, ns, corr=4.0, width=1.5)
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, (nt, ns))
    ut = 0.02 * rng.uniform(-1, 1, (nt, ns))
    up = 0.02 * rng.uniform(-1, 1, (nt, ns))
    return rho, ut, up, phi


def _run(params, fields, steps, schedule, chunks=None):
    s = vlb.Solver(params)
    s.set_schedule(schedule)
    s.set_fields(*fields)
    for k in (chunks or [steps]):
        s.step(k)
    out = s.get_state(), s.schedule()
    s.close()
    return out


@pytest.mark.parametrize("nt,ns,geometry,ch_mode", [(176, 64, 0, 0), (256, 512, 0, 0), (256, 256, 1, 0),
                                                    (192, 128, 0, 1), (1024, 2048, 0, 0)])
def test_wavefront_equals_stage_launches_bit_for_bit(nt, ns, geometry, ch_mode):
    p, params = _params(nt, ns, geometry, ch_mode)
    fields = _fields(nt, ns, 40 + nt)
    steps = 7 if nt < 1024 else 3
    (fw, pw), sw = _run(params, fields, steps, vlb.SCHED_WAVE)
    (fs, ps), ss = _run(params, fields, steps, vlb.SCHED_STAGES)
    assert sw == vlb.SCHED_WAVE and ss == vlb.SCHED_STAGES
    np.testing.assert_array_equal(fw, fs)
    np.testing.assert_array_equal(pw, ps)
    assert np.all(np.isfinite(fw))


def test_wavefront_grouping_and_diagnostic_cuts_do_not_change_the_result():
    nt, ns = 256, 512
    p, params = _params(nt, ns)
    fields = _fields(nt, ns, 7)
    (f1, p1), _ = _run(params, fields, 12, vlb.SCHED_WAVE)
    (f2, p2), _ = _run(params, fields, 12, vlb.SCHED_WAVE, chunks=[1, 5, 2, 4])
    _, params_d = _params(nt, ns, diag_every=5)
    (f3, p3), _ = _run(params_d, fields, 12, vlb.SCHED_WAVE)
    for f, ph in ((f2, p2), (f3, p3)):
        np.testing.assert_array_equal(f, f1)
        np.testing.assert_array_equal(ph, p1)


def test_wavefront_matches_the_oracle():
    nt, ns, steps = 176, 64, 20
    p, params = _params(nt, ns)
    rho, ut, up, phi = _fields(nt, ns, 9)
    s = vlb.Solver(params)
    assert s.schedule() == vlb.SCHED_STAGES  # the default
    s.set_schedule(vlb.SCHED_WAVE)
    s.set_fields(rho, ut, up, phi)
    assert s.schedule() == vlb.SCHED_WAVE
    s.step(steps)
    g = s.fields()
    s.close()
    geo = O.Geometry(oracle_params(p))
    f, ph = O.init_state(rho, ut, up, phi)
    f, ph = O.run(f, ph, geo, steps)
    n, u_t, u_p = O.moments(f)
    for got, want in zip(g[:4], (n, u_t, u_p, ph)):
        assert max_err(got, want) <= 2e-5


def test_wavefront_needs_its_grid():
    _, params = _params(160, 64)  # 10 bands: too few for the ticket order
    s = vlb.Solver(params)
    assert s.schedule() == vlb.SCHED_STAGES
    with pytest.raises(vlb.VlbError) as exc:
        s.set_schedule(vlb.SCHED_WAVE)
    assert exc.value.status == vlb.VLB_ERR_ARG
    s.close()


def test_wavefront_wait_times_out_instead_of_hanging():
    nt, ns = 256, 512
    _, params = _params(nt, ns, diag_every=4)
    fields = _fields(nt, ns, 11)
    s = vlb.Solver(params)
    s.set_schedule(vlb.SCHED_WAVE)
    s.set_fields(*fields)
    vlb.vlb_test_wave_timeout(s.h, 0, 2_000_000)  # CTA 0 never reports; waits give up after ~1 ms
    with pytest.raises(vlb.VlbError) as exc:
        s.step(4)
    assert exc.value.status == vlb.VLB_ERR_TIMEOUT
    with pytest.raises(vlb.VlbError) as exc:
        s.totals()
    assert exc.value.status == vlb.VLB_ERR_TIMEOUT
    vlb.vlb_test_wave_timeout(s.h, -1, 0)
    s.set_fields(*fields)
    s.step(4)
    assert np.all(np.isfinite(s.totals()))
    s.close()
