"""Physics pins of the FP64 oracle against the paper's closed forms for stripes (Sec. 3).

Both runs are azimuthally symmetric, so N_phi = 1 (as in the paper's own stripe runs).
Laplace pressure: Eq. stripe_laplace_gen at the measured centre and width, after relaxation.
Oscillation: a stripe displaced by pi/20 from theta = pi oscillates at omega_0 of
Eq. stripe_hydro_omega0_pi; the damping is checked only loosely, because the paper gives the
viscous part alpha_nu (Eq. stripe_alphanu) but no formula for the mobility part alpha_mu, which is
not small at these parameters.  The torus for the oscillation is the paper's shape a = 0.4 scaled to
r = 0.5 with kappa = 2e-3, so that one period is 27 time units (CPU time of the oracle).
"""
import math

import numpy as np
import pytest

from oracle import analysis as AN
from oracle import closed_forms as C
from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import inputs


def _stable_dt(p, factor):
    h = p.r * 2 * math.pi / p.n_theta
    lam = 4.0 / h ** 2
    return factor * min(h / math.sqrt(3 + math.sqrt(6)), 2.5 * p.tau, 2.5 / (p.M * lam * (p.kappa * lam + 2 * p.A)))


@pytest.mark.slow
def test_laplace_pressure_of_a_relaxed_stripe():
    R, r, A, kappa = 2.0, 0.8, 0.5, 1e-3
    nt, width = 128, 0.3 * math.pi
    p = O.Params(R=R, r=r, n_theta=nt, n_phi=1, dt=1.0, tau=0.3, M=0.01, A=A, kappa=kappa)
    p.dt = _stable_dt(p, 0.5)
    geo = O.Geometry(p)
    off = C.stripe_offset(R, r, kappa, A, math.pi, width)
    phi = inputs.stripe_phi(R, r, nt, 1, math.pi, width, math.sqrt(kappa / A), offset=off, inside=-1.0)
    f, ph = O.init_state(np.ones_like(phi), 0 * phi, 0 * phi, phi)
    f, ph = O.run(f, ph, geo, int(20.0 / p.dt))
    n, ut, _ = O.moments(f)
    tc, w = AN.stripe_centre(ph[:, 0], -1.0)
    dp = AN.band_pressure_jump(O.pressure(n[:, 0], ph[:, 0], A), tc, w)
    expect = C.laplace_pressure(R, r, kappa, A, tc, w)
    assert abs(tc - math.pi) < 1e-6  # sub-critical stripes sit at theta = pi
    assert abs(dp / expect - 1.0) < 0.06, (dp, expect)
    assert np.max(np.abs(ut)) < 1e-4  # relaxed


@pytest.mark.slow
def test_stripe_oscillation_frequency():
    from scipy.optimize import curve_fit
    R, r, A, kappa, nu, M = 1.25, 0.5, 0.5, 2e-3, 5e-3, 2.5e-3
    nt = 128
    area = C.stripe_area(R, r, math.pi, 0.28 * math.pi)
    _, w_eq = C.equilibrium(R, r, area)
    omega0 = C.omega0_subcritical(R, r, kappa, A, w_eq)
    theta0 = math.pi - math.pi / 20
    w_init = C.width_for_area(R, r, theta0, area)
    p = O.Params(R=R, r=r, n_theta=nt, n_phi=1, dt=1.0, tau=nu, M=M, A=A, kappa=kappa)
    p.dt = _stable_dt(p, 0.6)
    geo = O.Geometry(p)
    off = C.stripe_offset(R, r, kappa, A, theta0, w_init)
    phi = inputs.stripe_phi(R, r, nt, 1, theta0, w_init, math.sqrt(kappa / A), offset=off, inside=-1.0)
    f, ph = O.init_state(np.ones_like(phi), 0 * phi, 0 * phi, phi)
    steps = int(0.8 * 2 * math.pi / omega0 / p.dt)
    every = max(1, steps // 150)
    ts, tcs = [], []
    for k in range(steps + 1):
        if k % every == 0:
            ts.append(k * p.dt)
            tcs.append(AN.stripe_centre(ph[:, 0], -1.0)[0])
        f, ph = O.step(f, ph, geo)
    ts, tcs = np.array(ts), np.unwrap(np.array(tcs)) - math.pi

    def model(t, amp, w, phase, alpha, c):
        return amp * np.cos(w * t + phase) * np.exp(-alpha * t) + c

    popt, _ = curve_fit(model, ts, tcs, p0=[-math.pi / 20, omega0, 0.0, 1e-3, 0.0], maxfev=20000)
    assert abs(abs(popt[1]) / omega0 - 1.0) < 0.03, (popt[1], omega0)
    a_nu = C.alpha_nu(R, r, nu)
    assert 0.5 * a_nu < popt[3] < 5.0 * a_nu, (popt[3], a_nu)


def test_equal_area_drop_radii_match_the_printed_values():
    """The drop-drift figure prints R_0 for three drop centres (tests/golden/drop_radii_printed.txt).
    Solving the equal-area condition with the drop profile of Eq. drop_init (Euclidean distance, the
    A8 reading) and the torus area element reproduces all three to the printed three decimals."""
    import os
    R, r, kappa, A = 2.0, 0.8, 5e-4, 0.5
    xi = C.xi0(kappa, A)
    path = os.path.join(os.path.dirname(__file__), "golden", "drop_radii_printed.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for t0, r0 in rows:
        got = AN.equal_area_drop_radius(R, r, xi, float(t0) * math.pi, 0.0, 30.0 * xi)
        assert abs(got - float(r0)) <= 0.0006, (t0, got, r0)


def test_stripe_area_ratios_printed_with_the_equilibrium_figure():
    """The stripe-equilibrium subsection prints Delta A / Delta A_crit for its four stripes
    (tests/golden/stripe_fork_area_ratios_printed.txt).  The stripe area at theta_c = pi/2 over
    Eq. stripe_dA_crit reproduces all four to the printed two decimals."""
    import os
    R, r = 2.0, 0.8
    path = os.path.join(os.path.dirname(__file__), "golden", "stripe_fork_area_ratios_printed.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for w, ratio in rows:
        got = C.stripe_area(R, r, math.pi / 2, float(w) * math.pi) / C.critical_area(R, r)
        assert abs(got - float(ratio)) <= 0.006, (w, got, ratio)
