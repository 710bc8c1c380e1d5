"""Stripe suite on the CUDA path (FP32, the production precision) against the paper's closed forms
for stripes on a torus (Sec. 3): R = 3, r = 1, A = 0.5, xi = 0.05, M = 2.5e-3, 512 theta rows (grid
spacing xi / 4).  The stripes are azimuthally symmetric: the oscillation fits run on one varphi column
(the single-CTA axisymmetric kernel), the Laplace pressures on one and on four columns (the tile
kernel).

  * Laplace pressure at equilibrium on both branches: a wide sub-critical stripe at theta = pi and a
    super-critical one at its off-pi equilibrium (Eqs. stripe_laplace_gen, stripe_thceq);
  * the oscillation frequency of a super-critical stripe about theta_c^eq (Eq. stripe_hydro_omega0_npi);
  * the viscous damping: d alpha / d nu = 1 / (R^2 - r^2) (Eq. stripe_alphanu) for r = 0.8, 1, 1.2.  The paper gives no
    closed form for the mobility part of the damping, which the slope in nu cancels."""
import math

import numpy as np
import pytest

from oracle import analysis as AN
from oracle import closed_forms as C
from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import inputs, vlb

pytestmark = pytest.mark.gpu

R, r, A, KAPPA, M = 3.0, 1.0, 0.5, 1.25e-3, 2.5e-3
NT = 512
XI = math.sqrt(KAPPA / A)


def _params(tau, minor=r, ns=1):
    p = dict(geometry=0, R=R, r=minor, n_theta=NT, n_phi=ns, dt=1.0, tau=tau, M=M, A=A, kappa=KAPPA, advection=0,
             ch_mode=0)
    p["dt"] = 0.5 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
    return p


def _stripe(p, theta_c, width):
    """A phi = -1 band (the paper's convention) with the offset of Eq. stripe_phi0, at rest."""
    s = vlb.Solver(vlb.make_params(**p, precision=vlb.FP32))
    off = C.stripe_offset(R, p["r"], KAPPA, A, theta_c, width)
    phi = inputs.stripe_phi(R, p["r"], NT, p["n_phi"], theta_c, width, XI, offset=off, inside=-1.0)
    z = np.zeros_like(phi)
    s.set_fields(np.ones_like(phi), z, z, phi)
    return s


def _measure(s):
    rho, _, _, phi, _ = s.fields()
    tc, w = AN.stripe_centre(phi.mean(axis=1), -1.0)
    return tc, w, rho.mean(axis=1), phi.mean(axis=1)


def _oscillation(p, area, tc_eq, tc0, omega, periods):
    """Fit theta_c(t) - tc_eq to a damped cosine over `periods` periods of omega; returns (omega, alpha)."""
    from scipy.optimize import curve_fit
    s = _stripe(p, tc0, C.width_for_area(R, p["r"], tc0, area))
    steps = int(periods * 2 * math.pi / omega / p["dt"])
    every = max(1, steps // 300)
    ts, tcs = [], []
    for k in range(0, steps + 1, every):
        ts.append(k * p["dt"])
        tcs.append(_measure(s)[0])
        s.step(every)
    s.close()
    ts, tcs = np.array(ts), np.unwrap(np.array(tcs)) - tc_eq

    def model(t, amp, om, ph, al, c):
        return amp * np.cos(om * t + ph) * np.exp(-al * t) + c

    popt, _ = curve_fit(model, ts, tcs, p0=[tcs[0], omega, 0.0, 1e-3, 0.0], maxfev=20000)
    return abs(popt[1]), popt[3]


@pytest.mark.parametrize("ns", [1, 4])
@pytest.mark.parametrize("branch", ["subcritical", "supercritical"])
def test_laplace_pressure_at_equilibrium(branch, ns):
    area = C.stripe_area(R, r, math.pi, 1.2 if branch == "subcritical" else 3.4)
    assert (area > C.critical_area(R, r)) == (branch == "supercritical")
    tc_eq, w_eq = C.equilibrium(R, r, area)
    p = _params(0.1, ns=ns)
    s = _stripe(p, tc_eq, w_eq)
    s.step(int(30.0 / p["dt"]))
    tc, w, rho, phi = _measure(s)
    s.close()
    dp = AN.band_pressure_jump(O.pressure(rho, phi, A), tc, w)
    expect = C.laplace_pressure(R, r, KAPPA, A, tc, w)
    print(f"{branch}: theta_c {tc:.5f} (eq {tc_eq:.5f}), width {w:.5f}, dp {dp:.6g}, Eq. stripe_laplace_gen {expect:.6g}")
    assert abs(tc - tc_eq) < 2e-3  # the stripe stays at its equilibrium position
    assert abs(dp / expect - 1.0) < 0.02
    assert abs(C.laplace_pressure_eq(R, r, KAPPA, A, w_eq, branch == "subcritical") / expect - 1.0) < 0.01


@pytest.mark.parametrize("ns", [1, 4])
def test_narrow_stripe_laplace_pressure_with_the_gradient_terms(ns):
    """A narrow sub-critical stripe (w = 0.6 = 12 xi): the interface tails overlap at the band centre,
    where phi stops short of the bulk value by eps ~ 4 e^(-sqrt2 w / (2 xi)) and Delta phi ~ 2 eps / xi^2.
    The bulk formula n + p_binary there misses the gradient term -kappa phi Delta phi ~ -2 A eps of the
    normal pressure (25% of Delta p); the theta-theta component of the pressure tensor of Eq. pbin
    carries it and meets Eq. stripe_laplace_gen."""
    area = C.stripe_area(R, r, math.pi, 0.6)
    tc_eq, w_eq = C.equilibrium(R, r, area)
    p = _params(0.1, ns=ns)
    s = _stripe(p, tc_eq, w_eq)
    s.step(int(30.0 / p["dt"]))
    tc, w, rho, phi = _measure(s)
    s.close()
    expect = C.laplace_pressure(R, r, KAPPA, A, tc, w)
    dp_bulk = AN.band_pressure_jump(O.pressure(rho, phi, A), tc, w)
    dp = AN.band_pressure_jump(AN.stripe_normal_pressure(rho, phi, r, R, A, KAPPA), tc, w)
    print(f"narrow: dp (bulk formula) {dp_bulk:.6g}, dp (normal pressure) {dp:.6g}, Eq. stripe_laplace_gen {expect:.6g}")
    assert abs(dp / expect - 1.0) < 0.02
    assert dp_bulk < 0.85 * expect  # the gap the gradient terms close


def test_supercritical_stripe_oscillates_at_omega0():
    area = C.stripe_area(R, r, math.pi, 3.4)
    tc_eq, w_eq = C.equilibrium(R, r, area)
    omega0 = C.omega0_supercritical(R, r, KAPPA, A, tc_eq, w_eq)
    om, _ = _oscillation(_params(M), area, tc_eq, tc_eq + 0.06, omega0, 1.5)
    print(f"super-critical: omega fit {om:.5f}, Eq. stripe_hydro_omega0_npi {omega0:.5f}")
    assert abs(om / omega0 - 1.0) < 0.03


@pytest.mark.parametrize("minor", [0.8, 1.0, 1.2])
def test_viscous_damping_grows_as_nu_over_R2_minus_r2(minor):
    """d alpha / d nu = 1 / (R^2 - r^2) on three tube radii (Eq. stripe_alphanu): 0.1196, 0.125, 0.1323."""
    area = C.stripe_area(R, minor, math.pi, 0.6)
    _, w_eq = C.equilibrium(R, minor, area)
    omega0 = C.omega0_subcritical(R, minor, KAPPA, A, w_eq)
    fits = {nu: _oscillation(_params(nu, minor), area, math.pi, math.pi - math.pi / 20, omega0, 2.0)
            for nu in (0.01, 0.05)}
    slope = (fits[0.05][1] - fits[0.01][1]) / (0.05 - 0.01)
    expect = 1.0 / (R * R - minor * minor)
    print(f"r = {minor}: damping fits (omega, alpha) by nu: {fits}, slope {slope:.5f}, Eq. stripe_alphanu {expect:.5f}")
    assert abs(slope / expect - 1.0) < 0.08
    for om, _ in fits.values():  # the frequency does not depend on nu
        assert abs(om / omega0 - 1.0) < 0.03
