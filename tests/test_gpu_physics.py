"""Physics of the CUDA path: a stripe displaced by pi/20 from theta = pi oscillates at omega_0 of
Eq. stripe_hydro_omega0_pi, in FP64 and FP32, for both widths of the stripe workload (R = 3, r = 1,
xi = 0.05, tau = M = 2.5e-3).  The paper requires the grid spacing below the interface width
(Sec. 3.1); the workload's 128 x 384 grid has r dtheta = 0.049 ~ xi, so the check runs the same
stripe at N_theta = 512 (spacing xi / 4).  The stripe is azimuthally symmetric: N_phi = 4."""
import math

import numpy as np
import pytest

from oracle import analysis as AN
from oracle import closed_forms as C
from paper_1904_10070_gb300 import inputs, vlb
from tests.gpu_helpers import gpu_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [0.6, 1.2])
@pytest.mark.parametrize("precision", [vlb.FP64, vlb.FP32])
def test_stripe_oscillates_at_omega0(width, precision):
    from scipy.optimize import curve_fit
    base = inputs.workload("stripe_torus_128x384")["params"]
    p = dict(base, n_theta=512, n_phi=4)
    p["dt"] = 0.5 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
    w = inputs._stripe(p, width=width, steps=0)
    R, r, A, kappa = p["R"], p["r"], p["A"], p["kappa"]
    theta0 = math.pi - math.pi / 20
    area = C.stripe_area(R, r, theta0, width)
    tc_eq, w_eq = C.equilibrium(R, r, area)
    omega0 = C.omega0_subcritical(R, r, kappa, A, w_eq)
    s = vlb.Solver(gpu_params(p, precision))
    s.set_fields(w["rho"], w["ut"], w["up"], -w["phi"])  # the paper's convention: the band is phi = -1
    steps = int(1.0 * 2 * math.pi / omega0 / p["dt"])
    every = max(1, steps // 200)
    ts, tcs = [], []
    for k in range(0, steps + 1, every):
        phi = s.fields()[3]
        ts.append(k * p["dt"])
        tcs.append(AN.stripe_centre(phi.mean(axis=1), -1.0)[0])
        s.step(every)
    s.close()
    ts, tcs = np.array(ts), np.unwrap(np.array(tcs)) - tc_eq

    def model(t, amp, om, phase, alpha, c):
        return amp * np.cos(om * t + phase) * np.exp(-alpha * t) + c

    popt, _ = curve_fit(model, ts, tcs, p0=[-math.pi / 20, omega0, 0.0, 1e-3, 0.0], maxfev=20000)
    print(f"width {width} precision {precision}: omega fit {abs(popt[1]):.4f}, theory {omega0:.4f}")
    assert abs(abs(popt[1]) / omega0 - 1.0) < 0.05
