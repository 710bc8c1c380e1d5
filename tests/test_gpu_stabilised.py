"""The stabilised semi-implicit Cahn-Hilliard step (ch_stab = 1; not in the paper) through the C ABI
against the oracle's restatement (oracle.vlb_oracle.stabiliser / step), and what it is for: steps far
beyond the explicit dt ~ h^4 / (M kappa) limit that track the explicit solution.

Parity gates as for the explicit step: FP64 <= 1e-12 and FP32 <= 2e-5, relative L2 and element-wise."""
import numpy as np
import pytest

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import inputs, vlb
from tests.gpu_helpers import max_err, rel_err

pytestmark = pytest.mark.gpu

KEYS = ["R", "r", "n_theta", "n_phi", "dt", "tau", "M", "A", "kappa", "geometry", "advection", "ch_mode"]


def _fields(nt, ns, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, (nt, ns))
    ut, up = 0.03 * rng.uniform(-1, 1, (nt, ns)), 0.03 * rng.uniform(-1, 1, (nt, ns))
    phi = inputs.quenched_noise(seed, nt, ns, 2.0, 1.5)
    return rho, ut, up, phi


CASES = [  # (n_theta, n_phi, geometry, advection, ch_mode, multiple of the explicit Cahn-Hilliard limit)
    (32, 64, vlb.TORUS, vlb.UW3, vlb.HYDRO, 8.0),
    (64, 32, vlb.TORUS, vlb.UW3, vlb.DIFFUSIVE, 8.0),
    (16, 64, vlb.FLAT, vlb.WENO5, vlb.HYDRO, 5.0),
    (64, 128, vlb.TORUS, vlb.UW3, vlb.HYDRO, 10.0),
]


@pytest.mark.parametrize("nt,ns,geom,adv,mode,mult", CASES)
@pytest.mark.parametrize("precision,tol", [(vlb.FP64, 1e-12), (vlb.FP32, 2e-5)])
def test_stabilised_step_matches_the_oracle(nt, ns, geom, adv, mode, mult, precision, tol):
    p = dict(geometry=geom, R=2.5, r=1.0, n_theta=nt, n_phi=ns, dt=1.0, tau=0.3, M=0.5, A=0.3, kappa=0.05,
             advection=adv, ch_mode=mode)
    dt_exp = vlb.vlb_max_stable_dt(vlb.make_params(**p))
    dt_stab = vlb.vlb_max_stable_dt(vlb.make_params(**p, ch_stab=1))
    assert dt_stab > dt_exp
    p["dt"] = min(mult * dt_exp, 0.5 * dt_stab)
    steps = 40
    rho, ut, up, phi = _fields(nt, ns, nt + ns)
    s = vlb.Solver(vlb.make_params(**p, precision=precision, ch_stab=1))
    s.set_fields(rho, ut, up, phi)
    s.step(steps)
    g = s.fields()
    gt = s.totals()
    s.close()
    op = O.Params(**{k: p[k] for k in KEYS}, ch_stab=1)
    geo = O.Geometry(op)
    f, ph = O.init_state(rho, ut, up, phi)
    t0 = O.totals(f, ph, geo)
    f, ph = O.run(f, ph, geo, steps)
    n, u1, u2 = O.moments(f)
    for name, a, b in zip(("rho", "u_th", "u_ph", "phi"), g[:4], (n, u1, u2, ph)):
        assert rel_err(a, b) <= tol and max_err(a, b) <= tol, (name, rel_err(a, b), max_err(a, b))
    # conserved by the Fourier solve as by the explicit step
    assert abs(gt[0] - t0[0]) <= 1e-12 * abs(t0[0]) + (1e-6 * abs(t0[0]) if precision == vlb.FP32 else 0)
    assert abs(gt[1] - t0[1]) <= 1e-11 * np.sum(np.abs(phi) * geo.dA) + (
        1e-6 * np.sum(np.abs(phi) * geo.dA) if precision == vlb.FP32 else 0)


def test_large_steps_track_the_explicit_coarsening():
    """512 x 1024 torus at the coarsening parameters, from phi quenched into domains: ten times the
    explicit step, and 0.8 of the stabilised scheme's own stable step (about 13 times; the lattice-
    Boltzmann advection limit binds there), reach the same domain length (A / L_I) and phi as the
    explicit run at the same time."""
    nt, ns = 512, 1024
    p = dict(geometry=vlb.TORUS, R=2.0, r=1.0, n_theta=nt, n_phi=ns, dt=1.0, tau=0.6, M=2.5e-3, A=0.5,
             kappa=5e-4, advection=vlb.UW3, ch_mode=vlb.HYDRO)
    dt_exp = 0.9 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
    phi = inputs.quenched_noise(31, nt, ns, 6.0, 2.0)
    z = np.zeros_like(phi)
    dt_stab = 0.8 * vlb.vlb_max_stable_dt(vlb.make_params(**p, ch_stab=1))
    big = max(2, int(dt_stab / dt_exp))
    res = {}
    for stab, mult in ((0, 1), (1, 10), (1, big)):
        q = dict(p, dt=dt_exp * mult)
        s = vlb.Solver(vlb.make_params(**q, precision=vlb.FP32, ch_stab=stab))
        s.set_fields(np.ones_like(phi), z, z, phi)
        s.step(int(round(2000 / mult)))
        res[(stab, mult)] = (s.interface_length(), s.fields()[3], s.totals())
        s.close()
    L0, phi0, _ = res[(0, 1)]
    for key in ((1, 10), (1, big)):
        L, ph, tot = res[key]
        print(key, "L_I ratio", L / L0, "phi rel L2", rel_err(ph, phi0))
        assert abs(L / L0 - 1.0) < 0.02, (key, L / L0)
        assert rel_err(ph, phi0) < 0.05, key
        assert np.all(np.isfinite(tot))
