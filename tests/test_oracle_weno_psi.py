"""Pins of the oracle's WENO5-JS face value and of its free energy Psi.

Neither pin retypes the formula under test:

* WENO5-JS (Jiang & Shu 1996, the fidelity reading of the paper's finite-difference advection,
  Sec. 2.3): the face value is rebuilt from its *definition* -- candidate quadratics and the quartic
  that match cell averages, smoothness indicators as integrals of squared derivatives over the cell,
  linear weights solved from the requirement that the weighted candidates reproduce the quartic --
  with numpy polynomials and a linear solve; then fifth-order convergence of the derivative it
  implies, the essentially non-oscillatory choice of stencil next to a jump, the mirror image used
  for negative velocities, and the order of the semi-discrete advection term of the oracle's
  right-hand side.
* Psi (Eq. Landau): a relaxed flat interface carries the energy gamma per unit length with
  gamma = sqrt(8 kappa A / 9) (Eq. xi_gamma), so Psi of a band with two tanh interfaces must converge to
  gamma L_I, on a flat domain and on the torus (where the two interfaces are circles of different
  length 2 pi (R + r cos theta_i), App. A).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import polynomial as P

from oracle import vlb_oracle as O


# ------------------------------------------------------------------ WENO5-JS from its definition

def _fit_cell_averages(cells):
    """Coefficient maps: the polynomial of degree len(cells) - 1 whose averages over the unit cells
    centred at `cells` equal the data is sum_d data[d] * poly_d; returns the list of poly_d."""
    m = len(cells)
    # average of t^e over [c - 1/2, c + 1/2] = ((c + 1/2)^{e+1} - (c - 1/2)^{e+1}) / (e + 1)
    V = np.array([[((c + 0.5) ** (e + 1) - (c - 0.5) ** (e + 1)) / (e + 1) for e in range(m)] for c in cells])
    inv = np.linalg.inv(V)  # coefficients = inv @ data
    return [inv[:, d] for d in range(m)]


def _poly_of(data, cells):
    basis = _fit_cell_averages(cells)
    return sum(d * b for d, b in zip(data, basis))


def _smoothness(coef):
    """sum over l = 1, 2 of the integral over the cell [-1/2, 1/2] of (d^l p / dt^l)^2 (unit spacing)."""
    total = 0.0
    for l in (1, 2):
        dl = P.polyder(coef, l)
        sq = P.polyint(P.polymul(dl, dl))
        total += P.polyval(0.5, sq) - P.polyval(-0.5, sq)
    return total


def _linear_weights():
    """d_k such that sum_k d_k q_k = the quartic's face value for every data vector."""
    stencils = [(-2, -1, 0), (-1, 0, 1), (0, 1, 2)]
    rows = []
    for st in stencils:
        row = np.zeros(5)
        for d, b in zip(st, _fit_cell_averages(st)):
            row[d + 2] = P.polyval(0.5, b)
        rows.append(row)
    full = np.array([P.polyval(0.5, b) for b in _fit_cell_averages((-2, -1, 0, 1, 2))])
    d, *_ = np.linalg.lstsq(np.array(rows).T, full, rcond=None)
    assert np.allclose(np.array(rows).T @ d, full, atol=1e-14)
    return d


def _weno_from_definition(g, eps=1e-6):
    stencils = [(-2, -1, 0), (-1, 0, 1), (0, 1, 2)]
    d = _linear_weights()
    q, beta = [], []
    for st in stencils:
        coef = _poly_of([g[c + 2] for c in st], st)
        q.append(P.polyval(0.5, coef))
        beta.append(_smoothness(coef))
    alpha = [dk / (eps + bk) ** 2 for dk, bk in zip(d, beta)]
    return sum(a * qk for a, qk in zip(alpha, q)) / sum(alpha)


def test_weno_linear_weights_from_definition():
    np.testing.assert_allclose(_linear_weights(), [0.1, 0.6, 0.3], atol=1e-13)


@pytest.mark.parametrize("scale", [1e-4, 1e-2, 1.0, 30.0])
def test_weno_face_equals_definition(scale):
    rng = np.random.default_rng(int(scale * 1e4) + 1)
    for _ in range(50):
        g = scale * rng.normal(size=5)
        want = _weno_from_definition(g)
        got = O._weno5_face(*g)
        assert abs(got - want) <= 1e-12 * max(1.0, np.max(np.abs(g))), (g, got, want)


def test_weno_derivative_converges_at_fifth_order():
    """(F_{i+1/2} - F_{i-1/2}) / h -> f'(x_i) with error O(h^5) for a smooth f without critical points."""
    x0, errs = 0.3, []
    for h in (0.1, 0.05, 0.025, 0.0125):
        def face(xf):
            xi = xf - 0.5 * h
            return O._weno5_face(*[math.exp(xi + k * h) for k in (-2, -1, 0, 1, 2)])
        errs.append(abs((face(x0 + 0.5 * h) - face(x0 - 0.5 * h)) / h - math.exp(x0)))
    for a, b in zip(errs, errs[1:]):
        assert 26.0 < a / b < 36.0, errs
    assert errs[-1] < 1e-10


def test_weno_picks_the_smooth_stencil_next_to_a_jump():
    """Data 0 up to x_i, 1 from x_{i+2}: only the right candidate crosses the jump, and its weight
    must vanish (the face value stays 0 to ~1e-12) where the linear scheme undershoots by 3/60."""
    g = np.array([0.0, 0.0, 0.0, 0.0, 1.0])
    assert abs(O._weno5_face(*g)) < 1e-10
    lin = np.dot([2, -13, 47, 27, -3], g) / 60.0
    assert abs(lin + 0.05) < 1e-15
    # monotone data: the face value stays inside the data range
    rng = np.random.default_rng(11)
    for _ in range(200):
        g = np.sort(rng.uniform(-1, 1, 5))
        g[3:] += rng.uniform(0, 5)  # a jump between g2 and g3 or later
        g = np.sort(g)
        v = O._weno5_face(*g)
        assert g.min() - 1e-12 <= v <= g.max() + 1e-12


def test_negative_velocity_face_is_the_mirror_image():
    rng = np.random.default_rng(12)
    N = 17
    g = rng.normal(size=(N, 3))
    neg = O.face_values(g, 0, False, O.WENO5)
    pos_m = O.face_values(g[::-1], 0, True, O.WENO5)
    for i in range(N):
        np.testing.assert_allclose(neg[i], pos_m[(N - 2 - i) % N], rtol=0, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1])
def test_weno_advection_term_order(axis):
    """Flat domain, no collisions or forces: the right-hand side of every population is -v d_x f;
    the WENO5 flux form must approach it at (at least) fifth order."""
    errs = []
    for N in (16, 32, 64, 128):
        nt, ns = (N, 4) if axis == 0 else (4, N)
        p = O.Params(R=1.3, r=0.7, n_theta=nt, n_phi=ns, dt=1e-3, tau=np.inf, M=0.0, A=0.0, kappa=0.0,
                     geometry=O.FLAT, advection=O.WENO5, ch_mode=O.DIFFUSIVE)
        geo = O.Geometry(p)
        v, w = O.velocities(), O.weights()
        if axis == 0:
            x, ln = (np.arange(nt) * geo.dth)[:, None] * np.ones((1, ns)), p.r
        else:
            x, ln = np.ones((nt, 1)) * (np.arange(ns) * geo.dph)[None, :], p.R
        prof = 1.0 + 0.1 * np.sin(x) + 0.05 * np.cos(2 * x + 0.3)
        dprof = (0.1 * np.cos(x) - 0.1 * np.sin(2 * x + 0.3)) / ln
        f = (w[:, None, None, None] * w[None, :, None, None]) * prof[None, None]
        Lf, _ = O.rhs(f, np.zeros((nt, ns)), geo)
        e = 0.0
        for i in range(4):
            for j in range(4):
                vel = v[i] if axis == 0 else v[j]
                e = max(e, float(np.max(np.abs(Lf[i, j] + vel * w[i] * w[j] * dprof))))
        errs.append(e)
    for a, b in zip(errs[1:], errs[2:]):
        assert a / b > 26.0, errs
    assert errs[-1] < 1e-7


# ------------------------------------------------------------------ free energy (Eq. Landau, Eq. xi_gamma)

def _band_psi(nt, geom, A=0.5, kappa=5e-4, R=2.5, r=1.0, th1=math.pi / 4, th2=math.pi):
    p = O.Params(R=R, r=r, n_theta=nt, n_phi=4, dt=1e-3, tau=1.0, M=0.0, A=A, kappa=kappa, geometry=geom)
    geo = O.Geometry(p)
    th = geo.theta * np.ones((1, 4))
    xi = math.sqrt(kappa / A)
    # signed arc length r dtheta to the nearer interface, positive inside the band (th1, th2)
    d1 = (th - th1 + math.pi) % (2 * math.pi) - math.pi
    d2 = (th2 - th + math.pi) % (2 * math.pi) - math.pi
    d = r * np.where(np.abs(d1) < np.abs(d2), d1, d2)
    phi = np.tanh(d / (math.sqrt(2.0) * xi))  # the relaxed planar profile (Sec. 2.2)
    f = O.feq(np.ones_like(phi), 0 * phi, 0 * phi)
    psi = O.totals(f, phi, geo)[2]
    gamma = math.sqrt(8.0 * kappa * A / 9.0)
    if geom == O.TORUS:
        L = 2 * math.pi * (R + r * math.cos(th1)) + 2 * math.pi * (R + r * math.cos(th2))
    else:
        L = 2 * (2 * math.pi * R)
    return psi, gamma * L


@pytest.mark.parametrize("geom", [O.FLAT, O.TORUS])
def test_psi_of_relaxed_interfaces_is_gamma_times_length(geom):
    vals = [_band_psi(n, geom) for n in (512, 1024, 2048)]
    ref = vals[0][1]
    err = [v / ref - 1.0 for v, _ in vals]
    # central-difference gradients: second order, from below
    for a, b in zip(err, err[1:]):
        assert 3.6 < a / b < 4.4, err
    assert abs(err[-1]) < 1e-3
    # Richardson extrapolation removes the O(h^2) term; the torus keeps an O(xi^2 / (r R)) curvature
    # correction of the interface energy (~2e-5 here)
    ext = (4.0 * vals[2][0] - vals[1][0]) / 3.0
    assert abs(ext / ref - 1.0) < 1e-4, (ext, ref)
