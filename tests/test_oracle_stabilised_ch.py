"""Pins of the oracle's stabilised semi-implicit Cahn-Hilliard step (not in the paper: it lifts the
explicit dt ~ h^4 / (M kappa) limit of the finite-difference Cahn-Hilliard equation, Eq. CH).

The step advances phi' = P L_phi with P = J^{-1} (I + dt M kappa D^2)^{-1} J, D the constant-coefficient
periodic five-point Laplacian at the finest grid spacings.  Pinned against what the mathematics fixes:
a dense-matrix construction of P from explicit periodic index loops, exact conservation of
sum J phi (the integral of phi sqrt(g), App. A), the closed-form SSP-RK3 amplification of a Fourier
mode of the linear equation, stability far beyond the explicit limit where the explicit step blows
up, and first-order convergence to the explicit solution as dt shrinks."""
import math

import numpy as np
import pytest

from oracle import vlb_oracle as O


def _params(nt, ns, dt, geometry=O.TORUS, stab=1, **kw):
    base = dict(R=2.5, r=1.0, n_theta=nt, n_phi=ns, dt=dt, tau=0.3, M=0.5, A=0.3, kappa=0.05, geometry=geometry,
                ch_stab=stab)
    base.update(kw)
    return O.Params(**base)


def _dense_stabiliser(p):
    """The matrix J^{-1} (I + dt M kappa D^2)^{-1} J built node by node."""
    nt, ns = p.n_theta, p.n_phi
    n = nt * ns
    dth, dph = 2 * math.pi / nt, 2 * math.pi / ns
    h_t = p.r * dth
    h_p = ((p.R - p.r) if p.geometry == O.TORUS else p.R) * dph
    D = np.zeros((n, n))
    for q in range(nt):
        for s in range(ns):
            i = q * ns + s
            D[i, i] -= 2 / h_t ** 2 + 2 / h_p ** 2
            D[i, ((q + 1) % nt) * ns + s] += 1 / h_t ** 2
            D[i, ((q - 1) % nt) * ns + s] += 1 / h_t ** 2
            D[i, q * ns + (s + 1) % ns] += 1 / h_p ** 2
            D[i, q * ns + (s - 1) % ns] += 1 / h_p ** 2
    a = p.r / p.R if p.geometry == O.TORUS else 0.0
    J = np.repeat(1 + a * np.cos(np.arange(nt) * dth), ns)
    inner = np.linalg.inv(np.eye(n) + p.dt * p.M * p.kappa * D @ D)
    return np.diag(1 / J) @ inner @ np.diag(J)


@pytest.mark.parametrize("geometry", [O.TORUS, O.FLAT])
def test_stabiliser_equals_its_dense_matrix(geometry):
    p = _params(6, 10, 3e-3, geometry=geometry)
    geo = O.Geometry(p)
    rng = np.random.default_rng(21)
    x = rng.normal(size=(6, 10))
    want = (_dense_stabiliser(p) @ x.reshape(-1)).reshape(6, 10)
    np.testing.assert_allclose(O.stabiliser(x, geo), want, rtol=0, atol=1e-12)


def test_stabiliser_conserves_the_weighted_sum_and_damps():
    p = _params(16, 24, 5e-2)
    geo = O.Geometry(p)
    rng = np.random.default_rng(22)
    x = rng.normal(size=(16, 24))
    y = O.stabiliser(x, geo)
    assert abs(np.sum(geo.J * y) - np.sum(geo.J * x)) <= 1e-12 * np.sum(np.abs(geo.J * x))
    # a contraction of J x in the Euclidean norm, the identity on constants
    assert np.linalg.norm(geo.J * y) <= np.linalg.norm(geo.J * x)
    np.testing.assert_allclose(O.stabiliser(np.full((16, 24), 0.7) / geo.J, geo), np.broadcast_to(0.7 / geo.J, (16, 24)),
                               rtol=1e-13)


def test_linear_mode_follows_the_closed_form_amplification():
    """Flat domain, A = 0, no advection or force: phi' = P M Delta(-kappa Delta phi).  A Fourier mode is
    an eigenvector of Delta_h (= D on the flat grid) with eigenvalue -sqrt(lambda), so one step multiplies
    it by R(z) = 1 + z + z^2/2 + z^3/6 with z = -dt M kappa lambda / (1 + dt M kappa lambda), also at
    dt twenty times the explicit limit (z -> -1)."""
    nt, ns, kq, ks = 12, 16, 3, 5
    for dt in (1e-4, 2e-2):
        p = _params(nt, ns, dt, geometry=O.FLAT, A=0.0, ch_mode=O.DIFFUSIVE)
        geo = O.Geometry(p)
        th = geo.theta * np.ones((1, ns))
        ph = np.arange(ns)[None, :] * geo.dph * np.ones((nt, 1))
        phi0 = 0.1 * np.cos(kq * th + ks * ph)
        n = np.ones((nt, ns))
        f = O.feq(n, 0 * n, 0 * n)
        f1, phi1 = O.run(f, phi0, geo, 10)
        h_t, h_p = p.r * geo.dth, p.R * geo.dph
        lam = (4 / h_t ** 2 * math.sin(math.pi * kq / nt) ** 2 + 4 / h_p ** 2 * math.sin(math.pi * ks / ns) ** 2) ** 2
        s = dt * p.M * p.kappa * lam
        z = -s / (1 + s)
        G = 1 + z + z * z / 2 + z ** 3 / 6
        np.testing.assert_allclose(phi1, G ** 10 * phi0, rtol=0, atol=1e-13)


def _noisy_state(p, seed):
    geo = O.Geometry(p)
    rng = np.random.default_rng(seed)
    phi = np.tanh(2.0 * rng.uniform(-1, 1, (p.n_theta, p.n_phi)))
    n = 1.0 + 0.02 * rng.uniform(-1, 1, phi.shape)
    return O.feq(n, 0 * n, 0 * n), phi, geo


def test_stable_far_beyond_the_explicit_limit_and_conservative():
    # explicit Cahn-Hilliard limit of this grid ~1.2e-3; the step below is 17 times larger and still
    # under the lattice-Boltzmann advection limit (~3.6e-2)
    dt = 2e-2
    p = _params(32, 64, dt)
    f, phi, geo = _noisy_state(p, 23)
    t0 = O.totals(f, phi, geo)
    fs, ps = O.run(f, phi, geo, 60)
    t1 = O.totals(fs, ps, geo)
    assert np.all(np.isfinite(fs)) and np.max(np.abs(ps)) < 1.2
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    assert abs(t1[1] - t0[1]) <= 1e-12 * np.sum(np.abs(phi) * geo.dA)
    assert t1[2] < t0[2]  # the free energy falls (phase separation from noise)
    # the explicit step at the same dt blows up
    pe = _params(32, 64, dt, stab=0)
    with np.errstate(all="ignore"):
        fe, pe_ = O.run(f, phi, O.Geometry(pe), 60)
    assert not (np.all(np.isfinite(pe_)) and np.max(np.abs(pe_)) < 1.2)


def test_first_order_convergence_to_the_explicit_solution():
    """At a fixed time the stabilised solution approaches the (converged) explicit one as O(dt)."""
    T = 0.02
    p_ref = _params(16, 32, T / 400, stab=0)
    f, phi, _ = _noisy_state(p_ref, 24)
    _, ref = O.run(f, phi, O.Geometry(p_ref), 400)
    errs = []
    for nsteps in (10, 20, 40):
        p = _params(16, 32, T / nsteps)
        _, ps = O.run(f, phi, O.Geometry(p), nsteps)
        errs.append(np.max(np.abs(ps - ref)))
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.5, errs
