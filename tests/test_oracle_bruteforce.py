"""Brute-force check of the vectorised oracle on tiny grids.

An independent node-by-node restatement of one SSP-RK3 step (Eq. boltz_tor with BGK, Eq. CH,
Eq. mu, Eq. pbin) in plain Python loops, using the velocity kernels as PRINTED in the paper
(Sec. 2.3) rather than the oracle's Hermite sums, with explicit periodic index arithmetic
instead of array shifts.
"""
import math

import numpy as np
import pytest

from oracle import vlb_oracle as O
from tests.test_oracle_pins import _printed


def _face_pos(g, eps=1e-6, weno=False):
    """Face value between g[2] and g[3] of a five-point window g[0..4], upwind from the left."""
    if not weno:
        return (-g[1] + 5 * g[2] + 2 * g[3]) / 6
    c = [(2 * g[0] - 7 * g[1] + 11 * g[2]) / 6, (-g[1] + 5 * g[2] + 2 * g[3]) / 6,
         (2 * g[2] + 5 * g[3] - g[4]) / 6]
    b = [13 / 12 * (g[0] - 2 * g[1] + g[2]) ** 2 + 0.25 * (g[0] - 4 * g[1] + 3 * g[2]) ** 2,
         13 / 12 * (g[1] - 2 * g[2] + g[3]) ** 2 + 0.25 * (g[1] - g[3]) ** 2,
         13 / 12 * (g[2] - 2 * g[3] + g[4]) ** 2 + 0.25 * (3 * g[2] - 4 * g[3] + g[4]) ** 2]
    al = [d / (eps + bb) ** 2 for d, bb in zip((0.1, 0.6, 0.3), b)]
    return sum(a * cc for a, cc in zip(al, c)) / sum(al)


def _face(get, i, vel, weno):
    """Upwind face value at i+1/2; get(k) returns the value at periodic index k."""
    if vel > 0:
        return _face_pos([get(i + d) for d in (-2, -1, 0, 1, 2)], weno=weno)
    return _face_pos([get(i + d) for d in (3, 2, 1, 0, -1)], weno=weno)


def _rhs_loops(f, phi, p):
    pr = _printed()
    v, w, K, Kt = pr["v"], pr["w"], pr["K"], pr["Kt"]
    nq, ns = phi.shape
    dth, dph = 2 * math.pi / nq, 2 * math.pi / ns
    a = p.r / p.R if p.geometry == O.TORUS else 0.0
    J = lambda q: 1 + a * math.cos(q * dth)  # noqa: E731
    Jf = lambda x: 1 + a * math.cos(x)  # noqa: E731
    Gam = lambda q: (math.sin(q * dth) / (p.R * J(q))) if p.geometry == O.TORUS else 0.0  # noqa: E731
    P = lambda q, s: phi[q % nq, s % ns]  # noqa: E731

    def lap(x, q, s):
        return ((Jf((q + 0.5) * dth) * (x(q + 1, s) - x(q, s)) - Jf((q - 0.5) * dth) * (x(q, s) - x(q - 1, s)))
                / (p.r ** 2 * J(q) * dth ** 2)
                + (x(q, s + 1) - 2 * x(q, s) + x(q, s - 1)) / (p.R ** 2 * J(q) ** 2 * dph ** 2))

    mu = np.zeros((nq, ns))
    n = np.zeros((nq, ns)); ut = np.zeros((nq, ns)); up = np.zeros((nq, ns))
    for q in range(nq):
        for s in range(ns):
            mu[q, s] = -p.A * P(q, s) * (1 - P(q, s) ** 2) - p.kappa * lap(P, q, s)
            n[q, s] = sum(f[i, j, q, s] for i in range(4) for j in range(4))
            ut[q, s] = sum(v[i] * f[i, j, q, s] for i in range(4) for j in range(4)) / n[q, s]
            up[q, s] = sum(v[j] * f[i, j, q, s] for i in range(4) for j in range(4)) / n[q, s]
    MU = lambda q, s: mu[q % nq, s % ns]  # noqa: E731
    weno = p.advection == O.WENO5
    Lf = np.zeros_like(f)
    Lp = np.zeros_like(phi)
    for q in range(nq):
        for s in range(ns):
            if p.ch_mode == O.HYDRO:
                Ft = -P(q, s) / n[q, s] * (MU(q + 1, s) - MU(q - 1, s)) / (2 * p.r * dth)
                Fp = -P(q, s) / n[q, s] * (MU(q, s + 1) - MU(q, s - 1)) / (2 * p.R * J(q) * dph)
            else:
                Ft = Fp = 0.0
            usq = ut[q, s] ** 2 + up[q, s] ** 2
            for i in range(4):
                for j in range(4):
                    G = lambda k: J(k) * f[i, j, k % nq, s]  # noqa: E731
                    H = lambda k: f[i, j, q, k % ns]  # noqa: E731
                    adv = (-v[i] / (p.r * J(q) * dth) * (_face(G, q, v[i], weno) - _face(G, q - 1, v[i], weno))
                           - v[j] / (p.R * J(q) * dph) * (_face(H, s, v[j], weno) - _face(H, s - 1, v[j], weno)))
                    dvt = sum(K[i, m] * f[m, j, q, s] for m in range(4))
                    dvp = sum(K[j, m] * f[i, m, q, s] for m in range(4))
                    dfvp = sum(Kt[j, m] * f[i, m, q, s] for m in range(4))
                    xi = v[i] * ut[q, s] + v[j] * up[q, s]
                    fe = n[q, s] * w[i] * w[j] * (1 + xi + 0.5 * (xi * xi - usq) + xi * (xi * xi - 3 * usq) / 6)
                    Lf[i, j, q, s] = (adv - Ft * dvt - Fp * dvp + Gam(q) * (v[j] ** 2 * dvt - v[i] * dfvp)
                                      - (f[i, j, q, s] - fe) / p.tau)
            lp = p.M * lap(MU, q, s)
            if p.ch_mode == O.HYDRO:
                X = lambda k, l: J(k) * ut[k % nq, l % ns] * phi[k % nq, l % ns]  # noqa: E731
                Y = lambda k, l: up[k % nq, l % ns] * phi[k % nq, l % ns]  # noqa: E731
                lp -= (0.5 * (X(q, s) + X(q + 1, s)) - 0.5 * (X(q - 1, s) + X(q, s))) / (p.r * J(q) * dth)
                lp -= (0.5 * (Y(q, s) + Y(q, s + 1)) - 0.5 * (Y(q, s - 1) + Y(q, s))) / (p.R * J(q) * dph)
            Lp[q, s] = lp
    return Lf, Lp


def _step_loops(f, phi, p):
    L1, M1 = _rhs_loops(f, phi, p)
    f1, p1 = f + p.dt * L1, phi + p.dt * M1
    L2, M2 = _rhs_loops(f1, p1, p)
    f2, p2 = 0.75 * f + 0.25 * (f1 + p.dt * L2), 0.75 * phi + 0.25 * (p1 + p.dt * M2)
    L3, M3 = _rhs_loops(f2, p2, p)
    return f / 3 + 2 / 3 * (f2 + p.dt * L3), phi / 3 + 2 / 3 * (p2 + p.dt * M3)


@pytest.mark.parametrize("nq,ns", [(5, 7), (6, 1)])
@pytest.mark.parametrize("adv", [O.UW3, O.WENO5])
@pytest.mark.parametrize("geom,mode", [(O.TORUS, O.HYDRO), (O.FLAT, O.HYDRO), (O.TORUS, O.DIFFUSIVE)])
def test_vectorised_oracle_equals_node_loops(nq, ns, adv, geom, mode):
    p = O.Params(R=2.2, r=0.9, n_theta=nq, n_phi=ns, dt=4e-3, tau=0.3, M=0.07, A=0.4, kappa=0.03,
                 geometry=geom, advection=adv, ch_mode=mode)
    rng = np.random.default_rng(11)
    n = 1.0 + 0.1 * rng.uniform(-1, 1, (nq, ns))
    f = O.feq(n, 0.05 * rng.uniform(-1, 1, (nq, ns)), 0.05 * rng.uniform(-1, 1, (nq, ns)))
    f = f * (1 + 0.02 * rng.uniform(-1, 1, f.shape))
    phi = rng.uniform(-1, 1, (nq, ns))
    geo = O.Geometry(p)
    fa, pa = f, phi
    fb, pb = f, phi
    for _ in range(2):
        fa, pa = O.step(fa, pa, geo)
        fb, pb = _step_loops(fb, pb, p)
    np.testing.assert_allclose(fa, fb, rtol=0, atol=1e-13 * np.max(np.abs(fb)))
    np.testing.assert_allclose(pa, pb, rtol=0, atol=1e-13 * np.max(np.abs(pb)))


@pytest.mark.parametrize("adv", [O.UW3, O.WENO5])
def test_step_window_equals_full_grid_step(adv):
    """The node-by-node evaluation used at full size (a periodic window cut out around the node)
    gives the full-grid step at that node, including nodes on the wrap-around seams."""
    nq, ns = 31, 29
    p = O.Params(R=2.2, r=0.9, n_theta=nq, n_phi=ns, dt=2e-3, tau=0.3, M=0.07, A=0.4, kappa=0.03,
                 advection=adv)
    rng = np.random.default_rng(13)
    n = 1.0 + 0.1 * rng.uniform(-1, 1, (nq, ns))
    f = O.feq(n, 0.05 * rng.uniform(-1, 1, (nq, ns)), 0.05 * rng.uniform(-1, 1, (nq, ns)))
    phi = np.tanh(2 * rng.uniform(-1, 1, (nq, ns)))
    f1, p1 = O.step(f, phi, O.Geometry(p))
    for q, s in [(0, 0), (nq - 1, ns - 1), (15, 0), (0, 14), (7, 22)]:
        fw, pw = O.step_window(f, phi, p, q, s)
        np.testing.assert_allclose(fw, f1[:, :, q, s], rtol=0, atol=1e-14 * np.max(np.abs(f1)))
        assert abs(pw - p1[q, s]) <= 1e-14
