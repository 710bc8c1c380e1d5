"""Pins of the oracle's structure-factor length L_S = 2 pi sum S / sum |k| S (the Fourier measure of
the coarsening domain size beside Sec. 4.1's L_d = A / L_I).

Pinned against: the closed form of a single Fourier mode and of a two-mode mixture, a structure
factor summed with explicit index loops (a brute-force DFT, not the library FFT), the aliasing of a
frequency above N/2 to its negative, invariance under a lattice translation, and indifference to
the mean of phi."""
import cmath
import math

import numpy as np
import pytest

from oracle import vlb_oracle as O


def _geo(nt, ns, geometry=O.TORUS, R=2.0, r=1.0):
    return O.Geometry(O.Params(R=R, r=r, n_theta=nt, n_phi=ns, dt=1e-3, tau=1.0, M=1.0, A=1.0, kappa=1.0,
                               geometry=geometry))


def _grid(geo, nt, ns):
    th = geo.theta * np.ones((1, ns))
    ph = np.arange(ns)[None, :] * geo.dph * np.ones((nt, 1))
    return th, ph


@pytest.mark.parametrize("geometry", [O.TORUS, O.FLAT])
@pytest.mark.parametrize("m,n", [(1, 0), (0, 3), (3, 5), (-2, 7), (8, 0), (4, 16)])
def test_single_mode_closed_form(geometry, m, n):
    nt, ns = 16, 32
    geo = _geo(nt, ns, geometry)
    th, ph = _grid(geo, nt, ns)
    phi = 0.3 + 0.8 * np.cos(m * th + n * ph + 0.4)
    want = 2 * math.pi / math.hypot(m / geo.p.r, n / geo.p.R)
    assert O.structure_length(phi, geo) == pytest.approx(want, rel=1e-12)


def test_two_mode_mixture_closed_form():
    """Amplitudes a, b on modes k1, k2: L_S = 2 pi (a^2 + b^2) / (a^2 |k1| + b^2 |k2|)."""
    nt, ns = 16, 24
    geo = _geo(nt, ns, R=3.0, r=0.7)
    th, ph = _grid(geo, nt, ns)
    a, b = 0.9, 0.35
    phi = a * np.sin(2 * th + ph) + b * np.cos(5 * th - 7 * ph)
    k1 = math.hypot(2 / 0.7, 1 / 3.0)
    k2 = math.hypot(5 / 0.7, 7 / 3.0)
    want = 2 * math.pi * (a * a + b * b) / (a * a * k1 + b * b * k2)
    assert O.structure_length(phi, geo) == pytest.approx(want, rel=1e-12)


def test_structure_factor_by_explicit_loops():
    nt, ns = 6, 10
    rng = np.random.default_rng(31)
    phi = rng.uniform(-1, 1, (nt, ns))
    S = O.structure_factor(phi)
    geo = _geo(nt, ns, R=2.5, r=1.0)
    num = den = 0.0
    for m in range(nt):
        for n in range(ns):
            acc = 0j
            for q in range(nt):
                for s in range(ns):
                    acc += phi[q, s] * cmath.exp(-2j * math.pi * (m * q / nt + n * s / ns))
            assert abs(S[m, n] - abs(acc) ** 2) <= 1e-10
            if m == 0 and n == 0:
                continue
            ms = m if m <= nt // 2 else m - nt
            ns_ = n if n <= ns // 2 else n - ns
            k = math.hypot(ms / 1.0, ns_ / 2.5)
            num += abs(acc) ** 2
            den += k * abs(acc) ** 2
    assert O.structure_length(phi, geo) == pytest.approx(2 * math.pi * num / den, rel=1e-12)


def test_invariances():
    nt, ns = 32, 64
    geo = _geo(nt, ns)
    rng = np.random.default_rng(32)
    phi = np.tanh(3 * rng.uniform(-1, 1, (nt, ns)))
    L = O.structure_length(phi, geo)
    assert O.structure_length(np.roll(phi, (5, -11), axis=(0, 1)), geo) == pytest.approx(L, rel=1e-12)
    assert O.structure_length(phi + 0.37, geo) == pytest.approx(L, rel=1e-12)
    assert O.structure_length(-2.0 * phi, geo) == pytest.approx(L, rel=1e-12)
    # frequencies above N/2 are the negative ones: mode N_theta - 1 along theta is mode -1
    th, ph = _grid(geo, nt, ns)
    assert O.structure_length(np.cos((nt - 1) * th), geo) == pytest.approx(2 * math.pi * geo.p.r, rel=1e-12)


def test_uniform_phi_has_infinite_length():
    geo = _geo(8, 8)
    assert O.structure_length(np.full((8, 8), -0.4), geo) == math.inf
