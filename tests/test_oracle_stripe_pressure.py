"""Pins of oracle.analysis.stripe_normal_pressure, the theta-theta component of the pressure tensor
whose divergence is the force of Eq. pbin (used for the Laplace pressure of narrow stripes, whose
interface tails overlap at the band centre).

Pinned against: the bulk pressure n + p_binary of Sec. 3.2 on a uniform state; and the mechanical
equilibrium of a flat interface, whose normal pressure is uniform across the tanh profile
phi = tanh(x / (sqrt 2 xi)) (the continuum identity p_binary - kappa phi phi'' + kappa phi'^2 / 2 = A / 4),
to second order in the grid spacing -- where the bulk formula alone is off by A / 4 at the interface."""
import math

import numpy as np
import pytest

from oracle import analysis as AN
from oracle import vlb_oracle as O


def test_uniform_state_is_the_bulk_pressure():
    n = np.full(64, 1.3)
    for phi0 in (-1.0, -0.2, 0.7):
        phi = np.full(64, phi0)
        p = AN.stripe_normal_pressure(n, phi, 1.0, 2.5, 0.5, 1e-3)
        np.testing.assert_allclose(p, O.pressure(n, phi, 0.5), rtol=0, atol=1e-15)


@pytest.mark.parametrize("nt", [1024, 2048])
def test_flat_interface_has_uniform_normal_pressure(nt):
    A, kappa, r = 0.5, 1.25e-3, 1.0
    xi = math.sqrt(kappa / A)
    th = np.arange(nt) * 2 * math.pi / nt
    x = r * (th - math.pi)  # arc length from the band centre
    half = 0.5 * math.pi * r
    phi = np.tanh((half - np.abs(x)) / (math.sqrt(2) * xi))  # a wide band: tails meet at e^-44
    n = np.ones(nt)
    p = AN.stripe_normal_pressure(n, phi, r, 1.0, A, kappa, geometry=O.FLAT)
    dev = np.max(np.abs(p - (1.0 + A / 4)))
    bulk_dev = np.max(np.abs(O.pressure(n, phi, A) - (1.0 + A / 4)))
    h = 2 * math.pi * r / nt
    assert bulk_dev > 0.2 * A
    assert dev < 0.2 * A * (h / xi) ** 2, (dev, (h / xi) ** 2)


def test_second_order_convergence_of_the_flat_identity():
    A, kappa = 0.5, 1.25e-3
    xi = math.sqrt(kappa / A)
    devs = []
    for nt in (512, 1024, 2048):
        th = np.arange(nt) * 2 * math.pi / nt
        x = th - math.pi
        phi = np.tanh((0.5 * math.pi - np.abs(x)) / (math.sqrt(2) * xi))
        p = AN.stripe_normal_pressure(np.ones(nt), phi, 1.0, 1.0, A, kappa, geometry=O.FLAT)
        devs.append(np.max(np.abs(p - (1.0 + A / 4))))
    for a, b in zip(devs, devs[1:]):
        assert 3.2 < a / b < 4.8, devs
