"""Host-side analysis of azimuthally symmetric (stripe) profiles, for the physics checks.

TEST INFRASTRUCTURE, NOT PRODUCT CODE (same import rule as ``oracle.vlb_oracle``).

The paper does not define how the stripe centre theta_c is estimated (Sec. 3.3); the reading taken
here: the zero crossings of the varphi-averaged phi (linear interpolation between nodes) bound the
minority band, whose centre is the circular midpoint of the two crossings.
"""
from __future__ import annotations

import math

import numpy as np


def zero_crossings(prof: np.ndarray):
    """Angles (theta_q = q dtheta) where the periodic profile changes sign, linearly interpolated."""
    n = prof.size
    dth = 2.0 * math.pi / n
    out = []
    for q in range(n):
        a, b = prof[q], prof[(q + 1) % n]
        if a * b < 0.0:
            out.append((q + a / (a - b)) * dth)
    return out


def stripe_centre(prof: np.ndarray, inside_sign: float = -1.0):
    """(theta_c, width) of the single band where sign(phi) == inside_sign."""
    z = zero_crossings(prof)
    if len(z) != 2:
        raise ValueError(f"expected one band, found {len(z)} crossings")
    n = prof.size
    dth = 2.0 * math.pi / n
    a, b = z
    mid = 0.5 * (a + b)
    width = b - a
    q_mid = int(round(mid / dth)) % n
    if np.sign(prof[q_mid]) != inside_sign:  # the band is the other arc
        mid = (mid + math.pi) % (2.0 * math.pi)
        width = 2.0 * math.pi - width
    return mid, width


def band_pressure_jump(p: np.ndarray, theta_c: float, width: float):
    """p at the band centre minus p at the antipode (linear interpolation on the periodic grid)."""
    n = p.size
    dth = 2.0 * math.pi / n

    def at(theta):
        x = (theta % (2.0 * math.pi)) / dth
        q = int(math.floor(x))
        t = x - q
        return (1.0 - t) * p[q % n] + t * p[(q + 1) % n]

    return at(theta_c) - at(theta_c + math.pi)


def equal_area_drop_radius(R, r, xi, theta0, ref_theta0, ref_radius, n_theta=512, n_phi=1280):
    """R_0 of a drop (Eq. drop_init, phi = -1 inside, Euclidean distance) centred at (theta0, 0) with
    the same area as the drop (ref_theta0, ref_radius): the root of
    int (R + r cos theta) [phi_ref - phi(theta0, R_0)] dtheta dvarphi = 0 (Sec. 3.4), by bisection
    on a n_theta x n_phi midpoint grid."""
    from paper_1904_10070_gb300 import inputs
    th, _ = inputs.grid(n_theta, n_phi)
    wgt = R + r * np.cos(th)
    target = np.sum(wgt * inputs.drop_phi(R, r, n_theta, n_phi, ref_theta0, ref_radius, xi, inside=-1.0))
    lo, hi = 0.25 * ref_radius, 4.0 * ref_radius
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        # a larger drop holds more of the phi = -1 phase: the weighted integral falls as R_0 grows
        if np.sum(wgt * inputs.drop_phi(R, r, n_theta, n_phi, theta0, mid, xi, inside=-1.0)) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
