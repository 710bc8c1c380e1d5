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


def stripe_normal_pressure(n, phi, r: float, R: float, A: float, kappa: float, geometry: int = 0) -> np.ndarray:
    """P^{theta theta} of an azimuthally symmetric profile (n and phi of theta alone, one value per row):
    n + p_binary(phi) - kappa phi Delta phi + (kappa / 2) (d_theta phi / r)^2, with k_B T = 1.

    The force of Eq. pbin, n F = -grad p_binary + kappa phi grad Delta phi, is minus the divergence of
    the Korteweg stress (p_binary - kappa phi Delta phi - kappa |grad phi|^2 / 2) delta + kappa grad phi
    grad phi; for a profile of theta alone its theta-theta component is the expression above.  Where
    grad phi = 0 (the centre of a band, the bulk) it reduces to n + p_binary - kappa phi Delta phi, and
    in the bulk to the pressure n + p_binary of Sec. 3.2.  Delta is the Laplace-Beltrami operator of
    App. A in the scheme's conservative second-order form; d_theta is a central difference."""
    n = np.asarray(n, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    nt = phi.size
    dth = 2.0 * math.pi / nt
    th = np.arange(nt) * dth
    a = r / R if geometry == 0 else 0.0
    J = 1.0 + a * np.cos(th)
    Jp = 1.0 + a * np.cos(th + 0.5 * dth)
    Jm = 1.0 + a * np.cos(th - 0.5 * dth)
    up, dn = np.roll(phi, -1), np.roll(phi, 1)
    lap = (Jp * (up - phi) - Jm * (phi - dn)) / (r * r * J * dth * dth)
    dphi = (up - dn) / (2.0 * r * dth)
    pb = A * (-0.5 * phi ** 2 + 0.75 * phi ** 4)
    return n + pb - kappa * phi * lap + 0.5 * kappa * dphi ** 2
