"""Closed-form predictions printed in arXiv:1904.10070, used as pins for the oracle and the GPU path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE (same import rule as ``oracle.vlb_oracle``).

Notation: torus radii R > r, a = r/R; a stripe of angular width dth centred on theta_c.
"""
from __future__ import annotations

import math


def xi0(kappa, A):
    """Interface width xi_0 = sqrt(kappa/A)  (Eq. xi_gamma)."""
    return math.sqrt(kappa / A)


def surface_tension(kappa, A):
    """gamma = sqrt(8 kappa A / 9)  (Eq. xi_gamma)."""
    return math.sqrt(8.0 * kappa * A / 9.0)


def stripe_area(R, r, theta_c, dth):
    """Delta A = 2 pi r R [dth + 2 a sin(dth/2) cos theta_c]  (Eq. stripe_area)."""
    a = r / R
    return 2.0 * math.pi * r * R * (dth + 2.0 * a * math.sin(0.5 * dth) * math.cos(theta_c))


def critical_area(R, r):
    """Delta A_crit = 4 pi r R (arccos a - a sqrt(1 - a^2))  (Eq. stripe_dA_crit)."""
    a = r / R
    return 4.0 * math.pi * r * R * (math.acos(a) - a * math.sqrt(1.0 - a * a))


def critical_width(R, r):
    """Delta theta_crit = 2 arccos(a)  (Sec. 3.1, text above Eq. stripe_dA_crit)."""
    return 2.0 * math.acos(r / R)


def interface_total(R, r, theta_c, dth):
    """l_total = 4 pi R (1 + a cos theta_c cos(dth/2))  (Eq. stripe_ltot)."""
    a = r / R
    return 4.0 * math.pi * R * (1.0 + a * math.cos(theta_c) * math.cos(0.5 * dth))


def width_for_area(R, r, theta_c, area, lo=1e-9, hi=2.0 * math.pi - 1e-9):
    """Invert Eq. stripe_area for the width at fixed centre (bisection; the area is monotone in dth)."""
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if stripe_area(R, r, theta_c, mid) < area:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def equilibrium(R, r, area):
    """Equilibrium (theta_c^eq, dth_eq) of a stripe of given area (Eqs. minimaring, stripe_thceq).

    Sub-critical areas sit at theta_c = pi; super-critical ones at the root of
    a cos theta_c + cos(dth/2) = 0 with theta_c < pi (the mirror root pi + ... is equivalent).
    """
    a = r / R
    if area <= critical_area(R, r):
        return math.pi, width_for_area(R, r, math.pi, area)
    # on the super-critical branch cos theta_c = -cos(dth/2)/a; area(dth) along the branch is monotone
    def area_on_branch(dth):
        c = -math.cos(0.5 * dth) / a
        return 2.0 * math.pi * r * R * (dth + 2.0 * a * math.sin(0.5 * dth) * c)
    lo, hi = critical_width(R, r), 2.0 * math.pi - 1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if area_on_branch(mid) < area:
            lo = mid
        else:
            hi = mid
    dth = 0.5 * (lo + hi)
    theta_c = math.pi - math.acos(min(1.0, math.cos(0.5 * dth) / a))
    return theta_c, dth


def laplace_pressure(R, r, kappa, A, theta_c, dth):
    """Delta p = -(gamma/R) cos theta_c sin(dth/2) / (1 + a cos theta_c cos(dth/2))  (Eq. stripe_laplace_gen)."""
    a = r / R
    g = surface_tension(kappa, A)
    return -g / R * math.cos(theta_c) * math.sin(0.5 * dth) / (1.0 + a * math.cos(theta_c) * math.cos(0.5 * dth))


def laplace_pressure_eq(R, r, kappa, A, dth_eq, subcritical: bool):
    """The two equilibrium branches of Eq. stripe_laplace_eq."""
    a = r / R
    g = surface_tension(kappa, A)
    if subcritical:
        return g / R * math.sin(0.5 * dth_eq) / (1.0 - a * math.cos(0.5 * dth_eq))
    return g / r / math.tan(0.5 * dth_eq)


def stripe_offset(R, r, kappa, A, theta_c, dth):
    """phi_0 = xi_0/(3 R sqrt 2) cos theta_c sin(dth/2)/(1 + a cos theta_c cos(dth/2))  (Eq. stripe_phi0)."""
    a = r / R
    x = xi0(kappa, A)
    return x / (3.0 * R * math.sqrt(2.0)) * math.cos(theta_c) * math.sin(0.5 * dth) / (
        1.0 + a * math.cos(theta_c) * math.cos(0.5 * dth))


def alpha_nu(R, r, nu):
    """Viscous damping rate alpha_nu = nu / (R^2 - r^2)  (Eq. stripe_alphanu)."""
    return nu / (R * R - r * r)


def omega0_subcritical(R, r, kappa, A, dth_eq, n=1.0, m=1.0):
    """omega_0 for a stripe equilibrating at theta_c = pi  (Eq. stripe_hydro_omega0_pi)."""
    a = r / R
    g = surface_tension(kappa, A)
    c = math.cos(0.5 * dth_eq)
    w2 = g * math.sqrt(1.0 - a * a) / (math.pi * r * r * R * n * m) * (c - a) / (1.0 - a * c) ** 3
    return math.sqrt(w2)


def omega0_supercritical(R, r, kappa, A, theta_c_eq, dth_eq, n=1.0, m=1.0):
    """omega_0 for a stripe equilibrating off theta = pi  (Eq. stripe_hydro_omega0_npi)."""
    a = r / R
    g = surface_tension(kappa, A)
    w2 = 2.0 * g / (math.pi * r * R * R * n * m * (1.0 - a * a) ** 1.5) * (
        math.sin(theta_c_eq) / math.sin(0.5 * dth_eq)) ** 2
    return math.sqrt(w2)
