"""Seeded synthetic inputs and workload recipes shared by the tests, the bench and the oracle checks.

This module builds initial fields only; it contains none of the time-step arithmetic, so the
CUDA library and the CPU oracle each receive identical arrays from here and nothing else.

Initial conditions follow arXiv:1904.10070: the drop profile (Eq. drop_init, Euclidean 3-D
distance to the centre), the stripe profile with its Laplace offset (Eqs. stripe_tanh and
stripe_phi0), and the noisy mixture phi = phi_bar + delta phi (Eq. phirand).

Noise is counter-based so that any (seed, q, s) gives the same value on every machine:
SplitMix64 (Steele, Lea & Flood 2014) applied to a key built from the seed and the node, and
the top 53 bits mapped to [0, 1).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n_theta: int, n_phi: int) -> np.ndarray:
    """u[q, s] in [0, 1): SplitMix64 of key = mix(seed) + (q * 2^32 + s + 1) * golden."""
    q = np.arange(n_theta, dtype=np.uint64)[:, None]
    s = np.arange(n_phi, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        base = _mix64(np.array([seed], dtype=np.uint64) * _GOLDEN + _GOLDEN)[0]
        key = base + ((q << np.uint64(32)) + s + np.uint64(1)) * _GOLDEN
    z = _mix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def noise(seed: int, n_theta: int, n_phi: int, amplitude: float) -> np.ndarray:
    """Uniform noise in (-amplitude, amplitude) (Eq. phirand)."""
    return amplitude * (2.0 * uniform01(seed, n_theta, n_phi) - 1.0)


def quenched_noise(seed: int, n_theta: int, n_phi: int, corr: float, width: float) -> np.ndarray:
    """Seeded noise quenched into domains: uniform noise (seed) smoothed by a periodic Gaussian filter
    of `corr` grid cells (applied in Fourier space), scaled to zero mean and unit variance, then
    phi = tanh(G corr / width), so that domains a few `corr` across are separated by tanh walls about
    `width` cells wide.  A start in the coarsening regime of the phase-separation runs (Sec. 4)."""
    u = noise(seed, n_theta, n_phi, 1.0)
    fq = np.fft.fftfreq(n_theta)[:, None]
    fs = np.fft.fftfreq(n_phi)[None, :]
    g = np.fft.ifft2(np.fft.fft2(u) * np.exp(-2.0 * (math.pi * corr) ** 2 * (fq ** 2 + fs ** 2))).real
    g = (g - g.mean()) / g.std()
    return np.tanh(g * corr / width)


def grid(n_theta: int, n_phi: int):
    """Node angles theta_q = q dtheta, varphi_s = s dvarphi on the periodic grid."""
    th = np.arange(n_theta) * (2.0 * math.pi / n_theta)
    ph = np.arange(n_phi) * (2.0 * math.pi / n_phi)
    return np.meshgrid(th, ph, indexing="ij")


def embed(R: float, r: float, theta, varphi):
    """Torus embedding in R^3 (App. A, Eq. torus)."""
    rho = R + r * np.cos(theta)
    return rho * np.cos(varphi), rho * np.sin(varphi), r * np.sin(theta)


def drop_phi(R, r, n_theta, n_phi, theta0, radius, xi, inside=+1.0, varphi0=0.0):
    """Drop of radius `radius` centred on (theta0, varphi0): Eq. drop_init with Euclidean distance.

    The paper's profile is tanh((d - R_0)/(xi sqrt 2)), i.e. -1 inside; `inside=+1` flips it.
    """
    th, ph = grid(n_theta, n_phi)
    x, y, z = embed(R, r, th, ph)
    xc, yc, zc = embed(R, r, np.array(theta0), np.array(varphi0))
    d = np.sqrt((x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2)
    return -inside * np.tanh((d - radius) / (xi * math.sqrt(2.0)))


def wrap_angle(x):
    """Map an angle difference into (-pi, pi]."""
    return np.pi - np.mod(np.pi - x, 2.0 * np.pi)


def stripe_phi(R, r, n_theta, n_phi, theta_c, width, xi, offset=0.0, inside=-1.0):
    """Azimuthally symmetric stripe (Eq. stripe_tanh): phi_0 + tanh(r/(xi sqrt2)(|theta - theta_c| - w/2)).

    The paper's stripe is the phi = -1 phase (inside = -1); inside = +1 gives the mirror image
    phi -> -phi, which the model maps onto itself.  `offset` is phi_0 of Eq. stripe_phi0 for the
    paper's sign convention.
    """
    th, _ = grid(n_theta, n_phi)
    prof = offset + np.tanh(r / (xi * math.sqrt(2.0)) * (np.abs(wrap_angle(th - theta_c)) - 0.5 * width))
    return prof if inside < 0 else -prof


# --------------------------------------------------------------------------------------
# Workloads.  Sizes and parameters follow the configurations the method is measured on;
# dt values are below the explicit stability limits of the scheme (vlb_max_stable_dt).
# --------------------------------------------------------------------------------------

def workload(name: str) -> dict:
    """Parameters (keyword arguments of the parameter struct) and initial fields of a named workload."""
    if name == "drop_torus_32x64":
        # single drop, R=2.5, r=1, A=kappa=0.04, M=0.1, tau=0.8, r0=0.4 centred at (pi/2, 0)
        p = dict(geometry=0, R=2.5, r=1.0, n_theta=32, n_phi=64, dt=5e-3, tau=0.8, M=0.1, A=0.04,
                 kappa=0.04, advection=0, ch_mode=0)
        xi = math.sqrt(p["kappa"] / p["A"])
        phi = drop_phi(p["R"], p["r"], 32, 64, math.pi / 2, 0.4, xi, inside=+1.0)
        rho = np.ones_like(phi)
        return dict(params=p, rho=rho, ut=np.zeros_like(phi), up=np.zeros_like(phi), phi=phi, steps=500)
    if name == "stripe_torus_128x384":
        # stripe oscillation, R=3, r=1; xi = 0.05, nu = M = 2.5e-3; +1 band of width 0.6 rad
        # dt = 0.89 of the SSP-RK3 limit of relaxation and varphi advection together (4.5e-3)
        p = dict(geometry=0, R=3.0, r=1.0, n_theta=128, n_phi=384, dt=4e-3, tau=2.5e-3, M=2.5e-3,
                 A=0.5, kappa=0.5 * 0.05 ** 2, advection=0, ch_mode=0)
        return _stripe(p, width=0.6, steps=20000)
    if name in ("coarsen_torus_1024x2048", "coarsen_flat_1024x2048"):
        # spinodal coarsening from noise +-0.01, R=2, r=1, tau=0.6, A=0.5, kappa=5e-4, M=2.5e-3
        geom = 0 if "torus" in name else 1
        p = dict(geometry=geom, R=2.0, r=1.0, n_theta=1024, n_phi=2048, dt=7e-6, tau=0.6, M=2.5e-3,
                 A=0.5, kappa=5e-4, advection=0, ch_mode=0)
        phi = noise(1, 1024, 2048, 0.01)
        return dict(params=p, rho=np.ones_like(phi), ut=np.zeros_like(phi), up=np.zeros_like(phi),
                    phi=phi, steps=50000)
    raise KeyError(name)


def _stripe(p, width, steps, theta_eq=math.pi, displacement=-math.pi / 20):
    """Stripe of the given width centred at theta_eq + displacement, +1 inside, with its offset."""
    R, r, A, kappa = p["R"], p["r"], p["A"], p["kappa"]
    xi = math.sqrt(kappa / A)
    tc = theta_eq + displacement
    a = r / R
    off = xi / (3.0 * R * math.sqrt(2.0)) * math.cos(tc) * math.sin(width / 2) / (
        1.0 + a * math.cos(tc) * math.cos(width / 2))
    phi = stripe_phi(R, r, p["n_theta"], p["n_phi"], tc, width, xi, offset=off, inside=+1.0)
    z = np.zeros_like(phi)
    return dict(params=p, rho=np.ones_like(phi), ut=z, up=z.copy(), phi=phi, steps=steps)


ENSEMBLE_GRIDS = ((64, 128), (128, 256), (256, 512), (512, 1024))


def ensemble_workload(count: int = 48, seed: int = 4):
    """Batched-ensemble workload: `count` tori with r = 1 and R uniformly spaced in [1.3, 5], grids drawn
    (counter-based, with `seed`) from ENSEMBLE_GRIDS, each with its own noise +-0.01 (seed 1000 + i).

    Fluid parameters are the paper's phase-separation set (tau = M = 2.5e-3, A = 0.5, kappa = 5e-4,
    Sec. 4) with rho = 1.  dt is left to the caller (each member's own stable step).
    Returns a list of dicts with `params` (without dt) and the initial fields.
    """
    pick = uniform01(seed, count, 1)[:, 0]
    out = []
    for i in range(count):
        nt, ns = ENSEMBLE_GRIDS[int(pick[i] * len(ENSEMBLE_GRIDS))]
        R = 1.3 + i * (5.0 - 1.3) / max(count - 1, 1)
        p = dict(geometry=0, R=R, r=1.0, n_theta=nt, n_phi=ns, tau=2.5e-3, M=2.5e-3, A=0.5, kappa=5e-4,
                 advection=0, ch_mode=0)
        phi = noise(1000 + i, nt, ns, 0.01)
        z = np.zeros_like(phi)
        out.append(dict(params=p, rho=np.ones_like(phi), ut=z, up=z.copy(), phi=phi))
    return out
