"""Plain FP64 CPU oracle for the vielbein lattice-Boltzmann + Cahn-Hilliard time step on a torus.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It shares no code,
tables or constants with the CUDA library; the only thing both sides receive is the seeded
input arrays.

Method: Ambrus, Busuioc, Wagner, Paillusson & Kusumaatmaja, "Multicomponent flow on curved
surfaces: a vielbein lattice Boltzmann approach" (arXiv:1904.10070).  Every function cites
the section / equation it follows.  The paper defers its finite-difference details to a
Supplement that is not available; where the paper is silent this module takes these
readings (each one is listed with its reason in the project's design notes):

  * advection: conservative flux form; face values by the linear third-order upwind-biased
    reconstruction ("UW3") or by fifth-order WENO-JS (Jiang & Shu 1996); the quantity
    reconstructed along theta is (1 + a cos theta) f, along varphi it is f;
  * time integration: three-stage strong-stability-preserving Runge-Kutta (Shu & Osher 1988);
  * force: n F = -phi grad(mu) (Eq. pbin, first form) with central differences;
  * nodes at theta_q = q dtheta, varphi_s = s dvarphi, both periodic;
  * Laplace-Beltrami operator in conservative second-order form;
  * Cahn-Hilliard advective flux: face value = mean of the two nodal products.

Array layout: f has shape (4, 4, N_theta, N_phi); index [i, j] is the velocity
(v_i along theta-hat, v_j along varphi-hat), i.e. population k = 4 i + j.
phi, n, u have shape (N_theta, N_phi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

Q = 4  # quadrature order (Sec. 2.3: at least Q = 4 is needed off Cartesian coordinates)

TORUS = 0
FLAT = 1
UW3 = 0
WENO5 = 1
HYDRO = 0
DIFFUSIVE = 1


# --------------------------------------------------------------------------------------
# Velocity space (Sec. 2.3, Eq. vmatrix, the weight formula and the K^H kernels)
# --------------------------------------------------------------------------------------

def hermite(n: int, x):
    """Hermite polynomial He_n(x), orthogonal w.r.t. exp(-x^2/2)/sqrt(2 pi) (Sec. 2.3).

    Three-term recurrence He_{m+1} = x He_m - m He_{m-1}, He_0 = 1, He_1 = x.
    """
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.ones_like(x)
    h_prev, h = np.ones_like(x), x.copy()
    for m in range(1, n):
        h_prev, h = h, x * h - m * h_prev
    return h


def velocities() -> np.ndarray:
    """The four Q = 4 velocity roots of He_4 (Eq. vmatrix), ordered v_1 < ... < v_4."""
    s6 = math.sqrt(6.0)
    return np.array([-math.sqrt(3.0 + s6), -math.sqrt(3.0 - s6),
                     math.sqrt(3.0 - s6), math.sqrt(3.0 + s6)])


def weights() -> np.ndarray:
    """Quadrature weights w_k = Q! / He_{Q+1}(v_k)^2 (Sec. 2.3, formula below Eq. feq)."""
    v = velocities()
    return math.factorial(Q) / hermite(Q + 1, v) ** 2


def kernel_K() -> np.ndarray:
    """K^H_{i,m} = -w_i sum_{l=0}^{Q-1} He_{l+1}(v_i) He_l(v_m) / l!  (Sec. 2.3).

    (df/dv)_i = sum_m K^H_{i,m} f_m.
    """
    v, w = velocities(), weights()
    K = np.zeros((Q, Q))
    for i in range(Q):
        for m in range(Q):
            s = 0.0
            for l in range(Q):
                s += hermite(l + 1, v[i]) * hermite(l, v[m]) / math.factorial(l)
            K[i, m] = -w[i] * s
    return K


def kernel_Kt() -> np.ndarray:
    """K~^H_{i,m} = -w_i sum_l He_{l+1}(v_i) [He_{l+1}(v_m) + l He_{l-1}(v_m)] / l!  (Sec. 2.3).

    (d(f v)/dv)_i = sum_m K~^H_{i,m} f_m.  The l = 0 term has no He_{-1} contribution.
    """
    v, w = velocities(), weights()
    K = np.zeros((Q, Q))
    for i in range(Q):
        for m in range(Q):
            s = 0.0
            for l in range(Q):
                inner = hermite(l + 1, v[m])
                if l > 0:
                    inner = inner + l * hermite(l - 1, v[m])
                s += hermite(l + 1, v[i]) * inner / math.factorial(l)
            K[i, m] = -w[i] * s
    return K


# --------------------------------------------------------------------------------------
# Problem definition
# --------------------------------------------------------------------------------------

@dataclass
class Params:
    """Torus (R, r) or flat periodic domain (L_x = 2 pi R along varphi, L_y = 2 pi r along theta)."""
    R: float
    r: float
    n_theta: int
    n_phi: int
    dt: float
    tau: float            # BGK relaxation time; nu = tau (Eq. nu with k_B T = m = 1); inf = no collision
    M: float              # Cahn-Hilliard mobility (Eq. CH)
    A: float              # Landau free-energy parameters (Eq. Landau)
    kappa: float
    geometry: int = TORUS
    advection: int = UW3
    ch_mode: int = HYDRO  # DIFFUSIVE: no advection in CH and no force on the fluid (Sec. 4.1.1)
    ch_stab: int = 0      # 1: stabilised semi-implicit Cahn-Hilliard stages (not in the paper; see stabiliser)


class Geometry:
    """Per-theta-row geometric factors (App. A: Eq. torus, the metric, the vielbein, Eq. conn_torus).

    J_q = 1 + a cos theta_q with a = r/R, so sqrt(g) = r R J_q and R + r cos theta = R J_q;
    Jp/Jm are J at the cell faces theta_q +- dtheta/2;
    Gamma_q = sin theta_q / (R + r cos theta_q) is the only independent connection coefficient.
    All arrays have shape (N_theta, 1) so that they broadcast over varphi.
    """

    def __init__(self, p: Params, rows=None):
        """`rows` (optional) restricts the tables to the given theta-row indices of the full grid,
        for evaluating the scheme on a window cut out of a larger grid (see step_window)."""
        self.p = p
        self.dth = 2.0 * math.pi / p.n_theta
        self.dph = 2.0 * math.pi / p.n_phi
        idx = np.arange(p.n_theta) if rows is None else np.asarray(rows)
        th = idx.astype(np.float64) * self.dth
        self.theta = th[:, None]
        if p.geometry == TORUS:
            a = p.r / p.R
            self.J = 1.0 + a * np.cos(th)[:, None]
            self.Jp = 1.0 + a * np.cos(th + 0.5 * self.dth)[:, None]
            self.Jm = 1.0 + a * np.cos(th - 0.5 * self.dth)[:, None]
            self.Gamma = np.sin(th)[:, None] / (p.R * self.J)
        else:
            self.J = np.ones((th.size, 1))
            self.Jp = np.ones((th.size, 1))
            self.Jm = np.ones((th.size, 1))
            self.Gamma = np.zeros((th.size, 1))
        self.sqrtg = p.r * p.R * self.J
        self.dA = self.sqrtg * self.dth * self.dph  # area element of one cell


# --------------------------------------------------------------------------------------
# Moments, equilibrium (Sec. 2.3, Eq. feq)
# --------------------------------------------------------------------------------------

def moments(f: np.ndarray):
    """n = sum_k f_k,  n u = sum_k f_k v_k  (Sec. 2.3)."""
    v = velocities()
    n = f.sum(axis=(0, 1))
    nut = np.einsum("i,ijqs->qs", v, f)
    nup = np.einsum("j,ijqs->qs", v, f)
    return n, nut / n, nup / n


def feq(n, ut, up) -> np.ndarray:
    """Third-order Hermite equilibrium, Eq. feq, with k_B T = m = 1."""
    v, w = velocities(), weights()
    xi = v[:, None, None, None] * ut[None, None] + v[None, :, None, None] * up[None, None]
    usq = ut * ut + up * up
    poly = 1.0 + xi + 0.5 * (xi * xi - usq) + xi * (xi * xi - 3.0 * usq) / 6.0
    return n[None, None] * w[:, None, None, None] * w[None, :, None, None] * poly


# --------------------------------------------------------------------------------------
# Finite differences on the periodic grid
# --------------------------------------------------------------------------------------

def _sh(x, k, axis):
    """x shifted so that element i holds x[i + k] (periodic)."""
    return np.roll(x, -k, axis=axis)


def laplace_beltrami(x, geo: Geometry):
    """Second-order conservative Laplace-Beltrami operator on the torus (Eq. mu's Delta).

    Delta x = (1/(r^2 J)) d_theta(J d_theta x) + (1/(R^2 J^2)) d_phi^2 x, with J at faces.
    """
    p = geo.p
    ax_t, ax_p = x.ndim - 2, x.ndim - 1
    lt = (geo.Jp * (_sh(x, 1, ax_t) - x) - geo.Jm * (x - _sh(x, -1, ax_t))) / (p.r ** 2 * geo.J * geo.dth ** 2)
    lp = (_sh(x, 1, ax_p) - 2.0 * x + _sh(x, -1, ax_p)) / (p.R ** 2 * geo.J ** 2 * geo.dph ** 2)
    return lt + lp


def chemical_potential(phi, geo: Geometry):
    """mu = -A phi (1 - phi^2) - kappa Delta phi  (Eq. mu)."""
    p = geo.p
    return -p.A * phi * (1.0 - phi * phi) - p.kappa * laplace_beltrami(phi, geo)


def _uw3_face(gm1, g0, gp1):
    """Linear third-order upwind-biased face value at i+1/2 for a positive velocity."""
    return (-gm1 + 5.0 * g0 + 2.0 * gp1) / 6.0


def _weno5_face(gm2, gm1, g0, gp1, gp2, eps=1e-6):
    """Fifth-order WENO-JS face value at i+1/2 for a positive velocity (Jiang & Shu 1996)."""
    q0 = (2.0 * gm2 - 7.0 * gm1 + 11.0 * g0) / 6.0
    q1 = (-gm1 + 5.0 * g0 + 2.0 * gp1) / 6.0
    q2 = (2.0 * g0 + 5.0 * gp1 - gp2) / 6.0
    b0 = 13.0 / 12.0 * (gm2 - 2.0 * gm1 + g0) ** 2 + 0.25 * (gm2 - 4.0 * gm1 + 3.0 * g0) ** 2
    b1 = 13.0 / 12.0 * (gm1 - 2.0 * g0 + gp1) ** 2 + 0.25 * (gm1 - gp1) ** 2
    b2 = 13.0 / 12.0 * (g0 - 2.0 * gp1 + gp2) ** 2 + 0.25 * (3.0 * g0 - 4.0 * gp1 + gp2) ** 2
    a0 = 0.1 / (eps + b0) ** 2
    a1 = 0.6 / (eps + b1) ** 2
    a2 = 0.3 / (eps + b2) ** 2
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def face_values(g, axis: int, positive: bool, scheme: int):
    """Upwind face value of g at i+1/2 along `axis` for a velocity of the given sign."""
    if positive:
        pts = [_sh(g, k, axis) for k in (-2, -1, 0, 1, 2)]
    else:  # mirror image: the upwind side is i+1
        pts = [_sh(g, k, axis) for k in (3, 2, 1, 0, -1)]
    if scheme == UW3:
        return _uw3_face(pts[1], pts[2], pts[3])
    return _weno5_face(*pts)


def flux_difference(g, axis: int, positive: bool, scheme: int):
    """g_{i+1/2} - g_{i-1/2} with upwind face values."""
    F = face_values(g, axis, positive, scheme)
    return F - _sh(F, -1, axis)


# --------------------------------------------------------------------------------------
# Right-hand sides (Eq. boltz_tor with the BGK term; Eq. CH; Eq. pbin)
# --------------------------------------------------------------------------------------

def force(phi, n, mu, geo: Geometry):
    """F^a = -(phi/n) grad^a mu  (Eq. pbin), central differences; vielbein components."""
    p = geo.p
    dmu_t = (_sh(mu, 1, 0) - _sh(mu, -1, 0)) / (2.0 * p.r * geo.dth)
    dmu_p = (_sh(mu, 1, 1) - _sh(mu, -1, 1)) / (2.0 * p.R * geo.J * geo.dph)
    return -phi * dmu_t / n, -phi * dmu_p / n


def rhs(f, phi, geo: Geometry):
    """Time derivatives (df/dt, dphi/dt) of the semi-discrete system.

    df/dt = - v_theta/(r J) d_theta(J f) - v_phi/(R J) d_phi f
            - F^theta df/dv_theta - F^phi df/dv_phi
            + Gamma [v_phi^2 df/dv_theta - v_theta d(f v_phi)/dv_phi]
            - (f - f^eq)/tau                                      (Eq. boltz_tor, BGK)
    dphi/dt = - div(u phi) + M Delta mu                           (Eq. CH)
    """
    p = geo.p
    v = velocities()
    K, Kt = kernel_K(), kernel_Kt()
    n, ut, up = moments(f)
    mu = chemical_potential(phi, geo)

    # advection, conservative form (Eq. boltz_cons / boltz_tor), populations one at a time
    adv = np.empty_like(f)
    for i in range(Q):
        for j in range(Q):
            dG = flux_difference(geo.J * f[i, j], 0, v[i] > 0, p.advection)
            df = flux_difference(f[i, j], 1, v[j] > 0, p.advection)
            adv[i, j] = -v[i] * dG / (p.r * geo.J * geo.dth) - v[j] * df / (p.R * geo.J * geo.dph)

    # velocity-space derivatives (Sec. 2.3)
    df_dvt = np.einsum("ab,bjqs->ajqs", K, f)       # (df/dv_theta)_{ij}
    df_dvp = np.einsum("ab,ibqs->iaqs", K, f)       # (df/dv_phi)_{ij}
    dfvp_dvp = np.einsum("ab,ibqs->iaqs", Kt, f)    # (d(f v_phi)/dv_phi)_{ij}

    if p.ch_mode == HYDRO:
        Ft, Fp = force(phi, n, mu, geo)
    else:
        Ft, Fp = np.zeros_like(phi), np.zeros_like(phi)

    vt = v[:, None, None, None]
    vp = v[None, :, None, None]
    Lf = (adv
          - Ft[None, None] * df_dvt
          - Fp[None, None] * df_dvp
          + geo.Gamma[None, None] * (vp * vp * df_dvt - vt * dfvp_dvp)
          - (f - feq(n, ut, up)) / p.tau)

    # Cahn-Hilliard (Eq. CH): divergence in conservative form, face value = mean of nodes
    Lphi = p.M * laplace_beltrami(mu, geo)
    if p.ch_mode == HYDRO:
        gt = geo.J * ut * phi
        gp = up * phi
        face_t = 0.5 * (gt + _sh(gt, 1, 0))
        face_p = 0.5 * (gp + _sh(gp, 1, 1))
        Lphi = Lphi - (face_t - _sh(face_t, -1, 0)) / (p.r * geo.J * geo.dth) \
                    - (face_p - _sh(face_p, -1, 1)) / (p.R * geo.J * geo.dph)
    return Lf, Lphi


# --------------------------------------------------------------------------------------
# Stabilised semi-implicit Cahn-Hilliard (not in the paper: it lifts the explicit dt ~ h^4 limit)
# --------------------------------------------------------------------------------------

def biharmonic_symbol(geo: Geometry) -> np.ndarray:
    """lambda(k) = (symbol of the constant-coefficient periodic five-point Laplacian)^2 for every
    discrete Fourier mode k = (k_theta, k_phi) of the grid, with the finest spacings of the domain:
    h_theta = r dtheta and h_phi = (R - r) dvarphi on the torus (the inner equator), R dvarphi flat.
    The symbol of the Laplacian is -(4/h_theta^2) sin^2(pi m/N_theta) - (4/h_phi^2) sin^2(pi n/N_phi)."""
    p = geo.p
    h_t = p.r * geo.dth
    h_p = ((p.R - p.r) if p.geometry == TORUS else p.R) * geo.dph
    m = np.arange(p.n_theta)[:, None]
    n = np.arange(p.n_phi)[None, :]
    lap = 4.0 / h_t ** 2 * np.sin(np.pi * m / p.n_theta) ** 2 + 4.0 / h_p ** 2 * np.sin(np.pi * n / p.n_phi) ** 2
    return lap * lap


def stabiliser(x, geo: Geometry):
    """P x = J^{-1} F^{-1}[ F[J x] / (1 + dt sigma lambda(k)) ] with sigma = M kappa (F: the 2-D
    discrete Fourier transform).  P is the inverse of I + dt sigma J^{-1} D^2 J, D the constant-
    coefficient Laplacian above: every mode of J x is damped, the mean of J x (k = 0) is kept, so
    P conserves sum J x, i.e. the integral of x sqrt(g)."""
    p = geo.p
    lam = biharmonic_symbol(geo)
    z = np.fft.fft2(geo.J * x)
    return np.real(np.fft.ifft2(z / (1.0 + p.dt * p.M * p.kappa * lam))) / geo.J


def step(f, phi, geo: Geometry):
    """One SSP-RK3 step (Shu-Osher form) of the coupled (f, phi) system.

    With ch_stab the phi equation is advanced as phi' = P L_phi(f, phi) with the fixed preconditioner
    P of `stabiliser` (the same for the three stages): the stiff kappa Delta^2 modes, whose explicit
    limit is dt ~ h^4 / (M kappa), are damped to dt-eigenvalues within [-1, 0], while P -> I as
    dt -> 0 (a first-order perturbation of the time derivative)."""
    dt = geo.p.dt
    P = (lambda x: stabiliser(x, geo)) if geo.p.ch_stab else (lambda x: x)
    Lf, Lp = rhs(f, phi, geo)
    f1, p1 = f + dt * Lf, phi + P(dt * Lp)
    Lf, Lp = rhs(f1, p1, geo)
    f2, p2 = 0.75 * f + 0.25 * (f1 + dt * Lf), 0.75 * phi + 0.25 * (p1 + P(dt * Lp))
    Lf, Lp = rhs(f2, p2, geo)
    return (f / 3.0 + 2.0 / 3.0 * (f2 + dt * Lf),
            phi / 3.0 + 2.0 / 3.0 * (p2 + P(dt * Lp)))


def step_window(f, phi, p: Params, q: int, s: int, half: int = 12):
    """One step of the full periodic grid, evaluated only at node (q, s).

    A (2 half + 1)^2 window around the node is cut out (periodically) and stepped as if it were
    periodic itself; the wrong wrap-around at the window edges travels at most 3 nodes per
    Runge-Kutta stage (the widest stencil, WENO5 advection), so with half >= 9 the centre is
    exactly the full-grid result.  Returns (f[:, :, centre], phi[centre]).
    """
    if p.ch_stab:
        raise ValueError("step_window: the stabilised step is global (Fourier) and has no node window")
    rows = np.arange(q - half, q + half + 1) % p.n_theta
    cols = np.arange(s - half, s + half + 1) % p.n_phi
    geo = Geometry(p, rows=rows)
    fw = f[:, :, rows][:, :, :, cols]
    pw = phi[rows][:, cols]
    # the false seams of the cut-out window may overflow at its edges; the centre is still exact
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        f1, p1 = step(fw, pw, geo)
    fc, pc = f1[:, :, half, half], p1[half, half]
    if not (np.all(np.isfinite(fc)) and np.isfinite(pc)):
        raise FloatingPointError(f"step_window: non-finite value at the centre node ({q}, {s})")
    return fc, pc


def run(f, phi, geo: Geometry, nsteps: int):
    for _ in range(nsteps):
        f, phi = step(f, phi, geo)
    return f, phi


def init_state(rho, ut, up, phi):
    """Distributions initialised at equilibrium, f = f^eq(n, u) (Sec. 4, initial state)."""
    return feq(np.asarray(rho, float), np.asarray(ut, float), np.asarray(up, float)), np.array(phi, float)


# --------------------------------------------------------------------------------------
# Diagnostics (Eq. Landau, Sec. 3.2 pressure, Eq. cart_scaling_L0, Eq. phiavg)
# --------------------------------------------------------------------------------------

def totals(f, phi, geo: Geometry):
    """(int n sqrt(g), int phi sqrt(g), Psi, max |u|) on the grid.

    Psi = int [A/4 (1-phi^2)^2 + kappa/2 |grad phi|^2] dA (Eq. Landau), grad by central differences.
    """
    p = geo.p
    n, ut, up = moments(f)
    gt = (_sh(phi, 1, 0) - _sh(phi, -1, 0)) / (2.0 * p.r * geo.dth)
    gp = (_sh(phi, 1, 1) - _sh(phi, -1, 1)) / (2.0 * p.R * geo.J * geo.dph)
    dens = 0.25 * p.A * (1.0 - phi * phi) ** 2 + 0.5 * p.kappa * (gt * gt + gp * gp)
    return np.array([float(np.sum(n * geo.dA)), float(np.sum(phi * geo.dA)),
                     float(np.sum(dens * geo.dA)), float(np.max(np.sqrt(ut * ut + up * up)))])


def pressure(n, phi, A):
    """p = n k_B T + A(-phi^2/2 + 3 phi^4/4) with k_B T = 1 (Sec. 3.2)."""
    return n + A * (-0.5 * phi ** 2 + 0.75 * phi ** 4)


def interface_length(phi, geo: Geometry) -> float:
    """L_I by the cell walk of Sec. 4: every pair of neighbours with phi phi' < 0 adds the shared edge.

    Neighbours along varphi share an edge of length r dtheta (delta y on a flat domain);
    neighbours along theta share (R + r cos theta_{q+1/2}) dvarphi (delta x on a flat domain).
    Both directions are periodic.
    """
    p = geo.p
    total = 0.0
    nq, ns = phi.shape
    for q in range(nq):
        if p.geometry == TORUS:
            edge_t = (p.R + p.r * math.cos((q + 0.5) * geo.dth)) * geo.dph
        else:
            edge_t = p.R * geo.dph
        edge_p = p.r * geo.dth
        for s in range(ns):
            if phi[q, s] * phi[q, (s + 1) % ns] < 0.0:
                total += edge_p
            if phi[q, s] * phi[(q + 1) % nq, s] < 0.0:
                total += edge_t
    return total


def domain_length(phi, geo: Geometry) -> float:
    """L_d = A_total / L_I  (Eq. cart_scaling_L0)."""
    p = geo.p
    return 4.0 * math.pi ** 2 * p.r * p.R / interface_length(phi, geo)


def azimuthal_mean(phi):
    """<phi>_q = (1/N_phi) sum_s phi_{s,q}  (Eq. phiavg, discrete form)."""
    return phi.mean(axis=1)


def structure_factor(phi):
    """S(m, n) = |sum_{q,s} phi_{q,s} exp(-2 pi i (m q / N_theta + n s / N_phi))|^2 on the index grid.

    The structure factor of the coarsening runs (Sec. 4.1 measures the domain size; a Fourier
    measure is the usual alternative to L_d).  A library FFT is the transform."""
    return np.abs(np.fft.fft2(phi)) ** 2


def structure_length(phi, geo: Geometry) -> float:
    """L_S = 2 pi sum_k S(k) / sum_k |k| S(k) over all k != 0.

    Wavenumbers on the index grid with the physical lengths 2 pi r along theta and 2 pi R along
    varphi (the flat domain's sides; on the torus R is the mean circumference over 2 pi):
    k = (m'/r, n'/R) with m', n' the signed integer frequencies (m' = m - N_theta above N_theta/2).
    A single mode cos(m theta + n varphi) gives L_S = 2 pi / |k| exactly; a uniform phi gives +inf.
    """
    p = geo.p
    nt, ns = phi.shape
    S = structure_factor(phi)
    m = np.fft.fftfreq(nt, 1.0 / nt)[:, None]
    n = np.fft.fftfreq(ns, 1.0 / ns)[None, :]
    k = np.sqrt((m / p.r) ** 2 + (n / p.R) ** 2)
    S = S.copy()
    S[0, 0] = 0.0
    den = float((k * S).sum())
    return 2.0 * math.pi * float(S.sum()) / den if den > 0.0 else math.inf  # uniform phi: no domains
