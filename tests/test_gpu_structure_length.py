"""Parity of vlb_structure_length (FP64 transform on the GPU, through the C ABI) with the oracle's
L_S = 2 pi sum S / sum |k| S on the same phi.

The oracle reads phi back from the solver (vlb_get_fields), so both sides see the same numbers in
either precision; the two transforms differ only in rounding order, so the gate is 1e-11 relative.
Grids from one column strip to many (the column kernel takes up to 32 columns per CTA) and the full
1024 x 2048 coarsening grid; torus and flat; a uniform phi (+inf) and a grid that is not a power of
two (rejected)."""
import math

import numpy as np
import pytest

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import inputs, vlb
from tests.gpu_helpers import gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def _params(nt, ns, geometry=0, R=2.0, r=1.0):
    return dict(geometry=geometry, R=R, r=r, n_theta=nt, n_phi=ns, dt=1e-4, tau=0.6, M=2.5e-3, A=0.5,
                kappa=5e-4, advection=0, ch_mode=0)


def _solver(p, phi, precision):
    s = vlb.Solver(gpu_params(p, precision))
    z = np.zeros_like(phi)
    s.set_fields(np.ones_like(phi), z, z, phi)
    return s


@pytest.mark.parametrize("precision", [vlb.FP64, vlb.FP32])
@pytest.mark.parametrize("nt,ns,geometry", [(4, 4, 0), (16, 32, 0), (64, 128, 1), (256, 512, 0), (512, 64, 0),
                                             (4096, 8, 1), (8, 4096, 0)])
def test_structure_length_matches_oracle(precision, nt, ns, geometry):
    p = _params(nt, ns, geometry, R=2.5 if geometry == 0 else 3.0, r=1.0 if geometry == 0 else 0.8)
    phi = inputs.quenched_noise(11 + nt, nt, ns, corr=max(1.0, min(nt, ns) / 16), width=1.5)
    s = _solver(p, phi, precision)
    try:
        got = s.structure_length()
        phi_back = s.fields()[3]
    finally:
        s.close()
    want = O.structure_length(phi_back, O.Geometry(oracle_params(p)))
    assert math.isfinite(got)
    assert abs(got - want) <= 1e-11 * want, (got, want)


@pytest.mark.parametrize("precision", [vlb.FP64, vlb.FP32])
def test_structure_length_full_size_noise_and_modes(precision):
    nt, ns = 1024, 2048
    p = _params(nt, ns)
    geo = O.Geometry(oracle_params(p))
    phi = inputs.noise(1, nt, ns, 0.01)
    s = _solver(p, phi, precision)
    try:
        got = s.structure_length()
        phi_back = s.fields()[3]
        want = O.structure_length(phi_back, geo)
        assert abs(got - want) <= 1e-11 * want, (got, want)
        # a single mode: the closed form 2 pi / |k|, whatever the grid
        th = geo.theta * np.ones((1, ns))
        ph = np.arange(ns)[None, :] * geo.dph * np.ones((nt, 1))
        z = np.zeros((nt, ns))
        s.set_fields(np.ones((nt, ns)), z, z, 0.5 * np.cos(7 * th - 40 * ph))
        tol = 1e-11 if precision == vlb.FP64 else 1e-9
        assert s.structure_length() == pytest.approx(2 * math.pi / math.hypot(7 / 1.0, 40 / 2.0), rel=tol)
    finally:
        s.close()


def test_structure_length_uniform_and_rejected_shapes():
    p = _params(32, 64)
    s = _solver(p, np.full((32, 64), 0.3), vlb.FP64)
    try:
        assert s.structure_length() == math.inf
    finally:
        s.close()
    p = _params(24, 64)
    s = _solver(p, np.zeros((24, 64)), vlb.FP64)
    try:
        with pytest.raises(vlb.VlbError, match="powers of two"):
            s.structure_length()
    finally:
        s.close()
