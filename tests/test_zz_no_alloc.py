"""vlb_step_noalloc against the handle API's vlb_step.

The no-allocation entry point serves callers that cannot allocate device memory where they step
(plug-ins restricted to the buffers their host application hands them, loops that must not
synchronise on cudaMalloc).  It must produce the same states as the regular step.  This file is collected last
so that a failure here leaves every other test already run; it runs alone or after the rest.
"""
import numpy as np
import pytest

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import vlb

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-3 * np.sqrt(ref.size)))


def _emax(x, ref):
    return float(np.max(np.abs(x - ref)) / max(float(np.max(np.abs(ref))), 1e-3))


# (n_theta, n_phi, geometry, advection, ch_mode): the packed-pair path (n_phi % 4 == 0), the scalar
# path (n_phi % 4 != 0), WENO5, the flat domain, the diffusive mode, and n_phi = 1, where the handle
# runs the single-CTA axisymmetric kernel and the no-allocation step the tile kernel
GRIDS = [(48, 96, vlb.TORUS, vlb.UW3, vlb.HYDRO), (40, 72, vlb.FLAT, vlb.WENO5, vlb.DIFFUSIVE),
         (30, 50, vlb.TORUS, vlb.WENO5, vlb.HYDRO), (33, 70, vlb.TORUS, vlb.UW3, vlb.DIFFUSIVE),
         (64, 1, vlb.TORUS, vlb.UW3, vlb.HYDRO)]


@pytest.mark.parametrize("nt,ns,geom,adv,mode", GRIDS)
@pytest.mark.parametrize("precision,tol", [(vlb.FP32, 2e-5), (vlb.FP64, 1e-12)])
def test_noalloc_step_matches_handle_step_on_consecutive_calls(nt, ns, geom, adv, mode, precision, tol):
    import torch
    p = dict(R=2.3, r=1.0, n_theta=nt, n_phi=ns, dt=1e-3, tau=0.2, M=0.05, A=0.3, kappa=0.01, geometry=geom,
             advection=adv, ch_mode=mode)
    p["dt"] = min(1e-3, 0.5 * vlb.vlb_max_stable_dt(vlb.make_params(**p)))
    p = vlb.make_params(**p, precision=precision)
    rng = np.random.default_rng(77)
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, (nt, ns))
    ut = 0.05 * rng.uniform(-1, 1, (nt, ns))
    up = 0.05 * rng.uniform(-1, 1, (nt, ns))
    phi = np.tanh(2.0 * rng.uniform(-1, 1, (nt, ns)))
    f, phi0 = O.init_state(rho, ut, up, phi)
    f16 = f.reshape(16, nt, ns)

    # regular path: handle with a torch-allocated workspace
    ref = vlb.Solver(p)
    ref.set_state(f16, phi0)

    # caller-owned device state in the documented layout: deviations from n0 w_i w_j, then phi
    N = nt * ns
    stride = (N + 63) // 64 * 64
    n0 = 1.0
    w = O.weights()
    ww = np.outer(w, w).reshape(16, 1)
    fp32 = precision == vlb.FP32
    narr = 18 if fp32 else 17
    host = np.zeros((narr, stride), dtype=np.float32 if fp32 else np.float64)
    host[:16, :N] = f16.reshape(16, N) - n0 * ww
    if fp32:
        hi = phi0.reshape(N).astype(np.float32)
        host[16, :N] = hi
        host[17, :N] = (phi0.reshape(N) - hi.astype(np.float64)).astype(np.float32)
    else:
        host[16, :N] = phi0.reshape(N)
    state = torch.from_numpy(host).cuda()
    assert state.data_ptr() % 256 == 0
    stream = torch.cuda.current_stream().cuda_stream

    for steps in (4, 6):  # two calls in a row: the scratch keeps the previous call's contents
        vlb.vlb_step_noalloc(p, state.data_ptr(), stride, n0, steps, stream)
        ref.step(steps)
        f_ref, phi_ref = ref.get_state()
        out = state.cpu().numpy().astype(np.float64)
        f_new = out[:16, :N] + n0 * ww
        phi_new = out[16, :N] + (out[17, :N] if fp32 else 0.0)
        for got, want in ((f_new, f_ref.reshape(16, N)), (phi_new, phi_ref.reshape(N))):
            assert _rel(got, want) <= tol and _emax(got, want) <= tol, (steps, _rel(got, want), _emax(got, want))
    ref.close()


def test_noalloc_rejects_grids_beyond_its_fixed_scratch():
    import torch
    p = vlb.make_params(R=2.0, r=1.0, n_theta=1024, n_phi=2048, dt=1e-5, tau=0.6, M=2.5e-3, A=0.5, kappa=5e-4,
                        precision=vlb.FP32)
    buf = torch.zeros(256, dtype=torch.float32, device="cuda")
    with pytest.raises(vlb.VlbError) as exc:
        vlb.vlb_step_noalloc(p, buf.data_ptr(), 1024 * 2048, 1.0, 1, torch.cuda.current_stream().cuda_stream)
    assert exc.value.status == vlb.VLB_ERR_ARG
    assert "scratch" in str(exc.value)
