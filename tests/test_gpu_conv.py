"""The surrogate network's CUDA kernels (tensor-core BF16 convolutions with FP32 accumulation,
loss, optimiser) against the FP64 CPU oracle on the same BF16-rounded operands."""
import numpy as np
import pytest

from oracle import conv_oracle as CO
from paper_1904_10070_gb300 import vlb

pytestmark = pytest.mark.gpu

SHAPES = [(16, 64), (64, 64), (64, 16)]


def _dev(a, dtype):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(device="cuda", dtype=dtype).contiguous()


def _host(t):
    return t.float().cpu().numpy().astype(np.float64)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _rand(rng, shape, scale=1.0):
    return CO.bf16_round(scale * rng.normal(size=shape))


@pytest.mark.parametrize("cin,cout", SHAPES)
@pytest.mark.parametrize("H,W", [(2, 128), (6, 256)])
def test_forward_matches_oracle(cin, cout, H, W):
    import torch
    rng = np.random.default_rng(cin * 100 + cout + H)
    x = _rand(rng, (H, W, cin))
    w = _rand(rng, (cout, 3, 3, cin), 0.1)
    b = rng.normal(size=cout).astype(np.float32).astype(np.float64)
    yf = torch.empty((H, W, cout), dtype=torch.float32, device="cuda")
    yb = torch.empty((H, W, cout), dtype=torch.bfloat16, device="cuda")
    vlb.vlb_conv3x3_fwd(H, W, cin, cout, _dev(x, torch.bfloat16), _dev(w, torch.bfloat16), _dev(b, torch.float32),
                        None, 0, yb, yf, _stream())
    ref = CO.conv3x3(x, w, b)
    bound = 2 * 9 * cin * 2.0 ** -24 * CO.conv3x3(np.abs(x), np.abs(w)) + 2.0 ** -24 * np.abs(b)
    assert np.all(np.abs(_host(yf) - ref) <= bound + 1e-30)
    # bf16 output: the FP32 value rounded once
    assert np.all(np.abs(_host(yb) - CO.bf16_round(_host(yf))) <= 0.0)


def test_forward_relu_and_mask_epilogues():
    import torch
    H, W, cin, cout = 4, 128, 64, 64
    rng = np.random.default_rng(5)
    x, w = _rand(rng, (H, W, cin)), _rand(rng, (cout, 3, 3, cin), 0.1)
    mask = _rand(rng, (H, W, cout))
    yf = torch.empty((H, W, cout), dtype=torch.float32, device="cuda")
    vlb.vlb_conv3x3_fwd(H, W, cin, cout, _dev(x, torch.bfloat16), _dev(w, torch.bfloat16), None,
                        _dev(mask, torch.bfloat16), 1, None, yf, _stream())
    ref = CO.conv3x3(x, w, relu=True, mask=mask)
    bound = 2 * 9 * cin * 2.0 ** -24 * CO.conv3x3(np.abs(x), np.abs(w))
    assert np.all(np.abs(_host(yf) - ref) <= bound + 1e-30)
    assert np.all(_host(yf)[mask <= 0] == 0.0)


@pytest.mark.parametrize("cin,cout", [(64, 64), (64, 16)])
def test_backward_data_by_flipped_forward(cin, cout):
    import torch
    H, W = 6, 256
    rng = np.random.default_rng(cin + 3 * cout)
    w = _rand(rng, (cout, 3, 3, cin), 0.1)
    dy = _rand(rng, (H, W, cout))
    act = _rand(rng, (H, W, cin))  # the layer's input activation: the mask of the ReLU derivative
    wf = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device="cuda")
    vlb.vlb_conv3x3_flip(cin, cout, _dev(w, torch.bfloat16), wf, _stream())
    dxf = torch.empty((H, W, cin), dtype=torch.float32, device="cuda")
    vlb.vlb_conv3x3_fwd(H, W, cout, cin, _dev(dy, torch.bfloat16), wf, None, _dev(act, torch.bfloat16), 0, None, dxf,
                        _stream())
    ref = np.where(act > 0, CO.conv3x3_grad_input(dy, w), 0.0)
    bound = 2 * 9 * cout * 2.0 ** -24 * CO.conv3x3_grad_input(np.abs(dy), np.abs(w))
    assert np.all(np.abs(_host(dxf) - ref) <= bound + 1e-30)


@pytest.mark.parametrize("cin,cout", SHAPES)
def test_backward_weight_matches_oracle(cin, cout):
    import torch
    H, W = 4, 256
    rng = np.random.default_rng(7 * cin + cout)
    x, dy = _rand(rng, (H, W, cin)), _rand(rng, (H, W, cout))
    ws = torch.empty(vlb.vlb_conv3x3_wgrad_workspace_bytes(H, W, cin, cout), dtype=torch.uint8, device="cuda")
    dw = torch.empty((cout, 3, 3, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    vlb.vlb_conv3x3_bwd_weight(H, W, cin, cout, _dev(x, torch.bfloat16), _dev(dy, torch.bfloat16), dw, db, ws,
                               _stream())
    rdw, rdb = CO.conv3x3_grad_weight(x, dy)
    adw, _ = CO.conv3x3_grad_weight(np.abs(x), np.abs(dy))
    npx = H * W
    assert np.all(np.abs(_host(dw) - rdw) <= 2 * npx * 2.0 ** -24 * adw + 1e-30)
    assert np.all(np.abs(_host(db) - rdb) <= 2 * npx * 2.0 ** -24 * np.abs(dy).reshape(-1, cout).sum(0) + 1e-30)


def test_mse_and_adam_match_oracle():
    import torch
    rng = np.random.default_rng(9)
    n = 3000
    pred = rng.normal(size=(n, 16)).astype(np.float32).astype(np.float64)
    tgt = rng.normal(size=(n, 4)).astype(np.float32).astype(np.float64)
    work = torch.empty(vlb.vlb_reduce_workspace_bytes(), dtype=torch.uint8, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, 16), dtype=torch.bfloat16, device="cuda")
    vlb.vlb_mse_loss(n, _dev(pred, torch.float32), _dev(tgt, torch.float32), grad, work, loss, _stream())
    rl, rg = CO.mse(pred[:, :4], tgt)
    assert abs(float(loss.cpu()) - rl) <= 1e-7 * rl  # differences are formed in FP32
    g = _host(grad)
    assert np.all(g[:, 4:] == 0.0)
    assert np.all(np.abs(g[:, :4] - rg) <= 2 ** -8 * np.abs(rg) + 1e-30)
    # Adam on 1000 parameters for 3 steps
    p0 = rng.normal(size=1000)
    gs = [rng.normal(size=1000) for _ in range(3)]
    p, m, v = _dev(p0, torch.float32), torch.zeros(1000, device="cuda"), torch.zeros(1000, device="cuda")
    pb = torch.empty(1000, dtype=torch.bfloat16, device="cuda")
    rp, rm, rv = p0.astype(np.float32).astype(np.float64), np.zeros(1000), np.zeros(1000)
    for t, gg in enumerate(gs, start=1):
        gg32 = gg.astype(np.float32).astype(np.float64)
        vlb.vlb_adam_step(1000, p, _dev(gg32, torch.float32), m, v, t, 1e-2, 0.9, 0.999, 1e-8, pb, _stream())
        rp, rm, rv = CO.adam(rp, gg32, rm, rv, t, 1e-2)
    np.testing.assert_allclose(_host(p), rp, rtol=0, atol=1e-6)
    np.testing.assert_array_equal(_host(pb), CO.bf16_round(_host(p)))


def test_snapshot_roundtrip_restarts_at_equilibrium_and_conserves():
    import torch
    from oracle import vlb_oracle as O
    nt, ns = 32, 64
    p = vlb.make_params(R=2.5, r=1.0, n_theta=nt, n_phi=ns, dt=1e-3, tau=0.5, M=0.05, A=0.3, kappa=0.01,
                        precision=vlb.FP32)
    rng = np.random.default_rng(11)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, (nt, ns))
    ut, up = 0.03 * rng.uniform(-1, 1, (nt, ns)), 0.03 * rng.uniform(-1, 1, (nt, ns))
    phi = np.tanh(2 * rng.uniform(-1, 1, (nt, ns)))
    s = vlb.Solver(p)
    s.set_fields(rho, ut, up, phi)
    s.step(5)
    tot = s.totals()
    snap = torch.empty((nt * ns, 4), dtype=torch.float32, device="cuda")
    vlb.vlb_get_snapshot(s.h, snap)
    r0, u0, v0, p0, _ = s.fields()
    sn = snap.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(sn[:, 0], p0.ravel(), atol=1e-6)
    np.testing.assert_allclose(sn[:, 1], r0.ravel(), rtol=1e-6)
    # perturb, restart with conservation: totals come back, f is the equilibrium of the snapshot
    sn[:, 0] += 0.01
    sn[:, 1] *= 1.001
    vlb.vlb_set_snapshot(s.h, torch.tensor(sn, dtype=torch.float32, device="cuda"), (tot[0], tot[1]))
    t2 = s.totals()
    assert abs(t2[0] - tot[0]) <= 1e-6 * abs(tot[0]) and abs(t2[1] - tot[1]) <= 1e-5 * abs(tot[0])
    f16, _ = s.get_state()
    r, a, b, _, _ = s.fields()
    np.testing.assert_allclose(f16.reshape(4, 4, nt, ns), O.feq(r, a, b), rtol=0, atol=2e-6)
    s.close()


def test_snapshot_restart_keeps_the_nonequilibrium_part():
    """keep_neq: f := f + f^eq(n', u') - f^eq(n, u).  The state's own snapshot leaves the populations
    unchanged bit for bit; a changed one gives f the new moments and keeps f - f^eq."""
    import torch
    from oracle import vlb_oracle as O
    nt, ns = 32, 64
    p = vlb.make_params(R=2.5, r=1.0, n_theta=nt, n_phi=ns, dt=1e-3, tau=0.5, M=0.05, A=0.3, kappa=0.01,
                        precision=vlb.FP32)
    rng = np.random.default_rng(12)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, (nt, ns))
    ut, up = 0.03 * rng.uniform(-1, 1, (nt, ns)), 0.03 * rng.uniform(-1, 1, (nt, ns))
    s = vlb.Solver(p)
    s.set_fields(rho, ut, up, np.tanh(2 * rng.uniform(-1, 1, (nt, ns))))
    s.step(20)  # develops a non-equilibrium part
    f0, phi0 = s.get_state()
    snap = torch.empty((nt * ns, 4), dtype=torch.float32, device="cuda")
    vlb.vlb_get_snapshot(s.h, snap)
    vlb.vlb_set_snapshot(s.h, snap, None, keep_neq=True)
    f1, phi1 = s.get_state()
    np.testing.assert_array_equal(f1, f0)
    np.testing.assert_allclose(phi1, phi0, rtol=0, atol=1e-7)
    r0, a0, b0, _, _ = s.fields()
    neq0 = f0.reshape(4, 4, nt, ns) - O.feq(r0, a0, b0)
    assert np.max(np.abs(neq0)) > 1e-5  # there is a non-equilibrium part to keep
    sn = snap.cpu().numpy().astype(np.float64)
    sn[:, 1] *= 1.002
    sn[:, 2] += 0.01
    vlb.vlb_set_snapshot(s.h, torch.tensor(sn, dtype=torch.float32, device="cuda"), None, keep_neq=True)
    f2, _ = s.get_state()
    r2, a2, b2, _, _ = s.fields()
    np.testing.assert_allclose(r2.ravel(), sn[:, 1], rtol=2e-6)
    np.testing.assert_allclose(a2.ravel(), sn[:, 2], rtol=0, atol=2e-6)
    np.testing.assert_allclose(b2.ravel(), sn[:, 3], rtol=0, atol=2e-6)
    neq2 = f2.reshape(4, 4, nt, ns) - O.feq(r2, a2, b2)
    np.testing.assert_allclose(neq2, neq0, rtol=0, atol=2e-6)
    s.close()
