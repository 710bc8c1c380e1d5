"""The surrogate's convolution kernels at the size they run at (256 x 512, the learned-surrogate
workload), against the FP64 CPU oracle on the same BF16-rounded operands.

At this size the kernels take their production paths, which the small cases of test_gpu_conv.py do
not reach: the persistent forward kernel gives each CTA several work items (256 rows / 2 x 4
segments = 512 items over at most a few hundred CTAs), so the double-buffered patches, both
accumulators and the mbarrier phase flips after the first item are exercised; the 64 -> 64 weight
gradient splits the 1024 row segments into many pixel groups whose partial sums are reduced in a
fixed order; the 16-channel gradients cover many CTAs.  Every output element is checked against the
error bound of an FP32 sum of exact BF16 x BF16 products, and the convolutions' status flag must
stay clear."""
import numpy as np
import pytest

from oracle import conv_oracle as CO
from paper_1904_10070_gb300 import vlb

pytestmark = pytest.mark.gpu

H, W = 256, 512
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
def test_forward_full_size_with_bias_relu_and_mask(cin, cout):
    import torch
    rng = np.random.default_rng(1000 + cin + cout)
    x = _rand(rng, (H, W, cin))
    w = _rand(rng, (cout, 3, 3, cin), 0.1)
    b = rng.normal(size=cout).astype(np.float32).astype(np.float64)
    mask = _rand(rng, (H, W, cout))
    yf = torch.empty((H, W, cout), dtype=torch.float32, device="cuda")
    yb = torch.empty((H, W, cout), dtype=torch.bfloat16, device="cuda")
    vlb.vlb_conv3x3_fwd(H, W, cin, cout, _dev(x, torch.bfloat16), _dev(w, torch.bfloat16), _dev(b, torch.float32),
                        _dev(mask, torch.bfloat16), 1, yb, yf, _stream())
    vlb.vlb_conv_status(_stream(), clear=False)
    ref = CO.conv3x3(x, w, b, relu=True, mask=mask)
    bound = 2 * 9 * cin * 2.0 ** -24 * CO.conv3x3(np.abs(x), np.abs(w)) + 2.0 ** -24 * np.abs(b)
    got = _host(yf)
    bad = np.abs(got - ref) > bound + 1e-30
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])
    assert np.all(got[mask <= 0] == 0.0)
    np.testing.assert_array_equal(_host(yb), CO.bf16_round(got))


def test_backward_data_full_size():
    import torch
    cin, cout = 64, 64
    rng = np.random.default_rng(2024)
    w = _rand(rng, (cout, 3, 3, cin), 0.1)
    dy = _rand(rng, (H, W, cout))
    act = _rand(rng, (H, W, cin))
    wf = torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device="cuda")
    vlb.vlb_conv3x3_flip(cin, cout, _dev(w, torch.bfloat16), wf, _stream())
    dxf = torch.empty((H, W, cin), dtype=torch.float32, device="cuda")
    vlb.vlb_conv3x3_fwd(H, W, cout, cin, _dev(dy, torch.bfloat16), wf, None, _dev(act, torch.bfloat16), 0, None, dxf,
                        _stream())
    vlb.vlb_conv_status(_stream(), clear=False)
    ref = np.where(act > 0, CO.conv3x3_grad_input(dy, w), 0.0)
    bound = 2 * 9 * cout * 2.0 ** -24 * CO.conv3x3_grad_input(np.abs(dy), np.abs(w))
    assert np.all(np.abs(_host(dxf) - ref) <= bound + 1e-30)


@pytest.mark.parametrize("cin,cout", SHAPES)
def test_weight_gradient_full_size(cin, cout):
    import torch
    rng = np.random.default_rng(3000 + 7 * cin + cout)
    x, dy = _rand(rng, (H, W, cin)), _rand(rng, (H, W, cout))
    ws = torch.empty(vlb.vlb_conv3x3_wgrad_workspace_bytes(H, W, cin, cout), dtype=torch.uint8, device="cuda")
    dw = torch.empty((cout, 3, 3, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    vlb.vlb_conv3x3_bwd_weight(H, W, cin, cout, _dev(x, torch.bfloat16), _dev(dy, torch.bfloat16), dw, db, ws,
                               _stream())
    vlb.vlb_conv_status(_stream(), clear=False)
    rdw, rdb = CO.conv3x3_grad_weight(x, dy)
    adw, _ = CO.conv3x3_grad_weight(np.abs(x), np.abs(dy))
    npx = H * W
    gw = _host(dw)
    bad = np.abs(gw - rdw) > 2 * npx * 2.0 ** -24 * adw + 1e-30
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(gw - rdw) / (adw + 1e-30))))
    assert np.all(np.abs(_host(db) - rdb) <= 2 * npx * 2.0 ** -24 * np.abs(dy).reshape(-1, cout).sum(0) + 1e-30)
    # the reduction over pixel groups is in a fixed order: a second call gives the same bits
    dw2 = torch.empty_like(dw)
    vlb.vlb_conv3x3_bwd_weight(H, W, cin, cout, _dev(x, torch.bfloat16), _dev(dy, torch.bfloat16), dw2, None, ws,
                               _stream())
    assert torch.equal(dw, dw2)
