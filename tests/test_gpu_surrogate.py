"""The surrogate network on the GPU, layer by layer, against the FP64 CPU oracle of its operations.

Each kernel is checked on the inputs it actually received (the GPU's own bf16 activations and
incoming gradients), so the checks do not depend on how rounding differences propagate through
eight layers.  Bounds: a bf16 output may differ from the rounded FP64 value by one bf16 unit
(2^-7 relative, from FP32 accumulation order near a rounding boundary); FP32 outputs and weight
gradients are FP32 sums of exact bf16 x bf16 products (relative 1e-4 of the largest term sum)."""
import numpy as np
import pytest

from oracle import conv_oracle as CO
from paper_1904_10070_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

BF16_ULP = 2.0 ** -7


def _host(t):
    return t.float().cpu().numpy().astype(np.float64)


def _close_bf16(got, want, what):
    scale = max(np.max(np.abs(want)), 1e-30)
    bad = np.abs(got - want) > BF16_ULP * np.abs(want) + 1e-6 * scale
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - want))))


@pytest.mark.parametrize("H,W", [(4, 128), (6, 256), (256, 512)])
def test_network_layers_match_cpu_oracle(H, W):
    """(256, 512) is the surrogate workload's size: the persistent kernels' multi-item paths."""
    import torch
    net = S.SurrogateNet(H, W, seed=3)
    rng = np.random.default_rng(4)
    feat = np.zeros((H, W, 16))
    feat[:, :, :10] = rng.normal(size=(H, W, 10))
    feat = CO.bf16_round(feat)
    net.acts[0].copy_(torch.tensor(feat, dtype=torch.bfloat16, device="cuda"))
    for b in net.b32:  # non-zero biases so that the bias path is exercised
        b.copy_(torch.tensor(rng.normal(size=b.shape[0]) * 0.1, dtype=torch.float32, device="cuda"))
    target = rng.normal(size=(H * W, 4)).astype(np.float32).astype(np.float64)
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    net.forward()
    net.loss_and_grad(tgt)
    trace = []
    net.backward(trace)
    torch.cuda.synchronize()

    ws = [_host(w) for w in net.wb]  # the bf16 weights the kernels used
    bs = [b.cpu().numpy().astype(np.float64) for b in net.b32]
    acts = [_host(a) for a in net.acts]
    last = len(S.LAYERS) - 1
    for li in range(last):
        want = CO.bf16_round(CO.conv3x3(acts[li], ws[li], bs[li], relu=True))
        _close_bf16(acts[li + 1], want, ("forward", li))
    y = CO.conv3x3(acts[last], ws[last], bs[last])
    out = _host(net.out)
    terms = CO.conv3x3(np.abs(acts[last]), np.abs(ws[last]), np.abs(bs[last]))
    assert np.all(np.abs(out - y) <= 1e-4 * terms + 1e-30), "last layer"

    loss, g = CO.mse(out.reshape(-1, 16)[:, :4], target)
    assert abs(float(net.loss.cpu()) - loss) <= 1e-6 * loss
    g16 = np.zeros((H, W, 16))
    g16[:, :, :4] = g.reshape(H, W, 4)
    _close_bf16(_host(net.grad_out), CO.bf16_round(g16), "loss gradient")

    for k, li in enumerate(range(last, -1, -1)):
        dz = _host(trace[k])
        dw, db = CO.conv3x3_grad_weight(acts[li], dz)
        aw, _ = CO.conv3x3_grad_weight(np.abs(acts[li]), np.abs(dz))
        gw, gb = net.dw[li].cpu().numpy(), net.db[li].cpu().numpy()
        assert np.all(np.abs(gw - dw) <= 1e-4 * aw + 1e-30), ("weight gradient", li)
        assert np.all(np.abs(gb - db) <= 1e-4 * np.abs(dz).reshape(-1, dz.shape[2]).sum(0) + 1e-30), ("bias", li)
        if li > 0:
            want = CO.bf16_round(np.where(acts[li] > 0, CO.conv3x3_grad_input(dz, ws[li]), 0.0))
            _close_bf16(_host(trace[k + 1]), want, ("backward data", li))
