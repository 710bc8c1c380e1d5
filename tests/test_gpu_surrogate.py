"""The surrogate network end to end on the GPU: gradients of all eight layers against an FP64 CPU
network that rounds to bf16 at the same points (activations, loss gradient, backward-data outputs)."""
import numpy as np
import pytest

from oracle import conv_oracle as CO
from paper_1904_10070_gb300 import surrogate as S
from paper_1904_10070_gb300 import vlb

pytestmark = pytest.mark.gpu


def _host(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_network_gradients_match_cpu_oracle():
    import torch
    H, W = 4, 128
    net = S.SurrogateNet(H, W, seed=3)
    rng = np.random.default_rng(4)
    feat = np.zeros((H, W, 16))
    feat[:, :, :10] = rng.normal(size=(H, W, 10))
    feat = CO.bf16_round(feat)
    net.acts[0].copy_(torch.tensor(feat, dtype=torch.bfloat16, device="cuda"))
    target = rng.normal(size=(H * W, 4)).astype(np.float32).astype(np.float64)
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    net.forward()
    net.loss_and_grad(tgt)
    net.backward()
    torch.cuda.synchronize()

    ws = [_host(w) for w in net.wb]  # the bf16 weights the kernels used
    bs = [b.cpu().numpy().astype(np.float64) for b in net.b32]
    acts = [feat]
    last = len(S.LAYERS) - 1
    for li in range(last):
        acts.append(CO.bf16_round(CO.conv3x3(acts[-1], ws[li], bs[li], relu=True)))
    y = CO.conv3x3(acts[-1], ws[last], bs[last])
    np.testing.assert_allclose(_host(net.out), y, rtol=1e-3, atol=1e-3 * np.max(np.abs(y)))
    _, g = CO.mse(y.reshape(-1, 16)[:, :4], target)
    dz = np.zeros((H, W, 16))
    dz[:, :, :4] = g.reshape(H, W, 4)
    dz = CO.bf16_round(dz)
    for li in range(last, -1, -1):
        dw, db = CO.conv3x3_grad_weight(acts[li], dz)
        gw, gb = _host(net.dw[li]), net.db[li].cpu().numpy()
        rel = np.linalg.norm(gw - dw) / max(np.linalg.norm(dw), 1e-30)
        assert rel < 2e-2, (li, rel)
        assert np.linalg.norm(gb - db) <= 2e-2 * max(np.linalg.norm(db), 1e-30), li
        if li > 0:
            dz = CO.bf16_round(np.where(acts[li] > 0, CO.conv3x3_grad_input(dz, ws[li]), 0.0))
