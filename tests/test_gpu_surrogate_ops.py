"""The surrogate's non-convolution kernels and its advance loop, on the GPU.

Statistics, features, targets and outputs are checked against their definitions evaluated in
numpy; the comparison of snapshots is exact.  The advance loop is checked where its result is
fixed without a trained network: a judge that rejects every prediction leaves exactly the plain
solver's trajectory (bit for bit), and one that accepts every prediction keeps the conserved totals."""
import math

import numpy as np
import pytest

from oracle import conv_oracle as CO
from paper_1904_10070_gb300 import surrogate as S
from paper_1904_10070_gb300 import vlb

pytestmark = pytest.mark.gpu


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32), device="cuda")


def _snap(rng, N):
    s = np.empty((N, 4))
    s[:, 0] = np.tanh(3 * rng.uniform(-1, 1, N))
    s[:, 1] = 1.0 + 0.01 * rng.normal(size=N)
    s[:, 2:] = 0.02 * rng.normal(size=(N, 2))
    return s.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("fixed", [False, True])
def test_norm_statistics(fixed):
    import torch
    rng = np.random.default_rng(1)
    N = 3000
    s = _snap(rng, N)
    g = [0.5, 2.0, 3.0, 4.0]
    sn, su = (0.3, 0.7) if fixed else (0.0, 0.0)
    norm = S.Normaliser(sn, su, g)
    out = torch.empty(8, dtype=torch.float32, device="cuda")
    norm(_dev(s), out)
    got = out.cpu().numpy().astype(np.float64)
    n_mean = s[:, 1].mean()
    want4 = [n_mean, math.sqrt(np.mean(s[:, 0] ** 2)),
             sn if fixed else math.sqrt(np.mean((s[:, 1] - n_mean) ** 2)),
             su if fixed else math.sqrt(0.5 * np.mean(s[:, 2] ** 2 + s[:, 3] ** 2))]
    want = want4 + [g[0] * want4[1], g[1] * want4[2], g[2] * want4[3], g[3] * want4[3]]
    np.testing.assert_allclose(got, want, rtol=2e-6)
    s[7, 2] = np.nan
    norm(_dev(s), out)
    assert np.all(np.isnan(out.cpu().numpy()))


def test_features_targets_apply():
    import torch
    rng = np.random.default_rng(2)
    H, W = 6, 128
    N = H * W
    a = 1.0 / 2.7
    s = _snap(rng, N)
    after = s + 0.01 * rng.normal(size=s.shape)
    after = after.astype(np.float32).astype(np.float64)
    norm4 = np.array([1.001, 0.8, 0.01, 0.02], np.float32).astype(np.float64)
    d_norm = _dev(np.concatenate([norm4, [0.1, 0.2, 0.3, 0.4]]))
    feat = torch.empty((H, W, 16), dtype=torch.bfloat16, device="cuda")
    vlb.vlb_surrogate_features(H, W, a, _dev(s), d_norm, feat, _stream())
    th = (2 * np.pi * np.arange(H) / H)[:, None] * np.ones((1, W))
    J = 1 + a * np.cos(th)
    want = np.zeros((H, W, 16))
    sh = s.reshape(H, W, 4)
    want[..., 0] = sh[..., 0] / norm4[1]
    want[..., 1] = (sh[..., 1] - norm4[0]) / norm4[2]
    want[..., 2] = sh[..., 2] / norm4[3]
    want[..., 3] = sh[..., 3] / norm4[3]
    want[..., 4], want[..., 5], want[..., 6] = J, np.sin(th) / J, np.sin(th)
    want[..., 7], want[..., 8], want[..., 9] = np.cos(th), 1 / J, a
    got = feat.float().cpu().numpy().astype(np.float64)
    # bf16 of an FP32 value within a few FP32 units of the exact one: at most one bf16 unit apart
    # (the absolute floor covers sin(pi) = 0 on the device against 1.2e-16 in numpy)
    assert np.all(np.abs(got - CO.bf16_round(want)) <= 2.0 ** -7 * np.abs(want) + 1e-6)

    tgt = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    vlb.vlb_surrogate_targets(N, _dev(s), _dev(after), d_norm[4:], tgt, _stream())
    scale = np.array([0.1, 0.2, 0.3, 0.4])
    np.testing.assert_allclose(tgt.cpu().numpy(), (after - s) / scale, rtol=1e-5, atol=1e-7)
    pred16 = np.zeros((N, 16))
    pred16[:, :4] = rng.normal(size=(N, 4))
    out = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    vlb.vlb_surrogate_apply(N, _dev(s), _dev(pred16), d_norm[4:], out, _stream())
    np.testing.assert_allclose(out.cpu().numpy(), s + scale * pred16[:, :4], rtol=1e-6, atol=1e-7)


def test_snapshot_compare():
    import torch
    rng = np.random.default_rng(3)
    N = 100003
    a, b = _snap(rng, N), _snap(rng, N)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    work = torch.empty(vlb.vlb_reduce_workspace_bytes(), dtype=torch.uint8, device="cuda")
    vlb.vlb_snapshot_compare(N, _dev(a), _dev(b), work, out, _stream())
    got = out.cpu().numpy()
    d = a[:, 0] - b[:, 0]
    # maxima exact (FP32 difference of FP32 values), sums to FP64 rounding
    assert got[0] == float(np.abs(a[:, 0].astype(np.float32) - b[:, 0].astype(np.float32)).max())
    assert got[1] == float(np.abs(b[:, 0]).max())
    np.testing.assert_allclose(got[2:], [np.sum(d * d), np.sum(b[:, 0] ** 2)], rtol=1e-12)
    a[N - 1, 3] = np.inf
    vlb.vlb_snapshot_compare(N, _dev(a), _dev(b), work, out, _stream())
    got = out.cpu().numpy()
    assert got[0] == np.inf and got[2] == np.inf


def _solver(H, W, seed, own_stream=False):
    import torch
    p = S.member_params(2.5, H, W)
    s = vlb.Solver(vlb.make_params(**p, precision=vlb.FP32), stream=torch.cuda.Stream() if own_stream else None)
    phi = S.initial_phi(seed, H, W)
    z = np.zeros_like(phi)
    s.set_fields(np.ones_like(phi), z, z, phi)
    return s


def _trainer(H, W):
    net = S.SurrogateNet(H, W, seed=5)
    return S.Trainer(net, [0.1, 0.1, 0.1, 0.1], 1e-3, 1e-3)


@pytest.mark.parametrize("own_stream", [False, True])
def test_advance_rejecting_judge_reproduces_the_solver_bit_for_bit(own_stream):
    H, W = 16, 128
    ref, sur = _solver(H, W, 7), _solver(H, W, 7, own_stream)
    adv = S.Advancer(_trainer(H, W), sur, window=10, check_every=2, phi_tol=0.0)
    kinds = adv.advance(10)
    assert kinds == ["surrogate", "fallback", "solver", "solver"] * 2 + ["surrogate", "fallback"]
    ref.step(10 * len(kinds))
    f_ref, p_ref = ref.get_state()
    f_sur, p_sur = sur.get_state()
    np.testing.assert_array_equal(f_sur, f_ref)
    np.testing.assert_array_equal(p_sur, p_ref)


def test_advance_accepting_judge_conserves_totals():
    H, W = 16, 128
    s = _solver(H, W, 8, own_stream=True)
    t0 = s.totals()
    adv = S.Advancer(_trainer(H, W), s, window=10, check_every=3, phi_tol=math.inf)
    kinds = adv.advance(7)
    assert kinds == ["surrogate", "surrogate", "checked", "surrogate", "surrogate", "checked", "surrogate"]
    assert adv.graph is not None  # the later predicted windows replayed the captured graph
    t1 = s.totals()
    assert abs(t1[0] - t0[0]) <= 1e-6 * abs(t0[0])
    assert abs(t1[1] - t0[1]) <= 1e-5 * abs(t0[0])
    assert all(np.isfinite(adv.errors)) and all(np.isfinite(adv.errors_linf))


def test_graph_replay_matches_eager_prediction():
    """A predicted window replayed from the captured graph gives the same state as an eager one."""
    import torch
    H, W = 16, 128
    tr = _trainer(H, W)
    a, b = _solver(H, W, 9, own_stream=True), _solver(H, W, 9, own_stream=True)
    ea = S.Advancer(tr, a, window=10, check_every=0, graph=False)
    ga = S.Advancer(tr, b, window=10, check_every=0, graph=True)
    ea.advance(4)
    torch.cuda.synchronize()  # both advancers share the network's buffers
    ga.advance(4)
    assert ga.graph is not None and ea.graph is None
    fa, pa = a.get_state()
    fb, pb = b.get_state()
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(pa, pb)
