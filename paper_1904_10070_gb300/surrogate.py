"""Learned surrogate for blocks of solver steps (not part of the paper's method).

An 8-layer periodic-padding CNN -- 3x3 kernels, 64 hidden channels, ReLU -- maps the state of a torus
(phi, n, u_theta, u_phi plus six geometry channels) to its change over a window of solver steps.
It is trained on solver trajectories and used with the solver as fallback and judge.

This module only orchestrates: every tensor operation runs in libvlb's CUDA kernels (tensor-core
BF16 convolutions with FP32 accumulation, loss, Adam, features, snapshots); PyTorch allocates the
device memory.  Layer shapes: input 10 channels padded to 16, six 64 -> 64 layers, output 4
channels padded to 16 (the padding weights are zero and receive zero gradient).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, vlb

LAYERS = [(16, 64)] + [(64, 64)] * 6 + [(64, 16)]
N_IN, N_OUT = 10, 4


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class SurrogateNet:
    """Weights, optimiser state and activation buffers of the network for an H x W torus grid."""

    def __init__(self, H: int, W: int, seed: int = 0):
        import torch
        self.H, self.W = H, W
        rng = np.random.default_rng(seed)
        dev = "cuda"
        self.w32, self.b32, self.wb, self.wf = [], [], [], []
        self.mw, self.vw, self.mb, self.vb, self.dw, self.db = [], [], [], [], [], []
        for li, (cin, cout) in enumerate(LAYERS):
            fan_in = 9 * (N_IN if li == 0 else cin)
            w = rng.normal(size=(cout, 3, 3, cin)) * math.sqrt(2.0 / fan_in)
            if li == 0:
                w[:, :, :, N_IN:] = 0.0
            if li == len(LAYERS) - 1:
                w *= 0.1
                w[N_OUT:] = 0.0
            t = torch.tensor(w, dtype=torch.float32, device=dev)
            self.w32.append(t)
            self.b32.append(torch.zeros(cout, dtype=torch.float32, device=dev))
            self.wb.append(torch.empty((cout, 3, 3, cin), dtype=torch.bfloat16, device=dev))
            vlb.vlb_to_bf16(t.numel(), t, self.wb[-1], _stream())
            self.wf.append(torch.empty((cin, 3, 3, cout), dtype=torch.bfloat16, device=dev))
            for lst, shape in ((self.mw, t.shape), (self.vw, t.shape), (self.dw, t.shape)):
                lst.append(torch.zeros(shape, dtype=torch.float32, device=dev))
            for lst in (self.mb, self.vb, self.db):
                lst.append(torch.zeros(cout, dtype=torch.float32, device=dev))
        self.acts = [torch.empty((H, W, 16), dtype=torch.bfloat16, device=dev)]
        self.acts += [torch.empty((H, W, 64), dtype=torch.bfloat16, device=dev) for _ in range(len(LAYERS) - 1)]
        self.out = torch.empty((H, W, 16), dtype=torch.float32, device=dev)
        self.grad_out = torch.empty((H, W, 16), dtype=torch.bfloat16, device=dev)
        self.dz = [torch.empty((H, W, 64), dtype=torch.bfloat16, device=dev) for _ in range(2)]
        wsb = max(vlb.vlb_conv3x3_wgrad_workspace_bytes(H, W, ci, co) for ci, co in LAYERS)
        self.wg_ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        self.red_ws = torch.empty(vlb.vlb_reduce_workspace_bytes(), dtype=torch.uint8, device=dev)
        self.loss = torch.empty(1, dtype=torch.float64, device=dev)
        self.t = 0

    def forward(self):
        """acts[0] (bf16 features) -> out (f32, 16 channels, first 4 = predicted scaled change)."""
        st = _stream()
        last = len(LAYERS) - 1
        for li, (cin, cout) in enumerate(LAYERS):
            vlb.vlb_conv3x3_fwd(self.H, self.W, cin, cout, self.acts[li], self.wb[li], self.b32[li], None,
                                li < last, self.acts[li + 1] if li < last else None,
                                self.out if li == last else None, st)

    def loss_and_grad(self, target):
        vlb.vlb_mse_loss(self.H * self.W, self.out, target, self.grad_out, self.red_ws, self.loss, _stream())

    def backward(self):
        st = _stream()
        dz = self.grad_out
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout = LAYERS[li]
            vlb.vlb_conv3x3_bwd_weight(self.H, self.W, cin, cout, self.acts[li], dz, self.dw[li], self.db[li],
                                       self.wg_ws, st)
            if li > 0:
                vlb.vlb_conv3x3_flip(cin, cout, self.wb[li], self.wf[li], st)
                nxt = self.dz[li % 2]
                # dZ_{l-1} = (W_l^T dZ_l) * (A_{l-1} > 0): the forward kernel with flipped weights and mask
                vlb.vlb_conv3x3_fwd(self.H, self.W, cout, cin, dz, self.wf[li], None, self.acts[li], 0, nxt, None,
                                    st)
                dz = nxt

    def adam(self, lr: float):
        st = _stream()
        self.t += 1
        for li in range(len(LAYERS)):
            vlb.vlb_adam_step(self.w32[li].numel(), self.w32[li], self.dw[li], self.mw[li], self.vw[li], self.t, lr,
                              0.9, 0.999, 1e-8, self.wb[li], st)
            vlb.vlb_adam_step(self.b32[li].numel(), self.b32[li], self.db[li], self.mb[li], self.vb[li], self.t, lr,
                              0.9, 0.999, 1e-8, None, st)

    def parameters(self):
        return sum(int(w.numel()) + int(b.numel()) for w, b in zip(self.w32, self.b32))


# ------------------------------------------------------------------------------------------------
# Workload and dataset
# ------------------------------------------------------------------------------------------------

def member_params(R: float, H: int = 256, W: int = 512, dt_factor: float = 0.5) -> dict:
    """Coarsening member of the surrogate workload: r = 1, the given R, FP32 UW3 hydrodynamic,
    A = 0.5, kappa = 5e-4, M = 2.5e-3, tau = 0.6, dt = dt_factor x the stable step."""
    p = dict(geometry=0, R=R, r=1.0, n_theta=H, n_phi=W, dt=1.0, tau=0.6, M=2.5e-3, A=0.5, kappa=5e-4, advection=0,
             ch_mode=0)
    p["dt"] = dt_factor * vlb.vlb_max_stable_dt(vlb.make_params(**p))
    return p


def radius_for(seed: int) -> float:
    """R ~ U[1.5, 4] from the counter-based generator (r = 1)."""
    return 1.5 + 2.5 * float(inputs.uniform01(seed, 1, 1)[0, 0])


class Dataset:
    """Pairs (snapshot at t, snapshot at t + window) from solver trajectories, kept on the device,
    with the per-sample input normalisation (n_mean, s_phi, s_n, s_u) of each `before` snapshot."""

    def __init__(self, before, after, radii, norms):
        self.before, self.after, self.radii, self.norms = before, after, radii, norms

    def __len__(self):
        return len(self.radii)


class Normaliser:
    """Per-snapshot scales from FP64 channel sums (one small device reduction and read-back)."""

    def __init__(self):
        import torch
        self.work = torch.empty(vlb.vlb_reduce_workspace_bytes(), dtype=torch.uint8, device="cuda")
        self.sums = torch.empty(8, dtype=torch.float64, device="cuda")

    def __call__(self, snap):
        N = snap.shape[0]
        vlb.vlb_channel_sums(N, 4, snap, self.work, self.sums, _stream())
        s = self.sums.cpu().numpy()
        mean, sq = s[:4] / N, s[4:] / N
        s_phi = math.sqrt(max(sq[0], 0.0))
        s_n = math.sqrt(max(sq[1] - mean[1] ** 2, 0.0))
        s_u = math.sqrt(max(0.5 * (sq[2] + sq[3]), 0.0))
        if not np.all(np.isfinite(s)):
            return (float("nan"),) * 4
        return (float(mean[1]), max(s_phi, 1e-12), max(s_n, 1e-12), max(s_u, 1e-12))


def generate(seeds, H=256, W=512, window=50, pairs=5, spacing=100, batch=48, noise=0.01):
    """Runs one trajectory per seed (batched through the ensemble path) and keeps `pairs` windows of
    each: snapshots at steps k * spacing and k * spacing + window, k = 0 .. pairs - 1."""
    import torch
    N = H * W
    norm = Normaliser()
    before, after, radii, norms = [], [], [], []
    for i0 in range(0, len(seeds), batch):
        sel = seeds[i0:i0 + batch]
        ps = [member_params(radius_for(s), H, W) for s in sel]
        ens = vlb.Ensemble([vlb.make_params(**p, precision=vlb.FP32) for p in ps])
        for v, s in zip(ens.views, sel):
            phi = inputs.noise(s, H, W, noise)
            z = np.zeros_like(phi)
            vlb.vlb_set_fields(v, np.ones_like(phi), z, z, phi)
        snaps = {}
        marks = sorted({k * spacing for k in range(pairs)} | {k * spacing + window for k in range(pairs)})
        done = 0
        for m in marks:
            if m > done:
                ens.step(m - done)
                done = m
            snaps[m] = [torch.empty((N, 4), dtype=torch.float32, device="cuda") for _ in sel]
            for v, buf in zip(ens.views, snaps[m]):
                vlb.vlb_get_snapshot(v, buf)
        torch.cuda.synchronize()
        for j, s in enumerate(sel):
            for k in range(pairs):
                before.append(snaps[k * spacing][j])
                after.append(snaps[k * spacing + window][j])
                radii.append(ps[j]["R"])
                norms.append(norm(before[-1]))
        ens.close()
        del snaps
    return Dataset(before, after, radii, norms)


def target_ratios(ds: Dataset, sample: int = 64):
    """g_c = mean over a sample of rms(change of channel c) / (its input scale): targets are then O(1)."""
    import torch
    N = ds.before[0].shape[0]
    tgt = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    norm = Normaliser()
    idx = np.linspace(0, len(ds) - 1, min(sample, len(ds))).astype(int)
    acc = np.zeros(4)
    for i in idx:
        _, s_phi, s_n, s_u = ds.norms[i]
        vlb.vlb_surrogate_targets(N, ds.before[i], ds.after[i], [s_phi, s_n, s_u, s_u], tgt, _stream())
        vlb.vlb_channel_sums(N, 4, tgt, norm.work, norm.sums, _stream())
        sq = norm.sums.cpu().numpy()[4:] / N
        acc += np.sqrt(np.maximum(sq, 0.0))
    return [float(max(x / len(idx), 1e-6)) for x in acc]


class Trainer:
    def __init__(self, net: SurrogateNet, ratios):
        import torch
        self.net = net
        self.g = list(ratios)
        N = net.H * net.W
        self.target = torch.empty((N, 4), dtype=torch.float32, device="cuda")

    def out_scale(self, norm):
        _, s_phi, s_n, s_u = norm
        return [self.g[0] * s_phi, self.g[1] * s_n, self.g[2] * s_u, self.g[3] * s_u]

    def sample_loss(self, before, after, R, norm, train: bool, lr: float = 1e-3):
        net, st = self.net, _stream()
        N = net.H * net.W
        vlb.vlb_surrogate_features(net.H, net.W, 1.0 / R, before, norm, net.acts[0], st)
        vlb.vlb_surrogate_targets(N, before, after, self.out_scale(norm), self.target, st)
        net.forward()
        net.loss_and_grad(self.target)
        if train:
            net.backward()
            net.adam(lr)
        return net.loss

    def fit(self, ds: Dataset, epochs: int, lr: float = 1e-3, seed: int = 0, log_every: int = 0):
        import torch
        rng = np.random.default_rng(seed)
        hist = []
        n_it = epochs * len(ds)
        t0 = time.perf_counter()
        it = 0
        for ep in range(epochs):
            for i in rng.permutation(len(ds)):
                lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / n_it))  # cosine schedule
                loss = self.sample_loss(ds.before[i], ds.after[i], ds.radii[i], ds.norms[i], True, lr_t)
                it += 1
                if log_every and it % log_every == 0:
                    hist.append((it, float(loss.cpu())))
        torch.cuda.synchronize()
        return hist, time.perf_counter() - t0

    def evaluate(self, ds: Dataset):
        vals = [float(self.sample_loss(ds.before[i], ds.after[i], ds.radii[i], ds.norms[i], False).cpu())
                for i in range(len(ds))]
        return float(np.mean(vals))


# ------------------------------------------------------------------------------------------------
# Surrogate-accelerated stepping with the solver as fallback and judge
# ------------------------------------------------------------------------------------------------

class Advancer:
    """Advances a solver (FP32 handle) by windows of `window` steps with the network.

    Every `check_every` windows the solver itself runs the window from the unchanged state and its
    phi is compared with the prediction: a relative L-infinity error above `phi_tol` keeps the
    solver's result (a fallback), otherwise the prediction is taken.  A prediction whose free energy
    Psi rises is replaced by a solver window too.  A taken prediction restarts the solver at
    f = f^eq(n, u) with int n sqrt(g) and int phi sqrt(g) projected back to their values before the
    window (vlb_set_snapshot).
    """

    def __init__(self, trainer: Trainer, solver: vlb.Solver, window: int = 50):
        import torch
        self.tr, self.s, self.window = trainer, solver, window
        self.R = solver.p.R
        N = solver.p.n_theta * solver.p.n_phi
        self.snap = torch.empty((N, 4), dtype=torch.float32, device="cuda")
        self.pred = torch.empty((N, 4), dtype=torch.float32, device="cuda")
        self.check = torch.empty((N, 4), dtype=torch.float32, device="cuda")
        self.normaliser = Normaliser()
        self.fallbacks = 0
        self.checks = 0
        self.max_check_err = 0.0

    def predict(self):
        """pred := the network's estimate of the state one window ahead of the solver's state."""
        net, st = self.tr.net, _stream()
        vlb.vlb_get_snapshot(self.s.h, self.snap)
        norm = self.normaliser(self.snap)
        vlb.vlb_surrogate_features(net.H, net.W, 1.0 / self.R, self.snap, norm, net.acts[0], st)
        net.forward()
        vlb.vlb_surrogate_apply(net.H * net.W, self.snap, net.out, self.tr.out_scale(norm), self.pred, st)

    def window_step(self, k: int, check_every: int, phi_tol: float) -> str:
        s = self.s
        tot = s.totals()
        self.predict()
        if not all(math.isfinite(x) for x in self.normaliser(self.pred)):  # unusable prediction
            self.fallbacks += 1
            s.step(self.window)
            return "fallback"
        if check_every > 0 and (k + 1) % check_every == 0:
            s.step(self.window)  # the judge: the solver over the same window from the same state
            vlb.vlb_get_snapshot(s.h, self.check)
            pc = self.check[:, 0].cpu().numpy().astype(np.float64)
            pp = self.pred[:, 0].cpu().numpy().astype(np.float64)
            err = float(np.max(np.abs(pp - pc)) / max(np.max(np.abs(pc)), 1e-30))
            self.checks += 1
            self.max_check_err = max(self.max_check_err, err)
            if err > phi_tol:
                self.fallbacks += 1
                return "fallback"
        vlb.vlb_set_snapshot(s.h, self.pred, (tot[0], tot[1]))
        if s.totals()[2] > tot[2] * (1.0 + 1e-3) + 1e-12:  # Psi rose: redo the window with the solver
            self.fallbacks += 1
            vlb.vlb_set_snapshot(s.h, self.snap, (tot[0], tot[1]))
            s.step(self.window)
            return "fallback"
        return "surrogate"
