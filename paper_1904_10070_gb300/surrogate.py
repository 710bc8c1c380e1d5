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

    def backward(self, trace=None):
        """Weight and bias gradients of every layer; `trace` (a list) receives a copy of the gradient
        entering each layer, last layer first."""
        st = _stream()
        dz = self.grad_out
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout = LAYERS[li]
            if trace is not None:
                trace.append(dz.clone())
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


CORR_CELLS, WALL_CELLS = 4.0, 1.8


def initial_phi(seed: int, H: int, W: int, corr: float = CORR_CELLS) -> np.ndarray:
    """Start of a surrogate trajectory: seeded noise quenched into domains about `corr` cells across
    (inputs.quenched_noise); the default is a torus early in coarsening, larger values stand for later
    stages."""
    return inputs.quenched_noise(seed, H, W, corr, WALL_CELLS)


def corr_for(seed: int, lo: float, hi: float) -> float:
    """Domain scale of a training trajectory, uniform in [lo, hi] from the counter-based generator
    (an element of the seed's stream other than the one radius_for uses)."""
    return lo + (hi - lo) * float(inputs.uniform01(seed, 1, 2)[0, 1])


class Normaliser:
    """Input statistics of a snapshot on the device (vlb_surrogate_norm): fills an 8-float device
    array (n_mean, s_phi, s_n, s_u, then the output scales g_c s_c) without a host read-back."""

    def __init__(self, s_n: float = 0.0, s_u: float = 0.0, g=None):
        import torch
        self.work = torch.empty(vlb.vlb_reduce_workspace_bytes(), dtype=torch.uint8, device="cuda")
        self.sums = torch.empty(8, dtype=torch.float64, device="cuda")
        self.s_n, self.s_u, self.g = s_n, s_u, g

    def __call__(self, snap, out8):
        vlb.vlb_surrogate_norm(snap.shape[0], snap, self.s_n, self.s_u, self.g, self.work, self.sums, out8, _stream())

    def host(self, snap):
        """(n_mean, s_phi, s_n, s_u) of one snapshot, read back."""
        import torch
        out = torch.empty(8, dtype=torch.float32, device="cuda")
        self(snap, out)
        return tuple(float(x) for x in out[:4].cpu())


class Dataset:
    """Pairs (snapshot at t, snapshot at t + window) from solver trajectories, kept on the device.
    stats[i] = (n_mean, s_phi, rms(n - n_mean), rms|u|/sqrt2) of before[i]; s_n and s_u, the medians of
    the last two over the set, are the fixed input scales of n and u (per-snapshot values vanish at
    rest)."""

    def __init__(self, before, after, radii, stats):
        self.before, self.after, self.radii, self.stats = before, after, radii, stats
        self.s_n = float(np.median([t[2] for t in stats]))
        self.s_u = float(np.median([t[3] for t in stats]))
        self.norm8 = None  # per-pair device normalisation, filled by a Trainer

    def __len__(self):
        return len(self.radii)


def generate(seeds, H=256, W=512, window=50, pairs=8, spacing=100, start=100, batch=48, corr=None):
    """Runs one trajectory per seed from initial_phi(seed) at rest (batched through the ensemble path)
    and keeps `pairs` windows of each: snapshots at steps start + k spacing and start + k spacing +
    window, k = 0 .. pairs - 1.  corr = (lo, hi) draws each trajectory's initial domain scale from
    corr_for (larger domains stand for later coarsening); None keeps CORR_CELLS."""
    import torch
    N = H * W
    stat = Normaliser()
    before, after, radii, stats = [], [], [], []
    for i0 in range(0, len(seeds), batch):
        sel = seeds[i0:i0 + batch]
        ps = [member_params(radius_for(s), H, W) for s in sel]
        ens = vlb.Ensemble([vlb.make_params(**p, precision=vlb.FP32) for p in ps])
        for v, s in zip(ens.views, sel):
            phi = initial_phi(s, H, W, CORR_CELLS if corr is None else corr_for(s, *corr))
            z = np.zeros_like(phi)
            vlb.vlb_set_fields(v, np.ones_like(phi), z, z, phi)
        snaps = {}
        firsts = [start + k * spacing for k in range(pairs)]
        marks = sorted(set(firsts) | {m + window for m in firsts})
        done = 0
        for m in marks:
            if m > done:
                ens.step(m - done)
                done = m
            snaps[m] = [torch.empty((N, 4), dtype=torch.float32, device="cuda") for _ in sel]
            for v, buf in zip(ens.views, snaps[m]):
                vlb.vlb_get_snapshot(v, buf)
        for j, s in enumerate(sel):
            for m in firsts:
                before.append(snaps[m][j])
                after.append(snaps[m + window][j])
                radii.append(ps[j]["R"])
                stats.append(stat.host(before[-1]))
        ens.close()
        del snaps
    return Dataset(before, after, radii, stats)


def target_ratios(ds: Dataset, sample: int = 64):
    """g_c = mean over a sample of rms(change of channel c over the window) / (input scale of c), so
    that the targets are O(1)."""
    import torch
    N = ds.before[0].shape[0]
    tgt = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    norm = Normaliser(ds.s_n, ds.s_u)
    n8 = torch.empty(8, dtype=torch.float32, device="cuda")
    sums = torch.empty(8, dtype=torch.float64, device="cuda")
    idx = np.linspace(0, len(ds) - 1, min(sample, len(ds))).astype(int)
    acc = np.zeros(4)
    for i in idx:
        norm(ds.before[i], n8)
        vlb.vlb_surrogate_targets(N, ds.before[i], ds.after[i], n8[4:], tgt, _stream())
        vlb.vlb_channel_sums(N, 4, tgt, norm.work, sums, _stream())
        sq = sums.cpu().numpy()[4:] / N
        acc += np.sqrt(np.maximum(sq, 0.0))
    return [float(max(x / len(idx), 1e-6)) for x in acc]


class Trainer:
    """Fits the network to a Dataset.  Inputs are the snapshot scaled by (n_mean, s_phi, s_n, s_u);
    targets are the window's change divided by g_c times the input scale of channel c."""

    def __init__(self, net: SurrogateNet, ratios, s_n: float, s_u: float, weights=(1.0, 1.0, 1.0, 1.0)):
        import torch
        self.net = net
        # a loss weight w_c on channel c is a target scaled by w_c: g_c -> g_c / w_c
        self.g = [float(x) / float(w) for x, w in zip(ratios, weights)]
        self.s_n, self.s_u = float(s_n), float(s_u)
        self.normaliser = Normaliser(self.s_n, self.s_u, self.g)
        self.target = torch.empty((net.H * net.W, 4), dtype=torch.float32, device="cuda")

    def prepare(self, ds: Dataset):
        import torch
        if ds.norm8 is None or getattr(ds, "norm_key", None) != (self.s_n, self.s_u, tuple(self.g)):
            ds.norm8 = torch.empty((len(ds), 8), dtype=torch.float32, device="cuda")
            for i in range(len(ds)):
                self.normaliser(ds.before[i], ds.norm8[i])
            ds.norm_key = (self.s_n, self.s_u, tuple(self.g))

    def sample_loss(self, ds: Dataset, i: int, train: bool, lr: float = 1e-3):
        net, st = self.net, _stream()
        N = net.H * net.W
        vlb.vlb_surrogate_features(net.H, net.W, 1.0 / ds.radii[i], ds.before[i], ds.norm8[i], net.acts[0], st)
        vlb.vlb_surrogate_targets(N, ds.before[i], ds.after[i], ds.norm8[i, 4:], self.target, st)
        net.forward()
        net.loss_and_grad(self.target)
        if train:
            net.backward()
            net.adam(lr)
        return net.loss

    def fit(self, ds: Dataset, epochs: int, lr: float = 1e-3, seed: int = 0, log_every: int = 0):
        """Adam over the pairs in seeded random order with a cosine learning-rate schedule."""
        import torch
        self.prepare(ds)
        rng = np.random.default_rng(seed)
        hist = []
        n_it = epochs * len(ds)
        t0 = time.perf_counter()
        it = 0
        for _ in range(epochs):
            for i in rng.permutation(len(ds)):
                lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / n_it))
                loss = self.sample_loss(ds, int(i), True, lr_t)
                it += 1
                if log_every and it % log_every == 0:
                    hist.append((it, float(loss.cpu())))
        torch.cuda.synchronize()
        return hist, time.perf_counter() - t0

    def evaluate(self, ds: Dataset):
        self.prepare(ds)
        return float(np.mean([float(self.sample_loss(ds, i, False).cpu()) for i in range(len(ds))]))

    def predict(self, snap, R: float, norm8, out):
        """out := the network's estimate of snap one window ahead (all on the device)."""
        net, st = self.net, _stream()
        self.normaliser(snap, norm8)
        vlb.vlb_surrogate_features(net.H, net.W, 1.0 / R, snap, norm8, net.acts[0], st)
        net.forward()
        vlb.vlb_surrogate_apply(net.H * net.W, snap, net.out, norm8[4:], out, st)


# ------------------------------------------------------------------------------------------------
# Surrogate-accelerated stepping with the solver as fallback and judge (in the library)
# ------------------------------------------------------------------------------------------------

def export(trainer: Trainer):
    """The trained network as vlb_surrogate_create takes it: (bf16 weights of all layers concatenated,
    FP32 biases concatenated, s_n, s_u, g)."""
    import torch
    net = trainer.net
    w = torch.cat([t.reshape(-1) for t in net.wb]).contiguous()
    b = torch.cat([t.reshape(-1) for t in net.b32]).contiguous()
    return w, b, trainer.s_n, trainer.s_u, list(trainer.g)


class Advancer:
    """Advances an FP32 solver by windows of `window` steps, most of them with the network, through the
    library's vlb_surrogate_advance: every `check_every`-th window the solver judges the prediction by
    the relative L2 (norm="l2") or relative L-infinity (norm="linf") error of phi against `phi_tol`,
    keeping its own result, and rolls back and runs alone after a failed check (include/vlb.h has the
    full contract).  The network is copied from the trainer when the Advancer is made."""

    def __init__(self, trainer: Trainer, solver: vlb.Solver, window: int = 50, check_every: int = 4,
                 phi_tol: float = 1e-2, norm: str = "l2", graph: bool = True):
        if solver.p.precision != vlb.FP32:
            raise ValueError("the surrogate advances FP32 solvers")
        if norm not in ("l2", "linf"):
            raise ValueError("norm must be 'l2' or 'linf'")
        self.s, self.window = solver, window
        self.check_every, self.phi_tol, self.norm, self.use_graph = check_every, phi_tol, norm, graph
        w, b, s_n, s_u, g = export(trainer)
        self.sur = vlb.Surrogate(solver.p, w, b, s_n, s_u, g, window, stream=solver.stream)
        self.kinds, self.errors, self.errors_linf = [], [], []

    @property
    def graph(self):
        return True if self.sur.stats()["graph"] else None

    def advance(self, nwin: int):
        kinds, errs, _ = self.sur.advance(self.s.h, nwin, self.check_every, self.phi_tol,
                                          judge_linf=self.norm == "linf", graph=self.use_graph)
        for k, (e2, einf) in zip(kinds, errs):
            if k in ("checked", "fallback"):
                self.errors.append(float(e2))
                self.errors_linf.append(float(einf))
        self.kinds += kinds
        return kinds

    def window_step(self) -> str:
        return self.advance(1)[0]

    def close(self):
        self.sur.close()
