"""Thin ctypes binding of libvlb (include/vlb.h): argument marshalling only.

Every step of the time integration runs in the CUDA library; this module converts numpy
arrays to pointers, allocates the caller-owned device workspace with PyTorch and passes
PyTorch's current CUDA stream.  If the library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvlb.so")

VLB_OK, VLB_ERR_ARG, VLB_ERR_CUDA, VLB_ERR_UNSTABLE, VLB_ERR_TIMEOUT, VLB_ERR_WORKSPACE = 0, -1, -2, -3, -4, -5
TORUS, FLAT = 0, 1
FP64, FP32 = 0, 1
UW3, WENO5 = 0, 1
HYDRO, DIFFUSIVE = 0, 1

# every entry point declared in include/vlb.h
EXPORTS = ["vlb_workspace_bytes", "vlb_max_stable_dt", "vlb_create", "vlb_destroy", "vlb_set_fields",
           "vlb_set_state", "vlb_get_state", "vlb_step", "vlb_get_fields", "vlb_get_totals",
           "vlb_interface_length", "vlb_state_device", "vlb_steps_done", "vlb_last_error",
           "vlb_step_noalloc", "vlb_ensemble_workspace_bytes", "vlb_ensemble_create", "vlb_ensemble_step",
           "vlb_ensemble_member", "vlb_ensemble_tile_rows", "vlb_get_snapshot", "vlb_set_snapshot",
           "vlb_conv3x3_fwd", "vlb_conv3x3_flip", "vlb_conv3x3_wgrad_workspace_bytes", "vlb_conv3x3_bwd_weight",
           "vlb_reduce_workspace_bytes", "vlb_surrogate_norm", "vlb_surrogate_features", "vlb_surrogate_targets",
           "vlb_surrogate_apply", "vlb_snapshot_compare", "vlb_channel_sums", "vlb_mse_loss", "vlb_adam_step", "vlb_to_bf16",
           "vlb_conv_status", "vlb_test_raise_flag", "vlb_surrogate_workspace_bytes", "vlb_surrogate_create",
           "vlb_surrogate_advance", "vlb_surrogate_stats", "vlb_ensemble_configure", "vlb_ensemble_get_config",
           "vlb_structure_length", "vlb_set_schedule", "vlb_get_schedule", "vlb_test_wave_schedule",
           "vlb_test_wave_timeout"]

NOALLOC_SCRATCH_BYTES = 24 * 1024 * 1024


WINDOW_KINDS = {0: "surrogate", 1: "checked", 2: "fallback", 3: "solver"}
SUR_JUDGE_LINF, SUR_NO_GRAPH = 1, 2


class vlb_surrogate_net(ctypes.Structure):
    _fields_ = [("weights_bf16", ctypes.c_void_p), ("biases", ctypes.c_void_p), ("s_n", ctypes.c_float),
                ("s_u", ctypes.c_float), ("g", ctypes.c_float * 4), ("window", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


ENS_AUTO, ENS_BATCHED, ENS_PERSISTENT = 0, 1, 2


class vlb_ensemble_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("test_skip_cta", ctypes.c_int32), ("barrier_budget", ctypes.c_int64)]


class vlb_params(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("n_phi", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("advection", ctypes.c_int32), ("ch_mode", ctypes.c_int32),
                ("diag_every", ctypes.c_int32), ("ch_stab", ctypes.c_int32),
                ("R", ctypes.c_double), ("r", ctypes.c_double), ("dt", ctypes.c_double),
                ("tau", ctypes.c_double), ("M", ctypes.c_double), ("A", ctypes.c_double),
                ("kappa", ctypes.c_double)]


def make_params(R, r, n_theta, n_phi, dt, tau, M, A, kappa, geometry=TORUS, precision=FP64, advection=UW3,
                ch_mode=HYDRO, diag_every=0, ch_stab=0) -> vlb_params:
    return vlb_params(geometry=geometry, n_theta=n_theta, n_phi=n_phi, precision=precision, advection=advection,
                      ch_mode=ch_mode, diag_every=diag_every, ch_stab=ch_stab, R=R, r=r, dt=dt, tau=tau, M=M, A=A,
                      kappa=kappa)


class VlbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"vlb status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libvlb.so (built by paper_1904_10070_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1904_10070_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, D, I32, I64, S = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    PP = ctypes.POINTER(vlb_params)
    L.vlb_workspace_bytes.argtypes, L.vlb_workspace_bytes.restype = [PP], S
    L.vlb_max_stable_dt.argtypes, L.vlb_max_stable_dt.restype = [PP, D], I32
    L.vlb_create.argtypes, L.vlb_create.restype = [PP, P, S, P, ctypes.POINTER(P)], I32
    L.vlb_destroy.argtypes, L.vlb_destroy.restype = [P], I32
    L.vlb_set_fields.argtypes, L.vlb_set_fields.restype = [P, D, D, D, D], I32
    L.vlb_set_state.argtypes, L.vlb_set_state.restype = [P, D, D], I32
    L.vlb_get_state.argtypes, L.vlb_get_state.restype = [P, D, D], I32
    L.vlb_step.argtypes, L.vlb_step.restype = [P, I64], I32
    L.vlb_get_fields.argtypes, L.vlb_get_fields.restype = [P, D, D, D, D, D], I32
    L.vlb_get_totals.argtypes, L.vlb_get_totals.restype = [P, D], I32
    L.vlb_interface_length.argtypes, L.vlb_interface_length.restype = [P, D], I32
    L.vlb_structure_length.argtypes, L.vlb_structure_length.restype = [P, D], I32
    L.vlb_set_schedule.argtypes, L.vlb_set_schedule.restype = [P, ctypes.c_int32], I32
    L.vlb_get_schedule.argtypes, L.vlb_get_schedule.restype = [P, ctypes.POINTER(ctypes.c_int32)], I32
    L.vlb_test_wave_schedule.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.vlb_test_wave_schedule.restype = I32
    L.vlb_test_wave_timeout.argtypes, L.vlb_test_wave_timeout.restype = [P, ctypes.c_int32, I64], I32
    L.vlb_state_device.argtypes, L.vlb_state_device.restype = [P, ctypes.POINTER(P), ctypes.POINTER(I64)], I32
    L.vlb_steps_done.argtypes, L.vlb_steps_done.restype = [P, ctypes.POINTER(I64)], I32
    L.vlb_last_error.argtypes, L.vlb_last_error.restype = [P], ctypes.c_char_p
    L.vlb_step_noalloc.argtypes = [PP, P, I64, ctypes.c_double, I64, P, ctypes.POINTER(ctypes.c_char_p)]
    L.vlb_step_noalloc.restype = I32
    L.vlb_ensemble_workspace_bytes.argtypes, L.vlb_ensemble_workspace_bytes.restype = [PP, I32], S
    L.vlb_ensemble_create.argtypes, L.vlb_ensemble_create.restype = [PP, I32, P, S, P, ctypes.POINTER(P)], I32
    L.vlb_ensemble_step.argtypes, L.vlb_ensemble_step.restype = [P, I64], I32
    L.vlb_ensemble_member.argtypes, L.vlb_ensemble_member.restype = [P, I32, ctypes.POINTER(P)], I32
    F = ctypes.POINTER(ctypes.c_float)
    L.vlb_ensemble_tile_rows.argtypes = [P, ctypes.POINTER(I32), F, F]
    L.vlb_ensemble_tile_rows.restype = I32
    FP = ctypes.POINTER(ctypes.c_float)
    DP = ctypes.POINTER(ctypes.c_double)
    L.vlb_get_snapshot.argtypes, L.vlb_get_snapshot.restype = [P, P], I32
    L.vlb_set_snapshot.argtypes, L.vlb_set_snapshot.restype = [P, P, DP, I32], I32
    L.vlb_conv_status.argtypes, L.vlb_conv_status.restype = [P, I32], I32
    L.vlb_surrogate_workspace_bytes.argtypes, L.vlb_surrogate_workspace_bytes.restype = [PP], S
    L.vlb_surrogate_create.argtypes = [PP, ctypes.POINTER(vlb_surrogate_net), P, S, P, ctypes.POINTER(P)]
    L.vlb_surrogate_create.restype = I32
    L.vlb_surrogate_advance.argtypes = [P, P, I32, I32, ctypes.c_double, I32, ctypes.POINTER(I32), D,
                                        ctypes.POINTER(I32)]
    L.vlb_surrogate_advance.restype = I32
    L.vlb_surrogate_stats.argtypes, L.vlb_surrogate_stats.restype = [P, ctypes.POINTER(I64)], I32
    L.vlb_ensemble_configure.argtypes = [P, ctypes.POINTER(vlb_ensemble_config)]
    L.vlb_ensemble_configure.restype = I32
    L.vlb_ensemble_get_config.argtypes = [P, ctypes.POINTER(vlb_ensemble_config), ctypes.POINTER(ctypes.c_float)]
    L.vlb_ensemble_get_config.restype = I32
    L.vlb_test_raise_flag.argtypes, L.vlb_test_raise_flag.restype = [P, I32], I32
    L.vlb_conv3x3_fwd.argtypes = [I32, I32, I32, I32, P, P, P, P, I32, P, P, P]
    L.vlb_conv3x3_flip.argtypes = [I32, I32, P, P, P]
    L.vlb_conv3x3_wgrad_workspace_bytes.argtypes = [I32, I32, I32, I32]
    L.vlb_conv3x3_wgrad_workspace_bytes.restype = S
    L.vlb_conv3x3_bwd_weight.argtypes = [I32, I32, I32, I32, P, P, P, P, P, S, P]
    L.vlb_reduce_workspace_bytes.argtypes, L.vlb_reduce_workspace_bytes.restype = [], S
    L.vlb_surrogate_norm.argtypes = [I64, P, ctypes.c_float, ctypes.c_float, FP, P, P, P, P]
    L.vlb_surrogate_features.argtypes = [I32, I32, ctypes.c_double, P, P, P, P]
    L.vlb_surrogate_targets.argtypes = [I64, P, P, P, P, P]
    L.vlb_surrogate_apply.argtypes = [I64, P, P, P, P, P]
    L.vlb_snapshot_compare.argtypes = [I64, P, P, P, P, P]
    L.vlb_channel_sums.argtypes = [I64, I32, P, P, P, P]
    L.vlb_mse_loss.argtypes = [I64, P, P, P, P, P, P]
    L.vlb_adam_step.argtypes = [I64, P, P, P, P, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, P, P]
    L.vlb_to_bf16.argtypes = [I64, P, P, P]
    for name in ("vlb_conv3x3_fwd", "vlb_conv3x3_flip", "vlb_conv3x3_bwd_weight", "vlb_surrogate_norm",
                 "vlb_surrogate_features", "vlb_snapshot_compare",
                 "vlb_surrogate_targets", "vlb_surrogate_apply", "vlb_channel_sums", "vlb_mse_loss", "vlb_adam_step",
                 "vlb_to_bf16"):
        getattr(L, name).restype = I32
    _lib = L
    return L


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st: int, handle=None):
    if st != VLB_OK:
        msg = lib().vlb_last_error(handle).decode()
        raise VlbError(st, msg)


def vlb_workspace_bytes(p: vlb_params) -> int:
    return lib().vlb_workspace_bytes(ctypes.byref(p))


def vlb_max_stable_dt(p: vlb_params) -> float:
    out = ctypes.c_double()
    _check(lib().vlb_max_stable_dt(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def vlb_create(p: vlb_params, workspace_ptr: int, nbytes: int, stream_ptr: int):
    h = ctypes.c_void_p()
    _check(lib().vlb_create(ctypes.byref(p), ctypes.c_void_p(workspace_ptr), nbytes, ctypes.c_void_p(stream_ptr),
                            ctypes.byref(h)))
    return h


def vlb_destroy(h):
    _check(lib().vlb_destroy(h))


def vlb_set_fields(h, rho, ut, up, phi):
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, ut, up, phi)]
    _check(lib().vlb_set_fields(h, *[_dptr(x) for x in arrs]), h)


def vlb_set_state(h, f16, phi):
    f16 = np.ascontiguousarray(f16, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    _check(lib().vlb_set_state(h, _dptr(f16), _dptr(phi)), h)


def vlb_get_state(h, n_theta, n_phi):
    f16 = np.empty((16, n_theta, n_phi))
    phi = np.empty((n_theta, n_phi))
    _check(lib().vlb_get_state(h, _dptr(f16), _dptr(phi)), h)
    return f16, phi


def vlb_step(h, nsteps: int):
    _check(lib().vlb_step(h, nsteps), h)


def vlb_get_fields(h, n_theta, n_phi, out=None):
    """Returns (rho, u_theta, u_phi, phi, mu) as new arrays, or fills the 5 arrays in `out`."""
    arrs = out if out is not None else [np.empty((n_theta, n_phi)) for _ in range(5)]
    _check(lib().vlb_get_fields(h, *[_dptr(x) for x in arrs]), h)
    return tuple(arrs)


def vlb_get_totals(h) -> np.ndarray:
    out = np.empty(4)
    _check(lib().vlb_get_totals(h, _dptr(out)), h)
    return out


def vlb_interface_length(h) -> float:
    out = ctypes.c_double()
    _check(lib().vlb_interface_length(h, ctypes.byref(out)), h)
    return out.value


SCHED_AUTO, SCHED_STAGES, SCHED_WAVE = 0, 1, 2


def vlb_set_schedule(h, schedule: int):
    _check(lib().vlb_set_schedule(h, int(schedule)), h)


def vlb_get_schedule(h) -> int:
    out = ctypes.c_int32()
    _check(lib().vlb_get_schedule(h, ctypes.byref(out)), h)
    return out.value


def vlb_test_wave_schedule(n_bands: int, lag: int, nsteps: int) -> bool:
    """Host-only check of the wavefront ticket order (no GPU needed)."""
    return lib().vlb_test_wave_schedule(int(n_bands), int(lag), int(nsteps)) == 0


def vlb_test_wave_timeout(h, skip_cta: int, budget: int):
    _check(lib().vlb_test_wave_timeout(h, int(skip_cta), int(budget)), h)


def vlb_structure_length(h) -> float:
    out = ctypes.c_double()
    _check(lib().vlb_structure_length(h, ctypes.byref(out)), h)
    return out.value


def vlb_state_device(h):
    p = ctypes.c_void_p()
    s = ctypes.c_int64()
    _check(lib().vlb_state_device(h, ctypes.byref(p), ctypes.byref(s)), h)
    return p.value, s.value


def vlb_steps_done(h) -> int:
    s = ctypes.c_int64()
    _check(lib().vlb_steps_done(h, ctypes.byref(s)), h)
    return s.value


def vlb_step_noalloc(p: vlb_params, state_ptr: int, stride: int, n0: float, nsteps: int, stream_ptr: int):
    """Step a caller-owned device state in place with no device allocation (see include/vlb.h)."""
    err = ctypes.c_char_p()
    st = lib().vlb_step_noalloc(ctypes.byref(p), ctypes.c_void_p(state_ptr), stride, n0, nsteps,
                                ctypes.c_void_p(stream_ptr), ctypes.byref(err))
    if st != VLB_OK:
        raise VlbError(st, (err.value or b"").decode())


def _ptr(t):
    """Device address of a torch tensor (or None)."""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _scale4(scale):
    return (ctypes.c_float * 4)(*[float(x) for x in scale])


def vlb_get_snapshot(h, snap):
    _check(lib().vlb_get_snapshot(h, _ptr(snap)), h)


def vlb_set_snapshot(h, snap, conserve=None, keep_neq=False):
    c = None if conserve is None else (ctypes.c_double * 2)(*conserve)
    _check(lib().vlb_set_snapshot(h, _ptr(snap), c, 1 if keep_neq else 0), h)


def vlb_conv3x3_fwd(H, W, cin, cout, x, w, bias, mask, relu, y_bf16, y_f32, stream):
    _check(lib().vlb_conv3x3_fwd(H, W, cin, cout, _ptr(x), _ptr(w), _ptr(bias), _ptr(mask), int(relu), _ptr(y_bf16),
                                 _ptr(y_f32), ctypes.c_void_p(stream)))


def vlb_conv3x3_flip(cin, cout, w, w_flipped, stream):
    _check(lib().vlb_conv3x3_flip(cin, cout, _ptr(w), _ptr(w_flipped), ctypes.c_void_p(stream)))


def vlb_conv3x3_wgrad_workspace_bytes(H, W, cin, cout) -> int:
    return lib().vlb_conv3x3_wgrad_workspace_bytes(H, W, cin, cout)


def vlb_conv3x3_bwd_weight(H, W, cin, cout, x, dy, dw, db, workspace, stream):
    _check(lib().vlb_conv3x3_bwd_weight(H, W, cin, cout, _ptr(x), _ptr(dy), _ptr(dw), _ptr(db), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), ctypes.c_void_p(stream)))


def vlb_conv_status(stream, clear=True):
    """Synchronises `stream` and raises VlbError(VLB_ERR_TIMEOUT) if a tensor-core convolution's
    bounded wait gave up since the last clear."""
    _check(lib().vlb_conv_status(ctypes.c_void_p(stream), 1 if clear else 0))


def vlb_test_raise_flag(h, value: int):
    """Test hook: set the device flag of handle h (or, h = None, of the convolutions)."""
    _check(lib().vlb_test_raise_flag(h, int(value)), h)


def vlb_reduce_workspace_bytes() -> int:
    return lib().vlb_reduce_workspace_bytes()


def vlb_surrogate_norm(npix, snap, s_n_fixed, s_u_fixed, g, work, sums, norm8, stream):
    """norm8 (device, 8 floats) := (n_mean, s_phi, s_n, s_u, g0 s_phi, g1 s_n, g2 s_u, g3 s_u)."""
    gg = None if g is None else _scale4(g)
    _check(lib().vlb_surrogate_norm(npix, _ptr(snap), float(s_n_fixed), float(s_u_fixed), gg, _ptr(work), _ptr(sums),
                                    _ptr(norm8), ctypes.c_void_p(stream)))


def vlb_surrogate_features(H, W, r_over_R, snap, d_norm, out, stream):
    """d_norm: device (n_mean, s_phi, s_n, s_u)."""
    _check(lib().vlb_surrogate_features(H, W, r_over_R, _ptr(snap), _ptr(d_norm), _ptr(out), ctypes.c_void_p(stream)))


def vlb_surrogate_targets(npix, before, after, d_scale, target, stream):
    _check(lib().vlb_surrogate_targets(npix, _ptr(before), _ptr(after), _ptr(d_scale), _ptr(target),
                                       ctypes.c_void_p(stream)))


def vlb_surrogate_apply(npix, before, pred16, d_scale, after, stream):
    _check(lib().vlb_surrogate_apply(npix, _ptr(before), _ptr(pred16), _ptr(d_scale), _ptr(after),
                                     ctypes.c_void_p(stream)))


def vlb_snapshot_compare(npix, a, b, work, out4, stream):
    """out4 (device, 4 doubles) := (max |a.phi - b.phi|, max |b.phi|, sum (a.phi - b.phi)^2, sum b.phi^2)."""
    _check(lib().vlb_snapshot_compare(npix, _ptr(a), _ptr(b), _ptr(work), _ptr(out4), ctypes.c_void_p(stream)))


def vlb_channel_sums(npix, C, x, work, out, stream):
    _check(lib().vlb_channel_sums(npix, C, _ptr(x), _ptr(work), _ptr(out), ctypes.c_void_p(stream)))


def vlb_mse_loss(npix, pred16, target4, grad16, work, loss, stream):
    _check(lib().vlb_mse_loss(npix, _ptr(pred16), _ptr(target4), _ptr(grad16), _ptr(work), _ptr(loss),
                              ctypes.c_void_p(stream)))


def vlb_adam_step(n, p, g, m, v, t, lr, b1, b2, eps, p_bf16, stream):
    _check(lib().vlb_adam_step(n, _ptr(p), _ptr(g), _ptr(m), _ptr(v), t, lr, b1, b2, eps, _ptr(p_bf16),
                               ctypes.c_void_p(stream)))


def vlb_to_bf16(n, x, y, stream):
    _check(lib().vlb_to_bf16(n, _ptr(x), _ptr(y), ctypes.c_void_p(stream)))


def _param_array(members):
    arr = (vlb_params * len(members))()
    for i, m in enumerate(members):
        arr[i] = m
    return arr


def vlb_ensemble_workspace_bytes(members) -> int:
    return lib().vlb_ensemble_workspace_bytes(_param_array(members), len(members))


class Ensemble:
    """An ensemble handle, its torch-allocated workspace and one view per member."""

    def __init__(self, members, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("vlb.Ensemble needs a CUDA device")
        arr = _param_array(members)
        self.params = list(members)
        self.nbytes = lib().vlb_ensemble_workspace_bytes(arr, len(members))
        if self.nbytes == 0:
            _check(VLB_ERR_ARG)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.h = ctypes.c_void_p()
        _check(lib().vlb_ensemble_create(arr, len(members), ctypes.c_void_p(self.workspace.data_ptr()), self.nbytes,
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h)))
        self.views = []
        for i in range(len(members)):
            v = ctypes.c_void_p()
            _check(lib().vlb_ensemble_member(self.h, i, ctypes.byref(v)), self.h)
            self.views.append(v)

    def step(self, n: int):
        _check(lib().vlb_ensemble_step(self.h, n), self.h)

    def configure(self, mode=ENS_AUTO, tile_rows=0, ctas_per_sm=0, test_skip_cta=-1, barrier_budget=0):
        c = vlb_ensemble_config(mode=mode, tile_rows=tile_rows, ctas_per_sm=ctas_per_sm, test_skip_cta=test_skip_cta,
                                barrier_budget=barrier_budget)
        _check(lib().vlb_ensemble_configure(self.h, ctypes.byref(c)), self.h)

    def config(self):
        """(mode, tile_rows, ctas_per_sm, ms of the four candidates: batched 16/8, persistent 16/8)."""
        c = vlb_ensemble_config()
        ms = (ctypes.c_float * 4)()
        _check(lib().vlb_ensemble_get_config(self.h, ctypes.byref(c), ms), self.h)
        return {"mode": {0: None, 1: "batched", 2: "persistent"}[c.mode], "tile_rows": c.tile_rows,
                "ctas_per_sm": c.ctas_per_sm, "barrier_budget": c.barrier_budget, "ms": list(ms)}

    def tile_rows(self):
        rows = ctypes.c_int32()
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(lib().vlb_ensemble_tile_rows(self.h, ctypes.byref(rows), ctypes.byref(a), ctypes.byref(b)), self.h)
        return rows.value, a.value, b.value

    def close(self):
        if self.h is not None:
            vlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """A solver handle plus its torch-allocated device workspace on the current device/stream."""

    def __init__(self, params: vlb_params, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("vlb.Solver needs a CUDA device")
        self.p = params
        self.nbytes = vlb_workspace_bytes(params)
        if self.nbytes == 0:
            _check(VLB_ERR_ARG)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self.h = vlb_create(params, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)

    @property
    def shape(self):
        return (self.p.n_theta, self.p.n_phi)

    def set_fields(self, rho, ut, up, phi):
        vlb_set_fields(self.h, rho, ut, up, phi)

    def set_state(self, f16, phi):
        vlb_set_state(self.h, f16, phi)

    def get_state(self):
        return vlb_get_state(self.h, *self.shape)

    def step(self, n: int):
        vlb_step(self.h, n)

    def fields(self):
        return vlb_get_fields(self.h, *self.shape)

    def totals(self):
        return vlb_get_totals(self.h)

    def interface_length(self):
        return vlb_interface_length(self.h)

    def structure_length(self):
        return vlb_structure_length(self.h)

    def set_schedule(self, schedule: int):
        vlb_set_schedule(self.h, schedule)

    def schedule(self) -> int:
        return vlb_get_schedule(self.h)

    def close(self):
        if self.h is not None:
            vlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """A surrogate handle (vlb_surrogate_create) over a torch-allocated workspace: the network's
    weights (a bf16 device tensor of all layers, concatenated) and biases (FP32), its input scales
    and output ratios, for solvers with the grid of `geom`."""

    def __init__(self, geom: vlb_params, weights_bf16, biases, s_n: float, s_u: float, g, window: int, stream=None):
        import torch
        self.geom = geom
        self.nbytes = lib().vlb_surrogate_workspace_bytes(ctypes.byref(geom))
        if self.nbytes == 0:
            _check(VLB_ERR_ARG)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        net = vlb_surrogate_net(weights_bf16=weights_bf16.data_ptr(), biases=biases.data_ptr(), s_n=float(s_n),
                                s_u=float(s_u), g=(ctypes.c_float * 4)(*[float(x) for x in g]), window=int(window),
                                reserved=0)
        self.h = ctypes.c_void_p()
        _check(lib().vlb_surrogate_create(ctypes.byref(geom), ctypes.byref(net),
                                          ctypes.c_void_p(self.workspace.data_ptr()), self.nbytes,
                                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h)))

    def advance(self, solver_h, nwin: int, check_every: int, phi_tol: float, judge_linf=False, graph=True):
        """Returns (kinds, errors, fallbacks): kinds as strings, errors an (nwin, 2) array of
        (relative L2, relative L-infinity) phi errors of judged windows (NaN elsewhere)."""
        kinds = (ctypes.c_int32 * max(nwin, 1))()
        errs = np.empty((max(nwin, 1), 2))
        fb = ctypes.c_int32()
        opts = (SUR_JUDGE_LINF if judge_linf else 0) | (0 if graph else SUR_NO_GRAPH)
        _check(lib().vlb_surrogate_advance(solver_h, self.h, nwin, check_every, float(phi_tol), opts, kinds,
                                           _dptr(errs), ctypes.byref(fb)), self.h)
        return [WINDOW_KINDS[kinds[i]] for i in range(nwin)], errs[:nwin], fb.value

    def stats(self):
        out = (ctypes.c_int64 * 4)()
        _check(lib().vlb_surrogate_stats(self.h, out), self.h)
        return {"windows": out[0], "predicted": out[1], "fallbacks": out[2], "graph": bool(out[3])}

    def close(self):
        if self.h is not None:
            vlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
