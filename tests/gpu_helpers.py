"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and the oracle side by side."""
import numpy as np

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import vlb

PKEYS = ["R", "r", "n_theta", "n_phi", "dt", "tau", "M", "A", "kappa", "geometry", "advection", "ch_mode"]


def oracle_params(p: dict) -> O.Params:
    return O.Params(**{k: p[k] for k in PKEYS})


def gpu_params(p: dict, precision=vlb.FP64, diag_every=0) -> vlb.vlb_params:
    return vlb.make_params(**{k: p[k] for k in PKEYS}, precision=precision, diag_every=diag_every)


def rel_err(x, ref):
    """||x - ref||_2 / max(||ref||_2, 1e-3 sqrt(N)) -- a floor keeps near-zero fields (u) meaningful."""
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-3 * np.sqrt(ref.size)))


def max_err(x, ref, floor=1e-3):
    """Element-wise: max_i |x_i - ref_i| / max(max_i |ref_i|, floor).  Unlike rel_err it is not diluted
    by the grid size, so a single wrong node (a seam, a tile edge) shows at full weight."""
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(x - ref)) / max(float(np.max(np.abs(ref))), floor))


def oracle_fields(f, phi, geo):
    n, ut, up = O.moments(f)
    return n, ut, up, phi, O.chemical_potential(phi, geo)


def run_gpu(p: dict, rho, ut, up, phi, steps, precision=vlb.FP64):
    s = vlb.Solver(gpu_params(p, precision))
    s.set_fields(rho, ut, up, phi)
    s.step(steps)
    out = s.fields(), s.get_state(), s.totals()
    s.close()
    return out
