"""What the trained surrogate gains over the solver alone, on held-out seeds (256 x 512 tori).

The network is trained here, on the GPU, by the library's own kernels, on trajectories of the
surrogate workload (seeded quenched noise, R / r drawn from [1.5, 4]).  It must then
  * predict phi over a 50-step window at least twice as accurately as persistence (phi unchanged);
  * advance a held-out torus, judged every fourth window by the solver (relative L2 error in phi
    at most 1e-2, else fallback), in less wall time than the solver alone, with the domain length
    L_d = A / L_I within 2 % of the solver's at every judged window."""
import math
import time

import numpy as np
import pytest

from paper_1904_10070_gb300 import surrogate as S
from paper_1904_10070_gb300 import vlb

pytestmark = pytest.mark.gpu

H, W, WINDOW = 256, 512, 50
START, SPACING, PAIRS = 100, 200, 8
WARM, NWIN, CHECK = 400, 32, 4


@pytest.fixture(scope="module")
def trained():
    ds = S.generate(list(range(10000, 10096)), H, W, window=WINDOW, pairs=PAIRS, spacing=SPACING, start=START)
    tr = S.Trainer(S.SurrogateNet(H, W, seed=1), S.target_ratios(ds), ds.s_n, ds.s_u, weights=(1.0, 0.25, 0.25, 0.25))
    tr.fit(ds, epochs=8, lr=1e-3)
    del ds
    return tr


def test_network_beats_persistence(trained):
    import torch
    val = S.generate([20000, 20002], H, W, window=WINDOW, pairs=PAIRS, spacing=SPACING, start=START)
    pred = torch.empty((H * W, 4), dtype=torch.float32, device="cuda")
    n8 = torch.empty(8, dtype=torch.float32, device="cuda")
    ratios = []
    for i in range(len(val)):
        trained.predict(val.before[i], val.radii[i], n8, pred)
        a = val.after[i][:, 0].double().cpu().numpy()
        b = val.before[i][:, 0].double().cpu().numpy()
        p = pred[:, 0].double().cpu().numpy()
        ratios.append(np.linalg.norm(p - a) / np.linalg.norm(b - a))
    print("net / persistence L2 error:", np.round(ratios, 3))
    assert max(ratios) < 0.5


@pytest.mark.parametrize("seed", [20001, 20004])
def test_advance_is_faster_and_tracks_domain_length(trained, seed):
    import torch
    R = S.radius_for(seed)
    p = S.member_params(R, H, W)
    phi = S.initial_phi(seed, H, W)
    z = np.zeros_like(phi)

    def solver():
        s = vlb.Solver(vlb.make_params(**p, precision=vlb.FP32), stream=torch.cuda.Stream())
        s.set_fields(np.ones_like(phi), z, z, phi)
        s.step(WARM)
        return s

    ref, sur = solver(), solver()
    L_ref = []
    torch.cuda.synchronize()
    t_solver = 0.0
    for k in range(NWIN):
        t0 = time.perf_counter()
        ref.step(WINDOW)
        torch.cuda.synchronize()
        t_solver += time.perf_counter() - t0
        if (k + 1) % CHECK == 0:
            L_ref.append(ref.interface_length())
    adv = S.Advancer(trained, sur, window=WINDOW, check_every=CHECK, phi_tol=1e-2)
    L_sur = []
    t_sur = 0.0
    for k in range(NWIN):
        t0 = time.perf_counter()
        adv.window_step()
        torch.cuda.synchronize()
        t_sur += time.perf_counter() - t0
        if (k + 1) % CHECK == 0:
            L_sur.append(sur.interface_length())
    ratio = np.array(L_ref) / np.array(L_sur)  # L_d = A / L_I: the ratio of L_d is L_I,ref / L_I,sur
    print(f"R {R:.2f}: solver {t_solver * 1e3:.1f} ms, surrogate {t_sur * 1e3:.1f} ms, kinds",
          {k: adv.kinds.count(k) for k in set(adv.kinds)}, "L2 errors", np.round(adv.errors, 4),
          "L_d ratios", np.round(ratio, 4))
    assert all(math.isfinite(e) for e in adv.errors)
    assert adv.kinds.count("fallback") <= 1
    assert np.all(np.abs(ratio - 1.0) <= 0.02)
    assert t_sur < t_solver
