"""The batched ensemble (one launch per stage over all members, graph-replayed) against stepping each
member alone, against the FP64 oracle, and against sequential per-member launches in time."""
import time

import numpy as np
import pytest

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import inputs, vlb
from tests.gpu_helpers import max_err, oracle_params, rel_err

pytestmark = pytest.mark.gpu

KEYS = ["R", "r", "n_theta", "n_phi", "dt", "tau", "M", "A", "kappa", "geometry", "advection", "ch_mode"]


def _members(specs, seed0=300):
    out = []
    for i, (nt, ns, R) in enumerate(specs):
        p = dict(geometry=0, R=R, r=1.0, n_theta=nt, n_phi=ns, dt=1.0, tau=0.2, M=0.05, A=0.3, kappa=0.01,
                 advection=0, ch_mode=0)
        p["dt"] = 0.4 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
        rng = np.random.default_rng(seed0 + i)
        f = dict(rho=1.0 + 0.05 * rng.uniform(-1, 1, (nt, ns)), ut=0.03 * rng.uniform(-1, 1, (nt, ns)),
                 up=0.03 * rng.uniform(-1, 1, (nt, ns)), phi=np.tanh(2 * rng.uniform(-1, 1, (nt, ns))))
        out.append((p, f))
    return out


# grids: packed pairs (n_phi % 4 == 0, >= 40), scalar fallback (n_phi = 70), ragged tiles, both tile heights
SPECS = [(40, 64, 2.0), (64, 128, 3.1), (20, 44, 1.6), (33, 70, 2.5), (72, 96, 4.2)]


@pytest.mark.parametrize("mode,rows", [(vlb.ENS_AUTO, 0), (vlb.ENS_BATCHED, 8), (vlb.ENS_PERSISTENT, 16),
                                       (vlb.ENS_PERSISTENT, 8)])
def test_ensemble_matches_members_stepped_alone_and_the_oracle(mode, rows):
    mem = _members(SPECS)
    ens = vlb.Ensemble([vlb.make_params(**p, precision=vlb.FP32) for p, _ in mem])
    if mode != vlb.ENS_AUTO:
        ens.configure(mode=mode, tile_rows=rows)
    solo = []
    for v, (p, f) in zip(ens.views, mem):
        vlb.vlb_set_fields(v, f["rho"], f["ut"], f["up"], f["phi"])
        s = vlb.Solver(vlb.make_params(**p, precision=vlb.FP32))
        s.set_fields(f["rho"], f["ut"], f["up"], f["phi"])
        solo.append(s)
    steps = 12
    ens.step(5)
    ens.step(steps - 5)  # second call replays the recorded graphs
    cfg = ens.config()
    assert cfg["tile_rows"] in (8, 16)
    if mode == vlb.ENS_AUTO:
        assert all(ms > 0 for ms in cfg["ms"]), cfg  # all four candidates were timed
    else:
        assert cfg["mode"] == {vlb.ENS_BATCHED: "batched", vlb.ENS_PERSISTENT: "persistent"}[mode]
        assert cfg["tile_rows"] == rows
    for i, (v, (p, f)) in enumerate(zip(ens.views, mem)):
        solo[i].step(steps)
        g = vlb.vlb_get_fields(v, p["n_theta"], p["n_phi"])
        r = solo[i].fields()
        for a, b in zip(g[:4], r[:4]):
            assert rel_err(a, b) <= 1e-6 and max_err(a, b) <= 1e-6, (i, rel_err(a, b), max_err(a, b))
        geo = O.Geometry(oracle_params(p))
        fo, po = O.init_state(f["rho"], f["ut"], f["up"], f["phi"])
        fo, po = O.run(fo, po, geo, steps)
        n, ut, up = O.moments(fo)
        for a, b in zip(g[:4], (n, ut, up, po)):
            assert rel_err(a, b) <= 2e-5 and max_err(a, b) <= 2e-5, (i, rel_err(a, b), max_err(a, b))
        assert vlb.vlb_steps_done(v) == steps
        solo[i].close()
    ens.close()


def test_forty_eight_tori_conserve_and_beat_sequential_launches():
    import torch
    work = inputs.ensemble_workload(48)
    params = []
    for w in work:
        p = dict(w["params"], dt=1.0)
        p["dt"] = 0.5 * vlb.vlb_max_stable_dt(vlb.make_params(**p))
        params.append(vlb.make_params(**p, precision=vlb.FP32))
    ens = vlb.Ensemble(params)
    for v, w in zip(ens.views, work):
        vlb.vlb_set_fields(v, w["rho"], w["ut"], w["up"], w["phi"])
    t0 = [vlb.vlb_get_totals(v) for v in ens.views]
    ens.step(3)  # tunes and records the graphs
    torch.cuda.synchronize()
    n = 20
    a = time.perf_counter()
    ens.step(n)
    torch.cuda.synchronize()
    t_ens = time.perf_counter() - a
    a = time.perf_counter()
    for v in ens.views:  # the same members, one after another with per-member launches
        vlb.vlb_step(v, n)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - a
    nodes = sum(p.n_theta * p.n_phi for p in params)
    print(f"48 tori, {nodes} nodes: ensemble {1e3 * t_ens / n:.3f} ms/step, sequential {1e3 * t_seq / n:.3f} "
          f"ms/step, tile rows {ens.tile_rows()[0]}")
    for v, tt in zip(ens.views, t0):
        t1 = vlb.vlb_get_totals(v)
        assert np.all(np.isfinite(t1))
        assert abs(t1[0] - tt[0]) <= 1e-6 * abs(tt[0])
        assert abs(t1[1] - tt[1]) <= 1e-6 * np.abs(tt[0])
    assert t_ens < t_seq
    ens.close()


def test_persistent_and_batched_launches_agree_bit_for_bit():
    """The persistent launch runs the same tile arithmetic as the batched launches, only scheduled
    differently, so the states agree bit for bit (both tile heights, 40 steps over several graph
    replays and an eager remainder)."""
    mem = _members(SPECS, seed0=500)
    states = []
    for mode, rows in ((vlb.ENS_BATCHED, 16), (vlb.ENS_PERSISTENT, 16), (vlb.ENS_PERSISTENT, 8)):
        ens = vlb.Ensemble([vlb.make_params(**p, precision=vlb.FP32) for p, _ in mem])
        ens.configure(mode=mode, tile_rows=rows)
        for v, (p, f) in zip(ens.views, mem):
            vlb.vlb_set_fields(v, f["rho"], f["ut"], f["up"], f["phi"])
        ens.step(7)
        ens.step(33)
        states.append([vlb.vlb_get_state(v, p["n_theta"], p["n_phi"]) for v, (p, _) in zip(ens.views, mem)])
        ens.close()
    for other in states[1:]:
        for (fa, pa), (fb, pb) in zip(states[0], other):
            np.testing.assert_array_equal(fa, fb)
            np.testing.assert_array_equal(pa, pb)


def test_persistent_barrier_times_out_instead_of_hanging():
    """A CTA that never arrives at the grid barrier (the test hook) makes the others give up after the
    barrier budget (here about a millisecond of SM cycles): the launch ends, the ensemble's flag is
    raised, the members report VLB_ERR_TIMEOUT, and a reset state steps normally again."""
    mem = _members(SPECS[:3], seed0=600)
    ens = vlb.Ensemble([vlb.make_params(**p, precision=vlb.FP32) for p, _ in mem])
    ens.configure(mode=vlb.ENS_PERSISTENT, tile_rows=16, test_skip_cta=0, barrier_budget=2_000_000)
    for v, (p, f) in zip(ens.views, mem):
        vlb.vlb_set_fields(v, f["rho"], f["ut"], f["up"], f["phi"])
    ens.step(3)
    for v in ens.views:
        with pytest.raises(vlb.VlbError) as exc:
            vlb.vlb_get_totals(v)
        assert exc.value.status == vlb.VLB_ERR_TIMEOUT
    ens.configure(mode=vlb.ENS_PERSISTENT, tile_rows=16)
    for v, (p, f) in zip(ens.views, mem):
        vlb.vlb_set_fields(v, f["rho"], f["ut"], f["up"], f["phi"])
    ens.step(3)
    for v in ens.views:
        assert np.all(np.isfinite(vlb.vlb_get_totals(v)))
    ens.close()


def test_autotune_choice_is_cached(tmp_path, monkeypatch):
    """The first ensemble times the four candidates and writes its choice to VLB_AUTOTUNE_CACHE; a second
    ensemble with the same grids takes the cached choice (the same timings, to the bit) without timing."""
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("VLB_AUTOTUNE_CACHE", str(cache))
    specs = [(24, 64, 2.2), (48, 128, 3.3), (36, 96, 1.9)]
    mem = _members(specs, seed0=700)
    cfgs = []
    for _ in range(2):
        ens = vlb.Ensemble([vlb.make_params(**p, precision=vlb.FP32) for p, _ in mem])
        for v, (p, f) in zip(ens.views, mem):
            vlb.vlb_set_fields(v, f["rho"], f["ut"], f["up"], f["phi"])
        ens.step(2)
        cfgs.append(ens.config())
        ens.close()
    assert cfgs[0] == cfgs[1]
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and '"kind": "ensemble"' in lines[0]
    mode = {"batched": 1, "persistent": 2}[cfgs[0]["mode"]]
    assert f'"mode": {mode}, "tile_rows": {cfgs[0]["tile_rows"]}' in lines[0]
