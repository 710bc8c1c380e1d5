"""vlb_surrogate_advance (the library's surrogate loop, called through the C ABI) against the same
loop driven from the host primitive by primitive (tests/surrogate_reference.py), on a 256 x 512
torus of the surrogate workload: window kinds, judged errors and the final states must agree bit
for bit, with judges that accept everything, reject everything, or split the windows."""
import math

import numpy as np
import pytest

from paper_1904_10070_gb300 import surrogate as S
from paper_1904_10070_gb300 import vlb
from tests.surrogate_reference import ReferenceAdvancer

pytestmark = pytest.mark.gpu

H, W, WINDOW, NWIN = 256, 512, 20, 14


def _trainer():
    net = S.SurrogateNet(H, W, seed=11)
    # s_n, s_u, g of the order a trained network uses on this workload
    return S.Trainer(net, [0.05, 0.02, 0.02, 0.02], 2e-3, 1e-3, weights=(1.0, 0.25, 0.25, 0.25))


def _solver(own_stream):
    import torch
    p = S.member_params(2.7, H, W)
    s = vlb.Solver(vlb.make_params(**p, precision=vlb.FP32), stream=torch.cuda.Stream() if own_stream else None)
    phi = S.initial_phi(20007, H, W)
    z = np.zeros_like(phi)
    s.set_fields(np.ones_like(phi), z, z, phi)
    s.step(100)
    return s


def _run_both(tr, tol, norm, own_stream, check_every=3):
    import torch
    ref_s, lib_s = _solver(own_stream), _solver(own_stream)
    ref = ReferenceAdvancer(tr, ref_s, window=WINDOW, check_every=check_every, phi_tol=tol, norm=norm)
    ref.advance(NWIN)
    torch.cuda.synchronize()
    adv = S.Advancer(tr, lib_s, window=WINDOW, check_every=check_every, phi_tol=tol, norm=norm)
    kinds = adv.advance(NWIN // 2)
    kinds += adv.advance(NWIN - NWIN // 2)  # two calls: the loop's state carries over
    torch.cuda.synchronize()
    assert kinds == ref.kinds
    judged = [e for k, e in zip(ref.kinds, ref.errors) if k in ("checked", "fallback")]
    assert adv.errors == [e[0] for e in judged]
    assert adv.errors_linf == [e[1] for e in judged]
    f_r, p_r = ref_s.get_state()
    f_l, p_l = lib_s.get_state()
    np.testing.assert_array_equal(f_l, f_r)
    np.testing.assert_array_equal(p_l, p_r)
    stats = adv.sur.stats()
    assert stats["windows"] == NWIN and stats["fallbacks"] == kinds.count("fallback")
    return kinds, [e[0] for e in judged], adv


@pytest.mark.parametrize("own_stream", [True, False])
def test_library_loop_matches_host_loop_accepting_and_rejecting(own_stream):
    tr = _trainer()
    kinds, errs, adv = _run_both(tr, math.inf, "l2", own_stream)
    assert kinds.count("checked") == NWIN // 3 and "fallback" not in kinds
    assert adv.graph is (True if own_stream else None)  # predicted windows replay a graph on a stream
    kinds, _, _ = _run_both(tr, 0.0, "linf", own_stream)
    assert kinds[:5] == ["surrogate", "surrogate", "fallback", "solver", "solver"]


def test_library_loop_matches_host_loop_with_a_split_judge():
    tr = _trainer()
    _, errs, _ = _run_both(tr, math.inf, "l2", True)
    tol = float(np.median(errs))  # some judged windows pass, some fail
    kinds, _, _ = _run_both(tr, tol, "l2", True, check_every=2)
    assert "checked" in kinds and "fallback" in kinds, kinds


def test_advance_rejects_bad_arguments():
    import torch
    tr = _trainer()
    s = _solver(True)
    adv = S.Advancer(tr, s, window=WINDOW, check_every=2)
    for bad in (dict(nwin=-1), dict(phi_tol=math.nan), dict(check_every=-2)):
        args = dict(nwin=1, check_every=2, phi_tol=1e-2)
        args.update(bad)
        with pytest.raises(vlb.VlbError) as exc:
            adv.sur.advance(s.h, args["nwin"], args["check_every"], args["phi_tol"])
        assert exc.value.status == vlb.VLB_ERR_ARG
    other = vlb.Solver(vlb.make_params(**S.member_params(2.7, 128, 256), precision=vlb.FP32))
    with pytest.raises(vlb.VlbError) as exc:
        adv.sur.advance(other.h, 1, 2, 1e-2)
    assert exc.value.status == vlb.VLB_ERR_ARG and "grid" in str(exc.value)
    with pytest.raises(vlb.VlbError):  # a surrogate handle is not a solver
        vlb.vlb_step(adv.sur.h, 1)
    torch.cuda.synchronize()
