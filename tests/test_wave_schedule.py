"""Host-side check of the wavefront schedule's ticket order (no GPU): every band item (step, stage,
band) appears exactly once, and after the three band items of the previous sweep it reads (the band
and its two neighbours, across the periodic seam).  This is what makes the persistent launch free of
deadlock: the CTA holding the oldest unfinished ticket never waits on a later one."""
import pytest

from paper_1904_10070_gb300 import vlb


@pytest.mark.parametrize("n_bands", [11, 12, 16, 17, 64, 256])
@pytest.mark.parametrize("nsteps", [1, 2, 3, 7])
def test_ticket_order_is_topological(n_bands, nsteps):
    assert vlb.vlb_test_wave_schedule(n_bands, 4, nsteps)


@pytest.mark.parametrize("lag", [3, 5, 8])
def test_other_lags(lag):
    assert vlb.vlb_test_wave_schedule(2 * lag + 3, lag, 4)
    assert vlb.vlb_test_wave_schedule(64, lag, 5)


@pytest.mark.parametrize("n_bands,lag", [(10, 4), (8, 3), (64, 2), (4, 4)])
def test_rejected_when_a_dependency_would_come_later(n_bands, lag):
    assert not vlb.vlb_test_wave_schedule(n_bands, lag, 3)
