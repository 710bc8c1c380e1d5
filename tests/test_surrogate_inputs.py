"""Host-side inputs of the surrogate's training set (no GPU): the per-trajectory torus radius and initial
domain scale come from the counter-based generator, are reproducible, fill their ranges, and are drawn
from different elements of a seed's stream; a larger domain scale gives larger domains."""
import math

import numpy as np

from oracle import vlb_oracle as O
from paper_1904_10070_gb300 import surrogate as S


def test_domain_scale_draws_are_reproducible_and_fill_the_range():
    seeds = range(10000, 10400)
    c = np.array([S.corr_for(s, 4.0, 20.0) for s in seeds])
    assert np.array_equal(c, [S.corr_for(s, 4.0, 20.0) for s in seeds])
    assert c.min() >= 4.0 and c.max() < 20.0
    assert c.min() < 5.0 and c.max() > 19.0  # the range is filled
    r = np.array([S.radius_for(s) for s in seeds])
    assert abs(np.corrcoef(c, r)[0, 1]) < 0.2  # not the radius's draw


def test_larger_domain_scale_gives_longer_domains():
    H, W = 64, 128
    p = O.Params(R=2.5, r=1.0, n_theta=H, n_phi=W, dt=1e-3, tau=0.6, M=2.5e-3, A=0.5, kappa=5e-4)
    geo = O.Geometry(p)
    lengths = [O.domain_length(S.initial_phi(7, H, W, corr), geo) for corr in (2.0, 4.0, 8.0)]
    assert lengths[0] < lengths[1] < lengths[2]
    assert all(math.isfinite(x) for x in lengths)
