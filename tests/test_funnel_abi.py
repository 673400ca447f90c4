"""The funnel-inference update through the C ABI (host arithmetic: no GPU needed) against
the oracle's secant rule."""
import pytest

from oracle import lam as olam


def test_funnel_next_matches_oracle():
    from paper_2509_14185_gb300 import gn
    cases = [([0.7], [0.3], 0.01), ([0.5, 0.52], [0.39, 0.31], 0.02),
             ([1.0, 1.01, 0.97, 0.985], [-0.2, 0.05, -0.01, 0.003], 0.01)]
    for lams, rh, d in cases:
        assert gn.gn_funnel_next(lams, rh, d) == olam.funnel_next(lams, rh, d)
    with pytest.raises(gn.GNError):
        gn.gn_funnel_next([0.1, 0.2], [1.0, 1.0], 0.1)
    with pytest.raises(gn.GNError):
        gn.gn_funnel_next([], [], 0.1)
