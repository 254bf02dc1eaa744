"""Pin of the n0crit guard (Sec. 2.4): with n0crit = 0.1 the zeroed bins are
a small part -- under 11 % -- of the phase-space volume between the horizon
and the ergosphere, and far from the hole the guard zeroes nothing."""
import math

import numpy as np
import pytest

from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup


def _ergo_fraction(a, rmax, nr=16, nth=16, level=4):
    rp = 1.0 + math.sqrt(1.0 - a * a)
    xf = [np.linspace(rp, rmax, nr + 1), np.linspace(0.0, math.pi, nth + 1), np.array([0.0, 2.0 * math.pi])]
    st = Setup(Grid("ks_sph", a, xf, (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")), 2),
               GeodesicGrid(level))
    rc = 0.5 * (xf[0][1:] + xf[0][:-1])
    thc = 0.5 * (xf[1][1:] + xf[1][:-1])
    TH, R = np.meshgrid(thc, rc, indexing="ij")                   # [theta, r]
    inside = R < 1.0 + np.sqrt(1.0 - (a * np.cos(TH)) ** 2)       # within the ergosphere
    n0 = st.nlow[..., 0].numpy()[0]                                # [theta, r, bin]
    w = st.dV.numpy()[0][..., None] * st.ang.dOmega.numpy()[None, None, :]
    guarded = np.abs(n0) < 0.1
    m = np.broadcast_to(inside[..., None], n0.shape)
    frac_in = (w * guarded * m).sum() / (w * m).sum()
    return frac_in


@pytest.mark.parametrize("a", [0.5, 0.9, 0.99])
def test_guard_zeroes_under_11_percent_of_the_ergoregion(a):
    frac = _ergo_fraction(a, 2.0)
    assert 0.02 < frac < 0.11


def test_guard_is_inactive_away_from_the_hole():
    """Outgoing light just outside the horizon (also near the poles, where the
    ergosphere meets the horizon) has small |n_0|, so the guard can act
    outside the ergosphere close to r+; from r = 3 on it zeroes nothing."""
    a = 0.9
    xf = [np.linspace(3.0, 12.0, 13), np.linspace(0.0, math.pi, 13), np.array([0.0, 2.0 * math.pi])]
    st = Setup(Grid("ks_sph", a, xf, (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic")), 2),
               GeodesicGrid(4))
    assert (st.nlow[..., 0].abs() >= 0.1).all()
