"""Time-step bound.

The paper gives no formula; the reading used here is
  dt = C * min(dt_space, dt_angle)
  dt_space = min over cells, flux dimensions d and bins n of dx^d / |n^d / n^0|
             (cell-centre tetrad)
  dt_angle = min over cells and bins of dOmega_n n^0 / sum_{edges of n} l_e |V . nu_e|
where V . nu_e is the angular speed of Eq. flux_angle on the geodesic grid.
"""
import torch

from . import transport as TR


def cfl_dt(setup, C=0.3):
    grid, ang = setup.grid, setup.ang
    n0 = setup.nup[..., 0]
    best = torch.tensor(float("inf"), dtype=torch.float64)
    for d in range(grid.ndim):
        dx = grid.xf[d][1:] - grid.xf[d][:-1]
        shape = [1, 1, 1]
        shape[2 - d] = -1
        dx = dx.reshape(shape)[..., None]
        speed = (setup.nup[..., d + 1] / n0).abs()
        ratio = torch.where(speed > 0, dx / torch.where(speed > 0, speed, torch.ones_like(speed)),
                            torch.full_like(speed, float("inf")))
        best = torch.minimum(best, ratio.min())
    _, s = TR.angular_speeds(setup)
    rate = torch.zeros(grid.shape + (ang.n_ang,), dtype=torch.float64)
    p, q = ang.edges[:, 0], ang.edges[:, 1]
    w = ang.edge_len * s.abs()
    rate = rate.index_add(-1, p, w).index_add(-1, q, w)
    ok = rate > 0
    ratio = torch.where(ok, ang.dOmega * n0 / torch.where(ok, rate, torch.ones_like(rate)),
                        torch.full_like(rate, float("inf")))
    best = torch.minimum(best, ratio.min())
    return C * float(best)
