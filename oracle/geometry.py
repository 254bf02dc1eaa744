"""Metric, tetrad, Ricci rotation coefficients and finite volumes (Secs. 2.1-2.2).

Coordinates are (t, x1, x2, x3); every metric here is stationary (Eq.
stationary_metric) and independent of x3.  Three spacetimes:

  'mink_cart'  Minkowski, Cartesian (x, y, z)
  'mink_sph'   Minkowski, spherical (r, theta, phi)        (tests only)
  'ks_sph'     Kerr in spherical Kerr-Schild (r, theta, phi), M = 1, spin a
  'schw_sph'   Schwarzschild in Schwarzschild coordinates, M = 1 (tests only:
               its normal observers are the static ones)

Tetrad (Eq. tetrad and the normal-observer condition below it):
  e_0hat^alpha = -alpha g^{0 alpha}; the spatial legs have zero time
  component and come from Gram-Schmidt (with the spatial metric) on the
  coordinate basis vectors in a fixed order:
    Cartesian: z -> 3hat, x -> 1hat, y -> 2hat   (identity tetrad)
    spherical: theta -> 3hat, phi -> 1hat, r -> 2hat  (the paper's
               "spherical tetrad": n^3 along theta, n^1 along phi)

Ricci rotation coefficients (Eq. ricci):
  omega^c_{ab} = e^c_eps e^del_b nabla_del e^eps_a
with the covariant derivative written out with Christoffel symbols of the
second kind; the coordinate derivatives of e and g are exact
(forward-mode automatic differentiation of the analytic expressions).

Array conventions: e[..., mu, A] = e^mu_A (coordinate index first, tetrad
index second); omega[..., C, A, B] = omega^C_{AB}.
"""
import math

import torch
from torch.func import jacfwd, vmap

from . import DTYPE

KINDS = ("mink_cart", "mink_sph", "ks_sph", "schw_sph")


def metric(kind, a, x):
    """g_{mu nu} at spatial point x = (x1, x2, x3) (a 3-tensor)."""
    z = x[0] * 0.0
    one = z + 1.0
    if kind == "mink_cart":
        rows = [[-one, z, z, z], [z, one, z, z], [z, z, one, z], [z, z, z, one]]
    elif kind == "mink_sph":
        r, th = x[0], x[1]
        s = torch.sin(th)
        rows = [[-one, z, z, z], [z, one, z, z], [z, z, r * r, z],
                [z, z, z, r * r * s * s]]
    elif kind == "schw_sph":
        r, th = x[0], x[1]
        s = torch.sin(th)
        f = 1.0 - 2.0 / r
        rows = [[-f, z, z, z], [z, 1.0 / f, z, z], [z, z, r * r, z], [z, z, z, r * r * s * s]]
    elif kind == "ks_sph":
        r, th = x[0], x[1]
        s, c = torch.sin(th), torch.cos(th)
        sig = r * r + a * a * c * c
        q = 2.0 * r / sig
        gtt = -(1.0 - q)
        gtr = q
        gtp = -a * q * s * s
        grr = 1.0 + q
        grp = -a * (1.0 + q) * s * s
        gthth = sig
        gpp = s * s * (r * r + a * a + a * a * q * s * s)
        rows = [[gtt, gtr, z, gtp], [gtr, grr, z, grp], [z, z, gthth, z],
                [gtp, grp, z, gpp]]
    else:
        raise ValueError(kind)
    return torch.stack([torch.stack(rw) for rw in rows])


def leg_order(kind):
    """Coordinate index (1..3) Gram-Schmidt'ed into tetrad legs 3hat, 1hat, 2hat."""
    if kind == "mink_cart":
        return [(3, 3), (1, 1), (2, 2)]      # (coordinate, tetrad leg)
    return [(2, 3), (3, 1), (1, 2)]          # theta->3hat, phi->1hat, r->2hat


def tetrad(kind, a, x):
    """e^mu_A at x (Eq. tetrad; e_0hat is the normal observer)."""
    g = metric(kind, a, x)
    ginv = torch.linalg.inv(g)
    lapse = (-ginv[0, 0]) ** -0.5
    legs = [None] * 4
    legs[0] = -lapse * ginv[0, :]
    basis = []
    for (coord, leg) in leg_order(kind):
        v = torch.zeros(4, dtype=x.dtype) + x[0] * 0.0
        v = torch.where(torch.arange(4) == coord, v + 1.0, v)
        for b in basis:
            v = v - (b @ g @ v) * b
        v = v / torch.sqrt(v @ g @ v)
        basis.append(v)
        legs[leg] = v
    return torch.stack(legs, dim=1)          # e[mu, A]


ETA = torch.diag(torch.tensor([-1.0, 1.0, 1.0, 1.0], dtype=DTYPE))


def _pad_time(d):
    """Jacobian over (x1, x2, x3) -> derivative over (t, x1, x2, x3), d_t = 0."""
    zero = torch.zeros(d.shape[:-1] + (1,), dtype=d.dtype)
    return torch.cat([zero, d], dim=-1)


def christoffel(kind, a, x):
    """Gamma^e_{d s} = 1/2 g^{e k} (d_d g_{k s} + d_s g_{k d} - d_k g_{d s})."""
    g = metric(kind, a, x)
    dg = _pad_time(jacfwd(lambda y: metric(kind, a, y))(x))   # dg[k, s, d] = d_d g_{ks}
    ginv = torch.linalg.inv(g)
    low = 0.5 * (torch.einsum("ksd->kds", dg) + torch.einsum("kds->kds", dg)
                 - torch.einsum("dsk->kds", dg))                 # low[k, d, s]
    return torch.einsum("ek,kds->eds", ginv, low)


def ricci_rotation(kind, a, x):
    """omega^C_{AB} = e^C_eps e^del_B (d_del e^eps_A + Gamma^eps_{del sig} e^sig_A)."""
    e = tetrad(kind, a, x)
    de = _pad_time(jacfwd(lambda y: tetrad(kind, a, y))(x))    # de[eps, A, del]
    gam = christoffel(kind, a, x)
    einv = torch.linalg.inv(e)                                  # einv[C, eps] = e^C_eps
    cov = de + torch.einsum("eds,sA->eAd", gam, e)              # nabla_del e^eps_A
    return torch.einsum("Ce,dB,eAd->CAB", einv, e, cov)


def batched(fn, kind, a, X):
    """Evaluate fn(kind, a, x) for every row of X [P, 3]."""
    return vmap(lambda x: fn(kind, a, x))(X)


# ---------------------------------------------------------------- volumes
def cell_volume(kind, a, lo, hi):
    """Delta V = integral of sqrt(-g) over the cell (Sec. 2.2), exact.

    lo, hi: [..., 3] face coordinates.  For the spherical metrics
    sqrt(-g) = (r^2 + a^2 cos^2 theta) sin theta (a = 0 for flat space).
    """
    if kind == "mink_cart":
        return (hi - lo).prod(-1)
    r1, t1, p1 = lo.unbind(-1)
    r2, t2, p2 = hi.unbind(-1)
    aa = a * a if kind == "ks_sph" else 0.0
    c1, c2 = torch.cos(t1), torch.cos(t2)
    return (p2 - p1) * ((r2 ** 3 - r1 ** 3) / 3.0 * (c1 - c2)
                        + aa * (r2 - r1) * (c1 ** 3 - c2 ** 3) / 3.0)


def face_area(kind, a, axis, lo, hi):
    """Delta A_axis = integral of sqrt(-g) over the face at x_axis = lo[axis].

    lo/hi give the extent in the two other coordinates (the value of hi[axis]
    is ignored).
    """
    if kind == "mink_cart":
        w = hi - lo
        others = [d for d in range(3) if d != axis]
        return w[..., others[0]] * w[..., others[1]]
    r1, t1, p1 = lo.unbind(-1)
    r2, t2, p2 = hi.unbind(-1)
    aa = a * a if kind == "ks_sph" else 0.0
    c1, c2 = torch.cos(t1), torch.cos(t2)
    if axis == 0:      # constant r
        return (p2 - p1) * (r1 * r1 * (c1 - c2) + aa * (c1 ** 3 - c2 ** 3) / 3.0)
    if axis == 1:      # constant theta
        return (p2 - p1) * torch.sin(t1) * ((r2 ** 3 - r1 ** 3) / 3.0
                                            + aa * c1 * c1 * (r2 - r1))
    return (r2 ** 3 - r1 ** 3) / 3.0 * (c1 - c2) + aa * (r2 - r1) * (c1 ** 3 - c2 ** 3) / 3.0


def horizon_radius(a):
    return 1.0 + math.sqrt(1.0 - a * a)
