"""Radiation stress-energy moments (Sec. 2.5, the definition of R^{alpha beta}).

R^{AB} = sum_n I_n n^A n^B dOmega_n in the tetrad frame (n^0hat = 1); the
coordinate frame applies e^mu_A e^nu_B, the fluid frame the boost Lambda of
Sec. 2.1.  The ten independent components are returned in the order
00, 01, 02, 03, 11, 12, 13, 22, 23, 33.
"""
import torch

PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def tetrad_moments(I, ang):
    n4 = torch.cat([torch.ones(ang.n_ang, 1, dtype=I.dtype), ang.dir], dim=1)
    return torch.einsum("...n,nA,nB,n->...AB", I, n4, n4, ang.dOmega)


def boost(u):
    """Lambda^abar_Bhat for tetrad-frame fluid velocity u^ihat (Sec. 2.1)."""
    u0 = torch.sqrt(1.0 + (u * u).sum(-1))
    sh = u.shape[:-1]
    L = torch.zeros(sh + (4, 4), dtype=u.dtype)
    L[..., 0, 0] = u0
    L[..., 0, 1:] = -u                    # -u_ahat
    L[..., 1:, 0] = -u                    # -u^ahat
    L[..., 1:, 1:] = (torch.einsum("...a,...b->...ab", u, u) / (1.0 + u0)[..., None, None]
                      + torch.eye(3, dtype=u.dtype))
    return L


def moments(I, ang, frame="tetrad", e=None, u=None):
    R = tetrad_moments(I, ang)
    if frame == "coord":
        R = torch.einsum("...mA,...nB,...AB->...mn", e, e, R)
    elif frame == "fluid":
        L = boost(u)
        R = torch.einsum("...aA,...bB,...AB->...ab", L, L, R)
    return torch.stack([R[..., a, b] for (a, b) in PAIRS], dim=-1)
