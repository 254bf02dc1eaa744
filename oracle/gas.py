"""Gas energy-momentum update from the radiation source (end of Sec. 2.5: the
coupling's change of R^0_mu is subtracted from the gas, which then recovers
its primitive state).

Test infrastructure: a plain restatement used only by the tests, the smoke
check and the CPU baseline.

The gas is an ideal fluid of rest-mass density rho, temperature T (units
k_B / (mu m_p) = 1: p = rho T, internal energy rho T / (Gamma - 1)) and
tetrad-frame velocity u^ihat.  Its conserved variables are D = rho u^0 and
T^0_mu = w u^0 u_mu + p delta^0_mu (w = rho + Gamma p / (Gamma - 1)), which
the step's source src_mu = -dR^0_mu changes by src_mu while D is kept.  In
the normal observer's tetrad (e^0_ihat = 0, e^0_0hat = n^0) these read
    D-hat = rho gamma = D / n^0
    E     = -T^0hat_0hat = w gamma^2 - p = -(T^0_mu e^mu_0hat) / n^0
    S_i   =  T^0hat_ihat = w gamma u^ihat =  (T^0_mu e^mu_ihat) / n^0
and the primitive state follows from the one unknown p:
    v = S / (E + p),  gamma = (1 - v^2)^(-1/2),  rho = D-hat / gamma,
    w = (E + p) (1 - v^2),  p = (Gamma - 1) / Gamma (w - rho)
(the last is the equation solved, by bisection on [0, Gamma E], which
brackets its one root for every state with E > (S^2 + D-hat^2)^(1/2));
then u^ihat = gamma v, T = p / rho.
"""
import torch


def conserved(rho, u, T, setup, gamma):
    """(D, Q_mu = T^0_mu) of the gas state per cell."""
    e = setup.e                                              # e^mu_A
    g = setup.g
    u0h = torch.sqrt(1.0 + (u * u).sum(-1))
    uA = torch.cat([u0h[..., None], u], dim=-1)              # u^A
    umu = torch.einsum("...mA,...A->...m", e, uA)            # u^mu
    ulow = torch.einsum("...mn,...n->...m", g, umu)          # u_mu
    p = rho * T
    w = rho + gamma / (gamma - 1.0) * p
    Q = (w * umu[..., 0])[..., None] * ulow
    Q[..., 0] = Q[..., 0] + p
    return rho * umu[..., 0], Q


def gas_update(rho, u, T, src, setup, gamma, iters=200):
    """New (rho, u, T) after adding src [.., 4] to T^0_mu at fixed D.
    Returns (rho, u, T, ok)."""
    D, Q = conserved(rho, u, T, setup, gamma)
    Q = Q + src
    e = setup.e
    n0 = e[..., 0, 0]
    Qt = torch.einsum("...m,...mA->...A", Q, e) / n0[..., None]   # T^0hat_Ahat
    E, S = -Qt[..., 0], Qt[..., 1:]
    Dh = D / n0
    S2 = (S * S).sum(-1)
    gfac = (gamma - 1.0) / gamma

    def f(p):
        v2 = S2 / (E + p) ** 2
        w = (E + p) * (1.0 - v2)
        return p - gfac * (w - Dh * torch.sqrt(1.0 - v2))

    # a physical state has E > |S| (so v < 1 for every p >= 0) and
    # f(0) = -(Gamma-1)/Gamma (1 - v^2)^(1/2) ((E^2 - S^2)^(1/2) - D-hat) < 0;
    # f(p) >= p / Gamma - (Gamma - 1) E / Gamma, so f(Gamma E) > 0
    lo = torch.zeros_like(E)
    hi = gamma * torch.clamp(E, min=1e-300)
    ok = (E > torch.sqrt(S2)) & (Dh > 0) & (f(lo) < 0) & (f(hi) > 0)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        neg = f(mid) < 0.0
        lo = torch.where(neg, mid, lo)
        hi = torch.where(neg, hi, mid)
    p = 0.5 * (lo + hi)
    v = S / (E + p)[..., None]
    gam = 1.0 / torch.sqrt(1.0 - (v * v).sum(-1))
    rho_n = Dh / gam
    return rho_n, gam[..., None] * v, p / rho_n, ok
