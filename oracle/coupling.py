"""Locally implicit gas-radiation coupling (Sec. 2.5).

Per cell, with the fluid velocity u^ihat (tetrad frame) frozen:
  n^0bar  = u^0hat - u_ahat n^ahat              (boost, Sec. 2.1)
  Ibar    = Ihat (n^0bar)^4,   dOmega_bar = dOmega_hat / (n^0bar)^2
  Eq. implicit_ii  : Ibar+ = c1 Ibar- + c2 (alpha_P a T+^4 + alpha_s Ebar+)
                     c1 = n^0 / (n^0 + n^0bar alpha_E dt)
                     c2 = n^0bar dt / (4 pi (n^0 + n^0bar alpha_E dt))
  Eq. coupling_rad : Ebar+ - A1 - A2 (alpha_P a T+^4 + alpha_s Ebar+) = 0
  Eq. coupling_tot : c_v (T+ - T-) = -(Ebar+ - Ebar-),  c_v = rho / (Gamma - 1)
  quartic          : B4 T^4 + B1 T + B0 = 0 with B4 = A2 alpha_P a,
                     B1 = c_v (1 - A2 alpha_s), B0 = A1 - B1 T- - (1 - A2 alpha_s) Ebar-
Then the new intensities go back to the tetrad frame, and the change of
R^0_mu = sum I n^0 n_mu dOmega is reported (its negative is the gas source;
end of Sec. 2.5).

Readings: alpha_P = alpha_a (one gray absorption coefficient);
alpha_E = alpha_a + alpha_s; the fluid-frame solid angles are not
renormalised; units k_B/(mu m_p) = 1.

Mode 'emissivity' replaces the thermal emission alpha_P a T^4 / (4 pi) by a
given fluid-frame emissivity eta and keeps T fixed (the c_v -> infinity
limit); Eq. coupling_rad then gives Ebar+ = (A1 + 4 pi A2 eta)/(1 - A2 alpha_s).

Radiation-dominated velocity substitution (end of Sec. 2.5, option rad_dom):
where the fluid-frame radiation energy Ebar- exceeds the gas inertial
density rho + u_gas, the coupling uses, before and after, the velocity
  u^a = (1 - f^a) u_gas^a + f^a u_rad^a
with the radiation velocity v_rad^a = R^{0a} / R^{00} (tetrad frame, from
the intensities entering the coupling), its four-velocity u_rad, the
momentum densities T_gas^{0a} = w u_gas^0 u_gas^a and T_rad^{0a} =
w u_rad^0 u_rad^a (w = rho + u_gas + p), the coupling force
  G^a = -(alpha_P a T^4 + alpha_s Ebar) u^a - alpha_E u_b R^{ab}
at the gas velocity, and the fractions
  f^a = G^a dt / (T_rad^{0a} - T_gas^{0a}), clamped to [0, 1].
Readings: the printed fraction carries an extra factor u^a in its
denominator; it is read as f^a above (the fraction of the momentum gap that
the force closes in dt): with the factor, f^a would be singular for every
gas at rest.  f^a = 0 where the gap T_rad^{0a} - T_gas^{0a} is 0, and no
substitution where no subluminal radiation frame exists (R^{00} <= 0 or
|v_rad| >= 1).  u_gas = c_v T-, p = rho T- (k_B / (mu m_p) = 1).
"""
import math

import torch

FOUR_PI = 4.0 * math.pi


def quartic_root(B4, B1, B0, iters=200):
    """Positive root of B4 T^4 + B1 T + B0 (B4 >= 0, B1 > 0, B0 <= 0).

    Plain bisection on [0, min((-B0/B4)^(1/4), -B0/B1)] (both ends bound the
    root because f is increasing there), then Newton polish.  The last Newton
    step is taken on the attached coefficients, so that automatic
    differentiation sees dT = -(df/dB) / f'(T) (implicit-function theorem).
    Returns (T, ok) where ok is False for an unbracketed problem.
    """
    ok = (B1 > 0.0) & (B0 <= 0.0) & (B4 >= 0.0)
    b4, b1, b0 = B4.detach(), B1.detach(), B0.detach()
    safe_b1 = torch.where(ok, b1, torch.ones_like(b1))
    safe_b0 = torch.where(ok, b0, -torch.ones_like(b0))
    hi = -safe_b0 / safe_b1
    hi4 = torch.where(b4 > 0.0, (-safe_b0 / torch.where(b4 > 0.0, b4, torch.ones_like(b4))) ** 0.25,
                      hi)
    hi = torch.minimum(hi, hi4)
    lo = torch.zeros_like(hi)

    def f(T):
        return b4 * T ** 4 + safe_b1 * T + safe_b0

    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        neg = f(mid) < 0.0
        lo = torch.where(neg, mid, lo)
        hi = torch.where(neg, hi, mid)
    T = 0.5 * (lo + hi)
    for _ in range(3):
        T = T - f(T) / (4.0 * b4 * T ** 3 + safe_b1)
    T = T.detach()
    T = T - (B4 * T ** 4 + B1 * T + B0) / (4.0 * B4 * T ** 3 + B1)
    return torch.where(ok, T, torch.zeros_like(T)), ok


def substituted_velocity(I, T, gas, dt, setup, a_rad=1.0, gamma=5.0 / 3.0):
    """The coupling velocity of the radiation-dominated substitution (Sec. 2.5).

    Returns (u_sub [.., 3], f [.., 3], active [..]): u_sub equals the gas
    velocity wherever the substitution is inactive (active False)."""
    dOmega = setup.ang.dOmega
    nhat = setup.ang.dir
    u = gas["u"]
    u0 = torch.sqrt(1.0 + (u * u).sum(-1))
    nbar0 = u0[..., None] - torch.einsum("...i,ni->...n", u, nhat)
    Ebar = (I * nbar0 ** 2 * dOmega).sum(-1)            # sum Ibar dOmega_bar
    rho = gas["rho"]
    cv = rho / (gamma - 1.0)
    ugas = cv * T
    # tetrad-frame moments R^{AB} of the intensities entering the coupling
    n4 = torch.cat([torch.ones(nhat.shape[0], 1, dtype=I.dtype), nhat], dim=1)
    R = torch.einsum("...n,nA,nB,n->...AB", I, n4, n4, dOmega)
    R00, R0a = R[..., 0, 0], R[..., 0, 1:]
    v = R0a / torch.where(R00 > 0.0, R00, torch.ones_like(R00))[..., None]
    v2 = (v * v).sum(-1)
    active = (Ebar > rho + ugas) & (R00 > 0.0) & (v2 < 1.0)
    gam = 1.0 / torch.sqrt(torch.where(active, 1.0 - v2, torch.ones_like(v2)))
    urad = gam[..., None] * v
    w = rho + ugas + (gamma - 1.0) * ugas                 # rho + u_gas + p
    Tgas = (w * u0)[..., None] * u
    Trad = (w * gam)[..., None] * urad
    aa, a_s = gas["alpha_a"], gas["alpha_s"]
    # u_b R^{ab} with u_0 = -u^0 (orthonormal tetrad)
    uR = -u0[..., None] * R[..., 1:, 0] + torch.einsum("...b,...ab->...a", u, R[..., 1:, 1:])
    G = -(aa * a_rad * T ** 4 + a_s * Ebar)[..., None] * u - (aa + a_s)[..., None] * uR
    gap = Trad - Tgas
    f = torch.where(gap != 0.0, G * dt / torch.where(gap != 0.0, gap, torch.ones_like(gap)), torch.zeros_like(gap))
    f = torch.where(active[..., None], f.clamp(0.0, 1.0), torch.zeros_like(f))
    u_sub = torch.where(active[..., None], (1.0 - f) * u + f * urad, u)
    return u_sub, f, active


def couple(I, T, gas, dt, setup, a_rad=1.0, gamma=5.0 / 3.0, mode="thermal", rad_dom=False):
    """One implicit coupling of every cell over time dt (Sec. 2.5).

    I     [k, j, i, n] tetrad-frame primitive intensities after transport
    T     [k, j, i]    gas temperature before coupling
    gas   dict with rho, u [k, j, i, 3] (u^ihat), alpha_a, alpha_s, eta
    rad_dom: apply the radiation-dominated velocity substitution.
    Returns (I+, T+, dR [k, j, i, 4] = change of R^0_mu, ok).
    """
    dOmega = setup.ang.dOmega
    nhat = setup.ang.dir
    u = substituted_velocity(I, T, gas, dt, setup, a_rad, gamma)[0] if rad_dom else gas["u"]
    u0 = torch.sqrt(1.0 + (u * u).sum(-1))
    nbar0 = u0[..., None] - torch.einsum("...i,ni->...n", u, nhat)
    n0 = setup.nup[..., 0]
    aa, a_s = gas["alpha_a"], gas["alpha_s"]
    aE = (aa + a_s)[..., None]
    Ibar = I * nbar0 ** 4
    dOmbar = dOmega / nbar0 ** 2
    den = n0 + nbar0 * aE * dt
    c1 = n0 / den
    c2 = nbar0 * dt / (FOUR_PI * den)
    A2 = dt / FOUR_PI * (nbar0 / den * dOmbar).sum(-1)
    Em = (Ibar * dOmbar).sum(-1)
    # A1 - Ebar- as one integral of (c1 - 1) Ibar dOmega_bar (c1 - 1 =
    # -n^0bar alpha_E dt / den): the same quantity as the difference of the
    # two integrals, without its cancellation when alpha_E dt << 1
    D = (-(nbar0 * aE * dt) / den * Ibar * dOmbar).sum(-1)
    A1 = D + Em
    if mode == "thermal":
        cv = gas["rho"] / (gamma - 1.0)
        B4 = A2 * aa * a_rad
        B1 = cv * (1.0 - A2 * a_s)
        B0 = D + A2 * a_s * Em - B1 * T            # = A1 - B1 T- - (1 - A2 alpha_s) Ebar-
        Tp, ok = quartic_root(B4, B1, B0)
        Ep = Em - cv * (Tp - T)
        S = aa * a_rad * Tp ** 4 + a_s * Ep
    elif mode == "emissivity":
        eta = gas["eta"]
        Ep = (A1 + FOUR_PI * A2 * eta) / (1.0 - A2 * a_s)
        ok = (1.0 - A2 * a_s) > 0.0
        Tp = T
        S = FOUR_PI * eta + a_s * Ep
    else:
        raise ValueError(mode)
    Ibar_p = c1 * Ibar + c2 * S[..., None]
    Ip = Ibar_p / nbar0 ** 4
    dR = torch.einsum("...n,...n,...nm,n->...m", Ip - I, n0, setup.nlow, dOmega)
    return Ip, Tp, dR, ok
