"""Multigroup (frequency-resolved) transport (Sec. 2.2, Eq.
radiation_integral_frequency; the conclusion names the frequency term as
the only addition frequency dependence needs).

Test infrastructure: a plain restatement used only by the tests, the smoke
check and the CPU baseline.

The intensity is kept per group, I_g = the integral of I_nu over the group's
interval [nu_g, nu_{g+1}] of the tetrad-frame frequency (edges nu_0 < ... <
nu_G, nu_0 >= 0, nu_G possibly infinite), array layout I[g, k, j, i, n].
Each group obeys Eq. radiation_integral_frequency integrated over its
interval: the gray spatial and angular fluxes of Eq. radiation_integral plus
the difference of the frequency fluxes n^nu n_0 I_nu at its two edges, with
    n^nu = -nu n^A n^B omega^0hat_{AB}                      (Sec. 2.2)
evaluated with cell-centre geometry (like the angular fluxes).

Readings (the paper states the term, not its discretisation):
  * donor cell in frequency: at an interior edge nu_f the specific intensity
    is the upwind group's mean I_g / (nu_{g+1} - nu_g), the upwind group
    being the lower one where n^nu > 0 (blueshift) and the upper one where
    n^nu < 0; so the flux is F_f = nu_f s n_0 I_up / dnu_up with
    s = n^nu / nu = -omega^0hat_{AB} n^A n^B;
  * the end edges let radiation leave the resolved range and none enter: at
    nu_0 the flux is the lowest group's outflow where s < 0, else 0; at
    nu_G the highest group's outflow where s > 0, else 0; an edge at nu = 0
    or nu = infinity carries nothing (nu I_nu vanishes there), and a group
    reaching infinity has zero mean specific intensity;
  * each group is coupled to the gas on its own with the gray formulas of
    Sec. 2.5 in the fixed-emissivity or no-coupling mode (per-group alpha_a,
    alpha_s and eta).  The frequency shift between tetrad and fluid frames,
    which would couple neighbouring groups for a moving gas, is not
    modelled (the paper leaves frequency-dependent coupling to future
    work); for a gas at rest in the tetrad frame the two frames coincide;
  * the ergosphere guard and the RK2 scheme are the gray ones, applied to
    every group.
"""
import math

import torch

from . import coupling as C
from . import step as S


def omega0_nn(setup):
    """omega^0hat_{AB} n^A n^B per cell and bin (n^0hat = 1)."""
    return torch.einsum("...AB,nA,nB->...n", setup.omega[..., 0, :, :], setup.nhat4, setup.nhat4)


def frequency_fluxes(Ig, setup, edges):
    """F_f = n^nu n_0 I_nu at every group edge f = 0..G: [G + 1, k, j, i, n]."""
    G = Ig.shape[0]
    edges = [float(x) for x in edges]
    s = -omega0_nn(setup)                       # n^nu / nu
    n0 = setup.nlow[..., 0]
    zero = torch.zeros_like(Ig[0])
    mean = []
    for g in range(G):
        dnu = edges[g + 1] - edges[g]
        mean.append(zero if math.isinf(dnu) else Ig[g] / dnu)
    F = []
    for f in range(G + 1):
        nu = edges[f]
        if nu == 0.0 or math.isinf(nu):
            F.append(zero)
            continue
        below = mean[f - 1] if f >= 1 else zero
        above = mean[f] if f < G else zero
        up = torch.where(s > 0.0, below, above)
        F.append(nu * s * n0 * up)
    return torch.stack(F)


def frequency_divergence(Ig, setup, edges):
    """F_{g+1} - F_g per group (the frequency term of Eq.
    radiation_integral_frequency, integrated over the group)."""
    F = frequency_fluxes(Ig, setup, edges)
    return F[1:] - F[:-1]


def operator_L_groups(Ig, setup, opts, edges):
    """L_g = -(spatial + angular divergence of group g) - (F_{g+1} - F_g)."""
    Lg = torch.stack([S.operator_L(Ig[g], setup, opts) for g in range(Ig.shape[0])])
    return Lg - frequency_divergence(Ig, setup, edges)


def rk2_step_groups(I0, T0, gas, dt, setup, opts, edges):
    """One SSP-RK2 step of all groups.  gas: rho, u per cell; alpha_a,
    alpha_s and (emissivity mode) eta per group [G, ...].  opts.mode must be
    'emissivity' (T frozen) or opts.couple False.  Returns (I2, T2, src
    [G, .., 4], ok)."""
    assert (not opts.couple) or opts.mode == "emissivity", "multigroup coupling: fixed emissivity or none"
    G = I0.shape[0]
    f = setup.f
    mask = S.guard_mask(setup, opts)

    def couple(Is, dts):
        out, dR, ok = [], [], torch.ones_like(T0, dtype=torch.bool)
        for g in range(G):
            if opts.couple:
                gg = {"rho": gas["rho"], "u": gas["u"], "alpha_a": gas["alpha_a"][g],
                      "alpha_s": gas["alpha_s"][g], "eta": gas["eta"][g]}
                Ip, _, d, okg = C.couple(Is[g], T0, gg, dts, setup, opts.a_rad, opts.gamma, "emissivity")
                ok = ok & okg
            else:
                Ip, d = Is[g], torch.zeros(T0.shape + (4,), dtype=I0.dtype)
            out.append(torch.where(mask, torch.zeros_like(Ip), Ip))
            dR.append(d)
        return torch.stack(out), torch.stack(dR), ok

    U0 = f * I0
    I1s = S.to_primitive(U0 + dt * operator_L_groups(I0, setup, opts, edges), setup, mask)
    I1, dR1, ok1 = couple(I1s, dt)
    U2s = 0.5 * U0 + 0.5 * (f * I1 + dt * operator_L_groups(I1, setup, opts, edges))
    I2, dR2, ok2 = couple(S.to_primitive(U2s, setup, mask), 0.5 * dt)
    return I2, T0.clone(), -(0.5 * dR1 + dR2), ok1 & ok2


def frequency_dt(setup, edges):
    """Frequency part of the time-step bound (reading R10 carried over):
    min over cells, bins and finite groups of n^0 dnu_g / (nu_{g+1} |s|),
    the time in which a group's donor-cell outflow through its upper edge
    would empty it."""
    s = omega0_nn(setup).abs()
    n0 = setup.nup[..., 0]
    best = math.inf
    for g in range(len(edges) - 1):
        lo, hi = float(edges[g]), float(edges[g + 1])
        if math.isinf(hi):
            continue
        rate = hi * s
        ok = rate > 0
        if bool(ok.any()):
            best = min(best, float(((hi - lo) * n0[ok] / rate[ok]).min()))
    return best
