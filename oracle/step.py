"""Two-stage Runge-Kutta step of the radiation field with coupling (Sec. 2).

Readings (the paper names the stage tasks but not the integrator):
  * "RK2" is the SSP (Heun) scheme: stage s has weights (a_s, b_s, beta_s) =
    (0, 1, 1) then (1/2, 1/2, 1/2):
        U^s* = a_s U^0 + b_s (U^{s-1} + beta_s dt L(I^{s-1}))
    with L = -(spatial divergence + angular divergence) of Eq.
    radiation_integral and U = n^0 n_0 I.
  * the coupling of Sec. 2.5 follows every stage with dt_s = beta_s dt; the
    gas temperature entering stage 2 is the same average as U,
    1/2 T^0 + 1/2 T^1;
  * the n0crit guard of Sec. 2.4 zeroes I where |n_0| < n0crit after the
    coupling of every stage, and bins under the guard convert U -> I as 0;
  * the gas source over the step is -(1/2 dR^1 + dR^2), the RK-weighted
    change of R^0_mu produced by the two couplings;
  * the optical-depth flux weighting (Sec. 2.4) uses the step's dt in both
    stages (the stage operator L is the same function of I in both).
"""
from dataclasses import dataclass

import torch

from . import coupling as C
from . import transport as TR


@dataclass
class Opts:
    recon: str = "plm"          # 'dc' | 'plm'
    n0crit: float = 0.1
    zero_guard: bool = True
    mode: str = "thermal"       # 'thermal' | 'emissivity'
    a_rad: float = 1.0
    gamma: float = 5.0 / 3.0
    couple: bool = True
    tau_const: float = 0.0      # C of the optical-depth flux weighting (0: free streaming)
    rad_dom: bool = False       # radiation-dominated velocity substitution (Sec. 2.5)
    recon_ang: str = "dc"       # 'dc' | 'plm' (PLM along the lines of a latitude-longitude grid)
                                # | 'mapr' (minimum-angle planes on a geodesic grid)


def operator_L(I, setup, opts, tau=None, halos=None):
    """L(I) = -(div_space + div_angle), Eq. radiation_integral without sources;
    halos: ghost layers of faces shared with other blocks (fill_ghosts)."""
    Ie = TR.fill_ghosts(I, setup.grid, setup.ang.perm_pi2, halos)
    divS = TR.spatial_divergence(Ie, setup, opts.recon, tau)
    divA = TR.angular_divergence(I, setup, opts.recon_ang)
    return -(divS + divA)


def guard_mask(setup, opts):
    """True where the bin is zeroed (|n_0| < n0crit, Sec. 2.4)."""
    if not opts.zero_guard:
        return torch.zeros_like(setup.f, dtype=torch.bool)
    return setup.nlow[..., 0].abs() < opts.n0crit


def to_primitive(U, setup, mask):
    return torch.where(mask, torch.zeros_like(U), U / torch.where(mask, torch.ones_like(U), setup.f))


def rk2_step(I0, T0, gas, dt, setup, opts, exchange=None):
    """One full step.  Returns (I2, T2, src [.., 4], ok).

    exchange: for a block of a decomposed domain (faces with the 'halo'
    boundary), a callable taking the stage's input intensities and returning
    the ghost layers of those faces from the neighbouring blocks (the ghost
    exchange that precedes each stage's fluxes in the task list of Sec. 2)."""
    f = setup.f
    mask = guard_mask(setup, opts)
    # optical-depth flux weights: frozen gas, the step's dt in both stages
    assert exchange is None or opts.tau_const == 0.0, "the flux weighting needs the neighbours' gas"
    tau = TR.tau_weights(setup, gas, dt, opts.tau_const) if opts.tau_const > 0.0 else None
    U0 = f * I0
    # stage 1
    U1s = U0 + dt * operator_L(I0, setup, opts, tau, exchange(I0) if exchange else None)
    I1s = to_primitive(U1s, setup, mask)
    if opts.couple:
        I1, T1, dR1, ok1 = C.couple(I1s, T0, gas, dt, setup, opts.a_rad, opts.gamma, opts.mode, opts.rad_dom)
    else:
        I1, T1, dR1, ok1 = I1s, T0, torch.zeros(T0.shape + (4,), dtype=I0.dtype), torch.ones_like(T0, dtype=torch.bool)
    I1 = torch.where(mask, torch.zeros_like(I1), I1)
    # stage 2
    U2s = 0.5 * U0 + 0.5 * (f * I1 + dt * operator_L(I1, setup, opts, tau, exchange(I1) if exchange else None))
    I2s = to_primitive(U2s, setup, mask)
    Tm = 0.5 * (T0 + T1)
    if opts.couple:
        I2, T2, dR2, ok2 = C.couple(I2s, Tm, gas, 0.5 * dt, setup, opts.a_rad, opts.gamma, opts.mode,
                                     opts.rad_dom)
    else:
        I2, T2, dR2, ok2 = I2s, Tm, torch.zeros_like(dR1), ok1
    I2 = torch.where(mask, torch.zeros_like(I2), I2)
    src = -(0.5 * dR1 + dR2)
    return I2, T2, src, ok1 & ok2
