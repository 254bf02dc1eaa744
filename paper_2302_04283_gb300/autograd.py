"""torch.autograd bridge for the radiation step (argument marshalling only).

RadStepFn.apply(I, alpha_a, alpha_s, eta, step) runs rad_step on a copy of
I and, on the backward pass, rad_step_adjoint from the saved checkpoint I
(per-step checkpointing with recomputation inside the library).  The
gradient flows to I, alpha_a, alpha_s and eta.  Coupling must be the
fixed-emissivity (or no) coupling, where the gas temperature is frozen.

RadStepThermalFn.apply(I, T, alpha_a, alpha_s, step) is the same for the
thermal coupling: it returns (I, T) after the step, and the gradient flows
to I, T, alpha_a and alpha_s (through the quartic's root).
"""
import torch

from . import (rad_loss_outer, rad_step, rad_step_adjoint)


class StepConfig:
    """Everything the step needs besides the differentiated tensors."""

    def __init__(self, ctx, gas, dt, opts):
        self.ctx, self.gas, self.dt, self.opts = ctx, gas, dt, opts


class RadStepFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, I, alpha_a, alpha_s, eta, cfg):
        gas = dict(cfg.gas)
        gas.update(alpha_a=alpha_a.detach(), alpha_s=alpha_s.detach(),
                   eta=eta.detach() if eta is not None else None)
        out = I.detach().clone()
        T = gas["T"].clone()
        gas["T"] = T
        rad_step(cfg.ctx, out, gas, cfg.dt, cfg.opts)
        fctx.save_for_backward(I.detach(), alpha_a.detach(), alpha_s.detach(),
                               eta.detach() if eta is not None else torch.empty(0))
        fctx.cfg = cfg
        fctx.has_eta = eta is not None
        return out

    @staticmethod
    def backward(fctx, lam):
        I_n, aa, as_, eta = fctx.saved_tensors
        cfg = fctx.cfg
        gas = dict(cfg.gas)
        gas.update(alpha_a=aa, alpha_s=as_, eta=eta if fctx.has_eta else None)
        lam_n = torch.empty_like(I_n)
        g_aa = torch.zeros_like(aa)
        g_as = torch.zeros_like(as_)
        g_eta = torch.zeros_like(eta) if fctx.has_eta else None
        rad_step_adjoint(cfg.ctx, I_n, gas, cfg.dt, cfg.opts, lam.contiguous(), lam_n, None, None, g_aa, g_as,
                         g_eta)
        return lam_n, g_aa, g_as, g_eta, None


class RadStepThermalFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, I, T, alpha_a, alpha_s, cfg):
        gas = dict(cfg.gas)
        T_out = T.detach().clone()
        gas.update(alpha_a=alpha_a.detach(), alpha_s=alpha_s.detach(), eta=None, T=T_out)
        out = I.detach().clone()
        rad_step(cfg.ctx, out, gas, cfg.dt, cfg.opts)
        fctx.save_for_backward(I.detach(), T.detach(), alpha_a.detach(), alpha_s.detach())
        fctx.cfg = cfg
        return out, T_out

    @staticmethod
    def backward(fctx, lam, lamT):
        I_n, T_n, aa, as_ = fctx.saved_tensors
        cfg = fctx.cfg
        gas = dict(cfg.gas)
        gas.update(alpha_a=aa, alpha_s=as_, eta=None, T=T_n)
        lam = torch.zeros_like(I_n) if lam is None else lam.contiguous()
        lamT = None if lamT is None else lamT.contiguous()
        lam_n = torch.empty_like(I_n)
        lamT_n = torch.empty_like(T_n)
        g_aa = torch.zeros_like(aa)
        g_as = torch.zeros_like(as_)
        rad_step_adjoint(cfg.ctx, I_n, gas, cfg.dt, cfg.opts, lam, lam_n, lamT, lamT_n, g_aa, g_as, None)
        return lam_n, lamT_n, g_aa, g_as, None


class OuterLossFn(torch.autograd.Function):
    """L = outgoing-flux loss of rad_loss_outer, with its seed as gradient."""

    @staticmethod
    def forward(fctx, I, ctx, precision):
        L = torch.zeros(1, dtype=torch.float64, device=I.device)
        seed = torch.empty_like(I)
        rad_loss_outer(ctx, I.detach(), precision, L, seed)
        fctx.save_for_backward(seed)
        return L[0]

    @staticmethod
    def backward(fctx, g):
        (seed,) = fctx.saved_tensors
        return seed * g.to(seed.dtype), None, None
