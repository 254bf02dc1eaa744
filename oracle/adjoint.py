"""Outgoing-flux loss and its exact gradient.

The gradient of a scalar loss through one step is, by definition, the
vector-Jacobian product of the step.  The oracle obtains it by reverse-mode
automatic differentiation of the plain forward code in step.py (the quartic
root enters through one attached Newton step, i.e. the implicit-function
theorem), so it shares nothing with a hand-written adjoint.

Loss (reading of the outgoing-flux loss): the solid-angle weighted
intensity of the outermost x1 cells, over bins that move outward
(n^1 > 0) at the outer x1 face:
    L = sum_{k, j} sum_{n : n^1_face > 0} I[k, j, N1 - 1, n] dOmega_n
"""
import torch

from . import step as S


def outgoing_mask(setup):
    return setup.fsign[0][:, :, -1, :] > 0.0          # [k, j, n] at the outer x1 face


def loss_outer(I, setup):
    m = outgoing_mask(setup).to(I.dtype)
    return (I[:, :, -1, :] * m * setup.ang.dOmega).sum()


def loss_seed(I, setup):
    """dL/dI: dOmega_n on the outward bins of the outer cells, 0 elsewhere."""
    g = torch.zeros_like(I)
    g[:, :, -1, :] = outgoing_mask(setup).to(I.dtype) * setup.ang.dOmega
    return g


def step_vjp(I0, T0, gas, dt, setup, opts, lam, lamT=None):
    """(lambda_n, lambdaT_n, g_alpha_a, g_alpha_s, g_eta) for one step.

    lambda_n = (d I_{n+1} / d I_n)^T lambda (+ the T path), and g_theta the
    gradient of <lambda, I_{n+1}> + <lambdaT, T_{n+1}> w.r.t. each field.
    """
    I0 = I0.detach().clone().requires_grad_(True)
    T0 = T0.detach().clone().requires_grad_(True)
    g = {k: (v.detach().clone().requires_grad_(k in ("alpha_a", "alpha_s", "eta"))
             if v is not None else None) for k, v in gas.items()}
    I2, T2, _, _ = S.rk2_step(I0, T0, g, dt, setup, opts)
    obj = (I2 * lam).sum()
    if lamT is not None:
        obj = obj + (T2 * lamT).sum()
    wrt = [I0, T0, g["alpha_a"], g["alpha_s"]]
    has_eta = g.get("eta") is not None
    if has_eta:
        wrt.append(g["eta"])
    grads = torch.autograd.grad(obj, wrt, allow_unused=True)
    grads = [torch.zeros_like(w) if gr is None else gr for gr, w in zip(grads, wrt)]
    out = grads[:4] + ([grads[4]] if has_eta else [None])
    return tuple(out)


def gradient(I0, T0, gas, dt, setup, opts, nsteps):
    """dL/d(alpha_a, alpha_s, eta) of L(I after nsteps) by reverse-mode AD."""
    g = {k: (v.detach().clone().requires_grad_(k in ("alpha_a", "alpha_s", "eta"))
             if v is not None else None) for k, v in gas.items()}
    I, T = I0.detach(), T0.detach()
    for _ in range(nsteps):
        I, T, _, _ = S.rk2_step(I, T, g, dt, setup, opts)
    L = loss_outer(I, setup)
    wrt = [g["alpha_a"], g["alpha_s"]] + ([g["eta"]] if g.get("eta") is not None else [])
    grads = torch.autograd.grad(L, wrt, allow_unused=True)
    return L.detach(), [torch.zeros_like(w) if gr is None else gr for gr, w in zip(grads, wrt)]
