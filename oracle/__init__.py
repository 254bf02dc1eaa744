"""Plain FP64 CPU oracle of the finite-solid-angle GR radiation update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the CUDA library and its Python binding)
never calls it, and this package never imports the product package.

Every function restates one step of White et al. (2023), "General
Relativistic Radiation with a Finite-Solid-Angle Method" (arXiv 2302.04283),
citing the section / equation it follows.  Arithmetic is float64 PyTorch CPU
ops (torch is used as an array library and, for the adjoint and the Ricci
rotation coefficients, as an automatic differentiator).  There is no
blocking, fusion or reordering beyond what the cited definition states.

Modules
-------
angles    geodesic angle grid (Sec. 2.6)
geometry  metric, tetrad, Ricci rotation coefficients, cell/face volumes
          (Sec. 2.1, Eq. tetrad, Eq. ricci, finite-volume averages of Sec. 2.2)
transport boundary fill, reconstruction, upwind spatial and angular fluxes
          (Secs. 2.3, 2.4, Eq. flux_space, Eq. flux_angle, Eq. radiation_integral)
coupling  locally implicit gas-radiation coupling (Sec. 2.5)
step      two-stage Runge-Kutta step with coupling and the n0crit guard
moments   R^{mu nu} = sum I n^mu n^nu dOmega in tetrad / coordinate / fluid frames
cfl       time-step bound
adjoint   outgoing-flux loss and its exact gradient (reverse-mode AD of step)
"""
import torch

DTYPE = torch.float64
