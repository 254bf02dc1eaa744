"""rad_step_noalloc against rad_step.

rad_step_noalloc is the step for callers that may not allocate device
memory (a framework that owns all device memory through its own pool, or a
loop that cannot take cudaMalloc's implicit synchronisation): its stage
scratch lives in a 32 MiB static device array.  Two calls in a row must give
what two calls of rad_step give, within the parity tolerances of the other
GPU tests, and a grid that does not fit must be refused.  This file is
collected last so that a run stopping at its first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from tests.harness import GpuCase

pytestmark = pytest.mark.gpu


def _lib():
    L = rad.lib()
    fn = L.rad_step_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(rad.rad_gas), ctypes.c_double,
                   ctypes.POINTER(rad.rad_opts), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _state(gc, w, tdt):
    I = torch.tensor(w["I0"], dtype=tdt, device="cuda")
    I = torch.nn.functional.pad(I, (0, gc.n_ap - gc.n_ang)).contiguous()
    gas = gc.gas(w)
    src = torch.zeros(I.shape[:-1] + (4,), dtype=torch.float64, device="cuda")
    return I, gas, src


@pytest.mark.parametrize("name,n,level,prec,tol", [
    ("torus3d", (8, 6, 4), 2, rad.RAD_F64, 1e-12),
    ("turb3d", (9, 6, 7), 2, rad.RAD_F32, 2e-5),
    ("adjoint2d", (10, 8, 1), 2, rad.RAD_F64, 1e-12),
])
def test_noalloc_step_matches_rad_step(name, n, level, prec, tol):
    w = W.make(name, n=n, level=level)
    gc = GpuCase(w)
    fn = _lib()
    try:
        tdt = torch.float64 if prec == rad.RAD_F64 else torch.float32
        mode = {"thermal": rad.RAD_COUPLE_THERMAL, "emissivity": rad.RAD_COUPLE_EMISSIVITY}[w["mode"]]
        o = rad.rad_opts_default(precision=prec, coupling=mode)
        dt = rad.rad_cfl_dt(gc.ctx, w["cfl"])
        Ia, gas_a, src_a = _state(gc, w, tdt)
        Ib, gas_b, src_b = _state(gc, w, tdt)
        for _ in range(2):
            rad.rad_step(gc.ctx, Ia, gas_a, dt, o, src_a)
        for _ in range(2):
            g = rad._gas(gas_b)
            st = fn(gc.ctx, ctypes.c_void_p(Ib.data_ptr()), ctypes.byref(g), dt, ctypes.byref(o),
                    ctypes.c_void_p(src_b.data_ptr()))
            assert st == rad.RAD_OK, rad.rad_last_error(gc.ctx)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        a, b = Ia.double().cpu().numpy(), Ib.double().cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(a).max()
        ta, tb = gas_a["T"].cpu().numpy(), gas_b["T"].cpu().numpy()
        assert np.abs(ta - tb).max() <= tol * np.abs(ta).max()
        sa, sb = src_a.cpu().numpy(), src_b.cpu().numpy()
        assert np.abs(sa - sb).max() <= tol * max(np.abs(sa).max(), 1e-300)
    finally:
        gc.close()


def test_noalloc_refuses_a_grid_beyond_its_scratch():
    # 64 x 64 x 16 cells x 164 bins in FP64 needs ~86 MB of stage scratch
    w = W.make("turb3d", n=(64, 64, 16), level=4, with_intensity=False)
    gc = GpuCase(w)
    fn = _lib()
    try:
        I = torch.zeros((16, 64, 64, gc.n_ap), dtype=torch.float64, device="cuda")
        gas = gc.gas(w)
        g = rad._gas(gas)
        o = rad.rad_opts_default()
        st = fn(gc.ctx, ctypes.c_void_p(I.data_ptr()), ctypes.byref(g), 1e-3, ctypes.byref(o), None)
        assert st == rad.RAD_EINVAL
        assert "static array" in rad.rad_last_error(gc.ctx)
    finally:
        gc.close()
