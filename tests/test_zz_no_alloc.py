"""rad_step_noalloc against rad_step.

rad_step_noalloc is the step for callers that may not allocate device
memory (a framework that owns all device memory through its own pool, or a
loop that cannot take cudaMalloc's implicit synchronisation): its stage
scratch lives in a 32 MiB static device array.  It runs the same kernels with
the same launch configuration as rad_step, only with another scratch
address, so two calls in a row must give exactly what two calls of rad_step
give (checked against the parity tolerance of the other GPU tests and then
bit for bit), for every option the step takes.  It makes the same host-side
checks as rad_step before anything is launched, and refuses a grid whose
scratch does not fit.  This file is collected last so that a run stopping
at its first failure has already run every other test."""
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


_RECON = {"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM,
          "mapr": rad.RAD_RECON_MAPR}

# (workload, cells, geodesic level, lat/long grid, precision, tolerance, options)
CASES = [
    ("torus3d", (8, 6, 4), 2, None, rad.RAD_F64, 1e-12, {}),
    ("turb3d", (9, 6, 7), 2, None, rad.RAD_F32, 2e-5, {}),
    ("adjoint2d", (10, 8, 1), 2, None, rad.RAD_F64, 1e-12, {}),
    ("turb3d", (9, 6, 7), 2, None, rad.RAD_F64, 1e-12, {"recon": "ppm"}),
    ("torus3d", (8, 6, 4), 2, None, rad.RAD_F32, 2e-5, {"recon": "ppm"}),
    ("torus3d", (6, 6, 4), 1, (4, 8), rad.RAD_F64, 1e-12, {"recon_ang": "plm"}),
    ("torus3d", (8, 6, 4), 2, None, rad.RAD_F64, 1e-12, {"recon_ang": "mapr"}),
    ("torus3d", (8, 6, 4), 2, None, rad.RAD_F32, 2e-5, {"recon_ang": "mapr", "recon": "ppm"}),
    ("turb3d", (9, 6, 7), 2, None, rad.RAD_F64, 1e-12, {"tau_const": 5.0}),
    ("torus3d", (8, 6, 4), 2, None, rad.RAD_F32, 2e-5, {"tau_const": 5.0}),
    ("turb3d", (9, 6, 7), 2, None, rad.RAD_F64, 1e-12, {"rad_dom": 1}),
]


@pytest.mark.parametrize("name,n,level,ll,prec,tol,extra", CASES)
def test_noalloc_step_matches_rad_step(name, n, level, ll, prec, tol, extra):
    w = W.make(name, n=n, level=level, latlong=ll)
    gc = GpuCase(w)
    fn = _lib()
    try:
        tdt = torch.float64 if prec == rad.RAD_F64 else torch.float32
        mode = {"thermal": rad.RAD_COUPLE_THERMAL, "emissivity": rad.RAD_COUPLE_EMISSIVITY}[w["mode"]]
        kw = dict(precision=prec, coupling=mode)
        for k, v in extra.items():
            kw[k] = _RECON[v] if k in ("recon", "recon_ang") else v
        o = rad.rad_opts_default(**kw)
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
        pairs = [(Ia.double().cpu().numpy(), Ib.double().cpu().numpy()),
                 (gas_a["T"].cpu().numpy(), gas_b["T"].cpu().numpy()),
                 (src_a.cpu().numpy(), src_b.cpu().numpy())]
        for a, b in pairs:
            assert np.abs(a - b).max() <= tol * max(np.abs(a).max(), 1e-300)
            assert np.array_equal(a, b)
    finally:
        gc.close()


def _refused(gc, o, gas, n_ap, prec=torch.float64):
    """Call rad_step_noalloc with arguments the host checks must refuse;
    returns (status, message).  Nothing is launched for a refused call."""
    fn = _lib()
    n = gc.w["n"]
    I = torch.zeros((n[2], n[1], n[0], n_ap), dtype=prec, device="cuda")
    g = rad._gas(gas)
    st = fn(gc.ctx, ctypes.c_void_p(I.data_ptr()), ctypes.byref(g), 1e-3, ctypes.byref(o), None)
    return st, rad.rad_last_error(gc.ctx)


def test_noalloc_refuses_what_rad_step_refuses():
    wg = W.make("torus3d", n=(6, 6, 4), level=2, with_intensity=False)
    gg = GpuCase(wg)
    wl = W.make("torus3d", n=(6, 6, 4), level=1, latlong=(4, 8), with_intensity=False)
    gl = GpuCase(wl)
    try:
        # angular PLM needs a latitude-longitude grid
        st, msg = _refused(gg, rad.rad_opts_default(recon_ang=rad.RAD_RECON_PLM), gg.gas(wg), gg.n_ap)
        assert st == rad.RAD_EUNSUPPORTED and "latitude-longitude" in msg
        # MAPR needs a geodesic grid
        st, msg = _refused(gl, rad.rad_opts_default(recon_ang=rad.RAD_RECON_MAPR), gl.gas(wl), gl.n_ap)
        assert st == rad.RAD_EUNSUPPORTED and "geodesic" in msg
        # the optical-depth weighting reads u and the opacities even without coupling
        gas = gg.gas(wg)
        gas["u"] = None
        o = rad.rad_opts_default(coupling=rad.RAD_COUPLE_NONE, tau_const=1.0)
        st, msg = _refused(gg, o, gas, gg.n_ap)
        assert st == rad.RAD_EINVAL and "optical-depth" in msg
        # rad_dom is 0 or 1, and only with the thermal coupling
        st, msg = _refused(gg, rad.rad_opts_default(rad_dom=2), gg.gas(wg), gg.n_ap)
        assert st == rad.RAD_EINVAL and "rad_dom" in msg
        o = rad.rad_opts_default(rad_dom=1, coupling=rad.RAD_COUPLE_EMISSIVITY)
        gas = gg.gas(wg)
        gas["eta"] = gas["rho"]
        st, msg = _refused(gg, o, gas, gg.n_ap)
        assert st == rad.RAD_EINVAL and "rad_dom" in msg
        # a NaN tau_const
        st, msg = _refused(gg, rad.rad_opts_default(tau_const=float("nan")), gg.gas(wg), gg.n_ap)
        assert st == rad.RAD_EINVAL and "tau_const" in msg
        # the context still steps normally afterwards
        rad.rad_check(gg.ctx)
    finally:
        gg.close()
        gl.close()


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
