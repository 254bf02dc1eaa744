"""GPU parity of the angle grid, time-step bound, moments and loss, and the
C-ABI's argument checks."""
import math

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import adjoint as OA
from oracle import cfl as OCFL
from oracle import moments as OM
from oracle.angles import GeodesicGrid
from tests.harness import GpuCase, match_bins, oracle_setup, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("level", [1, 2, 4, 6, 8, 10])
def test_angle_grid_matches_oracle(level):
    ctx = rad.rad_create()
    try:
        na, nap = rad.rad_init_angles(ctx, level)
        assert na == 10 * level * level + 2 and nap % 4 == 0 and nap >= na
        d, w, nb = rad.rad_get_angles(ctx, na)
        ora = GeodesicGrid(level)
        g = match_bins(d, ora.dir.numpy())
        assert np.abs(w[g] - ora.dOmega.numpy()).max() < 1e-14
        inv = np.argsort(g)
        for n in range(na):
            mine = sorted(int(inv[m]) for m in nb[g[n]] if m >= 0)
            assert mine == sorted(ora.nbr[n])
    finally:
        rad.rad_destroy(ctx)


@pytest.mark.parametrize("level", [3, 4, 5, 7, 8, 9])
def test_bins_are_numbered_in_sign_pairs(level):
    """The library numbers its bins so that bins 2t and 2t + 1 have no
    direction component of opposite sign (the flat-space stage kernel's
    threads own such pairs); these levels admit a full pairing."""
    ctx = rad.rad_create()
    try:
        na, _ = rad.rad_init_angles(ctx, level)
        d, _, _ = rad.rad_get_angles(ctx, na)
        s = np.where(np.abs(d) < 1e-12, 0.0, np.sign(d))
        assert (s[0::2] * s[1::2] >= 0).all()
    finally:
        rad.rad_destroy(ctx)


@pytest.mark.parametrize("name,n,level", [("turb3d", (8, 6, 4), 2), ("torus3d", (8, 6, 4), 3),
                                          ("adjoint2d", (12, 8, 1), 2)])
def test_cfl_matches_oracle(name, n, level):
    w = W.make(name, n=n, level=level, with_intensity=False)
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        assert abs(rad.rad_cfl_dt(gc.ctx, 0.3) - OCFL.cfl_dt(st, 0.3)) < 1e-12 * OCFL.cfl_dt(st, 0.3)
    finally:
        gc.close()


@pytest.mark.parametrize("frame", [rad.RAD_FRAME_TETRAD, rad.RAD_FRAME_COORD, rad.RAD_FRAME_FLUID])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_moments_match_oracle(frame, prec):
    w = W.make("torus3d_big", n=(7, 6, 4), level=3)
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        tdt = torch.float64 if prec == "f64" else torch.float32
        Ig = gc.to_gpu_I(w["I0"], gmap, tdt)
        R = torch.zeros(Ig.shape[:-1] + (10,), dtype=tdt, device="cuda")
        rad.rad_moments(gc.ctx, Ig, rad.RAD_F64 if prec == "f64" else rad.RAD_F32, frame, rad.RAD_MOM_SIMT,
                        gc.gas(w), R)
        torch.cuda.synchronize()
        fr = {rad.RAD_FRAME_TETRAD: "tetrad", rad.RAD_FRAME_COORD: "coord", rad.RAD_FRAME_FLUID: "fluid"}[frame]
        ref = OM.moments(torch.tensor(w["I0"]), st.ang, fr, e=st.e, u=torch.tensor(w["u"])).numpy()
        tol = 1e-13 if prec == "f64" else 2e-6
        assert rel_err(R.double().cpu().numpy(), ref) < tol
    finally:
        gc.close()


def test_loss_and_seed_match_oracle():
    w = W.make("adjoint2d", n=(10, 8, 1), level=2)
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float64)
        L = torch.zeros(1, dtype=torch.float64, device="cuda")
        seed = torch.zeros_like(Ig)
        rad.rad_loss_outer(gc.ctx, Ig, rad.RAD_F64, L, seed)
        torch.cuda.synchronize()
        I0 = torch.tensor(w["I0"])
        assert abs(L.item() - float(OA.loss_outer(I0, st))) < 1e-13 * abs(float(OA.loss_outer(I0, st)))
        # the two grids' solid angles agree to rounding
        assert np.abs(gc.from_gpu_I(seed, gmap) - OA.loss_seed(I0, st).numpy()).max() < 1e-15
    finally:
        gc.close()


def test_argument_errors_are_reported():
    ctx = rad.rad_create()
    try:
        with pytest.raises(rad.RadError) as e:
            rad.rad_init_angles(ctx, 0)
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:
            rad.rad_cfl_dt(ctx, 0.3)
        assert e.value.status == rad.RAD_ESTATE
        rad.rad_init_angles(ctx, 2)
        xf = [np.linspace(0, 1, 5), np.linspace(0, 1, 5), np.array([0.0, 1.0])]
        with pytest.raises(rad.RadError) as e:     # polar on a Cartesian metric
            rad.rad_set_metric(ctx, "mink_cart", 0.0, 2, xf, (("periodic",) * 2, ("polar",) * 2, ("periodic",) * 2))
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:     # decreasing faces
            rad.rad_set_metric(ctx, "mink_cart", 0.0, 2, [xf[0][::-1].copy(), xf[1], xf[2]],
                               (("periodic",) * 2,) * 3)
        assert e.value.status == rad.RAD_EINVAL
        rad.rad_set_metric(ctx, "mink_cart", 0.0, 2, xf, (("periodic",) * 2,) * 3)
        I = torch.zeros(1, 4, 4, 44, dtype=torch.float64, device="cuda")
        o = rad.rad_opts_default()
        f = lambda *s: torch.ones(*s, dtype=torch.float64, device="cuda")
        gas = {"T": f(1, 4, 4), "rho": f(1, 4, 4), "u": 0 * f(1, 4, 4, 3), "alpha_a": f(1, 4, 4),
               "alpha_s": f(1, 4, 4)}
        with pytest.raises(rad.RadError) as e:     # dt <= 0
            rad.rad_step(ctx, I, gas, 0.0, o)
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:     # emissivity coupling without eta
            rad.rad_step(ctx, I, gas, 0.1, rad.rad_opts_default(coupling=rad.RAD_COUPLE_EMISSIVITY))
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:     # negative optical-depth constant
            rad.rad_step(ctx, I, gas, 0.1, rad.rad_opts_default(tau_const=-1.0))
        assert e.value.status == rad.RAD_EINVAL
        lam = torch.zeros_like(I)
        with pytest.raises(rad.RadError) as e:     # unknown reconstruction
            rad.rad_step(ctx, I, gas, 0.01, rad.rad_opts_default(recon=7))
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:     # the velocity substitution needs the thermal coupling
            rad.rad_step(ctx, I, gas, 0.01, rad.rad_opts_default(coupling=rad.RAD_COUPLE_NONE, rad_dom=1))
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:     # rad_dom is a flag
            rad.rad_step(ctx, I, gas, 0.01, rad.rad_opts_default(rad_dom=2))
        assert e.value.status == rad.RAD_EINVAL
        with pytest.raises(rad.RadError) as e:     # the adjoint checks the options like the step
            rad.rad_step_adjoint(ctx, I, gas, 0.01,
                                 rad.rad_opts_default(rad_dom=1, coupling=rad.RAD_COUPLE_EMISSIVITY),
                                 lam, torch.zeros_like(I), None, None, f(1, 4, 4), f(1, 4, 4))
        assert e.value.status == rad.RAD_EINVAL
        rad.rad_step(ctx, I, gas, 0.01, o)         # a valid call on the same context still works
        rad.rad_check(ctx)
    finally:
        rad.rad_destroy(ctx)


def test_empty_and_tiny_grids():
    """A grid without cells is refused; one cell with periodic boundaries
    everywhere is its own neighbour."""
    ctx = rad.rad_create(torch.cuda.current_stream())
    try:
        rad.rad_init_angles(ctx, 1)
        with pytest.raises(rad.RadError) as e:
            rad.rad_set_metric(ctx, "mink_cart", 0.0, 3, [np.zeros(1), np.linspace(0, 1, 3), np.linspace(0, 1, 3)],
                               (("periodic", "periodic"),) * 3)
        assert e.value.status == rad.RAD_EINVAL
    finally:
        rad.rad_destroy(ctx)
    w = W.make("turb3d", n=(1, 1, 1), level=1)
    from tests.harness import run_both
    r = run_both(w, 2, "f64")
    try:
        assert rel_err(r["I_g"], r["I_o"]) < 1e-12
    finally:
        r["gc"].close()


@pytest.mark.parametrize("frame", [rad.RAD_FRAME_TETRAD, rad.RAD_FRAME_COORD, rad.RAD_FRAME_FLUID])
@pytest.mark.parametrize("level,n", [(3, (7, 6, 4)), (2, (33, 5, 4)), (8, (5, 4, 2))])
def test_moments_split_bf16_tensor_cores(frame, level, n):
    """Split-bf16 tcgen05 moments vs the FP64 oracle.  Tolerance: every
    component within 1e-4 of the cell's R^00 (three bf16 products with FP32
    accumulation: about 2^-16 relative per term)."""
    w = W.make("torus3d_big", n=n, level=level)
    gc = GpuCase(w)
    try:
        st = oracle_setup(w)
        gmap = match_bins(gc.dir, st.ang.dir.numpy())
        Ig = gc.to_gpu_I(w["I0"], gmap, torch.float32)
        R = torch.full(Ig.shape[:-1] + (10,), float("nan"), dtype=torch.float32, device="cuda")
        rad.rad_moments(gc.ctx, Ig, rad.RAD_F32, frame, rad.RAD_MOM_BF16X3, gc.gas(w), R)
        torch.cuda.synchronize()
        rad.rad_check(gc.ctx)
        fr = {rad.RAD_FRAME_TETRAD: "tetrad", rad.RAD_FRAME_COORD: "coord", rad.RAD_FRAME_FLUID: "fluid"}[frame]
        ref = OM.moments(torch.tensor(w["I0"]), st.ang, fr, e=st.e, u=torch.tensor(w["u"])).numpy()
        got = R.double().cpu().numpy()
        scale = np.abs(ref[..., :1])
        assert np.isfinite(got).all()
        assert (np.abs(got - ref) / scale).max() < 1e-4
    finally:
        gc.close()


def test_element_limit_is_refused():
    """256 x 256 x 261 cells x 252 bins = 4.31e9 > 2^32 elements: refused with
    RAD_EUNSUPPORTED before any scratch is allocated or kernel launched (the
    17 GB FP32 intensity buffer itself is allocated, so no access could leave
    it even without the check)."""
    n = (256, 256, 261)
    ctx = rad.rad_create(torch.cuda.current_stream())
    try:
        na, nap = rad.rad_init_angles(ctx, 5)
        xf = [np.linspace(0, 1, m + 1) for m in n]
        rad.rad_set_metric(ctx, "mink_cart", 0.0, 3, xf, (("periodic", "periodic"),) * 3)
        assert n[0] * n[1] * n[2] * nap > 2 ** 32
        I = torch.empty((n[2], n[1], n[0], nap), dtype=torch.float32, device="cuda")
        sh = (n[2], n[1], n[0])
        gas = {k: torch.ones(sh, dtype=torch.float64, device="cuda") for k in ("rho", "alpha_a", "alpha_s", "T")}
        gas["u"] = torch.zeros(sh + (3,), dtype=torch.float64, device="cuda")
        gas["eta"] = None
        o = rad.rad_opts_default(precision=rad.RAD_F32)
        with pytest.raises(rad.RadError) as e:
            rad.rad_step(ctx, I, gas, 1e-3, o)
        assert e.value.status == rad.RAD_EUNSUPPORTED
        del I
    finally:
        rad.rad_destroy(ctx)
        torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_host_pipeline_matches_device_path(prec):
    """rad_step_host on seven items (different intensities and temperatures,
    pinned and pageable host buffers, with and without I_out; more items than
    device slots, so slots are reused) gives bit for bit what rad_step +
    rad_moments give on device copies of the same inputs."""
    w = W.make("torus3d_big", n=(6, 4, 4), level=2)
    gc = GpuCase(w)
    try:
        f32 = prec == "f32"
        tdt = torch.float32 if f32 else torch.float64
        o = rad.rad_opts_default(precision=rad.RAD_F32 if f32 else rad.RAD_F64)
        method = rad.RAD_MOM_BF16X3 if f32 else rad.RAD_MOM_SIMT
        dt = rad.rad_cfl_dt(gc.ctx, 0.3)
        sh = w["T"].shape
        rng = np.random.default_rng(4)
        items, expect = [], []
        for n in range(7):
            I = np.zeros(sh + (gc.n_ap,))
            I[..., :gc.n_ang] = rng.uniform(0.5, 1.5, sh + (gc.n_ang,)) / (4 * np.pi)
            T = rng.uniform(0.8, 1.2, sh)
            pin = n not in (1, 4)
            h = lambda a, dtp=torch.float64: (torch.tensor(a, dtype=dtp).pin_memory() if pin
                                              else torch.tensor(a, dtype=dtp))
            item = {"I": h(I, tdt), "rho": h(w["rho"]), "u": h(w["u"]), "alpha_a": h(w["alpha_a"]),
                    "alpha_s": h(w["alpha_s"]), "eta": None, "T": h(T),
                    "R": torch.full(sh + (10,), float("nan"), dtype=tdt),
                    "I_out": None if n == 5 else torch.zeros(sh + (gc.n_ap,), dtype=tdt)}
            items.append(item)
            # device path
            Id = torch.tensor(I, dtype=tdt, device="cuda")
            gas = gc.gas(w, T=T)
            for _ in range(2):
                rad.rad_step(gc.ctx, Id, gas, dt, o)
            Rd = torch.zeros(sh + (10,), dtype=tdt, device="cuda")
            rad.rad_moments(gc.ctx, Id, o.precision, rad.RAD_FRAME_TETRAD, method, gas, Rd)
            torch.cuda.synchronize()
            expect.append((Id.cpu(), gas["T"].cpu(), Rd.cpu()))
        rad.rad_step_host(gc.ctx, items, dt, o, 2, rad.RAD_FRAME_TETRAD, method)
        rad.rad_check(gc.ctx)
        for item, (Ie, Te, Re) in zip(items, expect):
            if item["I_out"] is not None:
                assert torch.equal(item["I_out"], Ie)
            assert torch.equal(item["T"], Te)
            assert torch.equal(item["R"], Re)
    finally:
        gc.close()


def test_bounded_device_wait_reports_a_timeout():
    """A device wait on an mbarrier that nothing arrives at gives up after its
    time limit and records the timeout status, which rad_check reads; the
    context stays usable (a step afterwards succeeds)."""
    import time
    w = W.make("turb3d", n=(4, 4, 4), level=1)
    gc = GpuCase(w)
    try:
        t0 = time.time()
        rad.rad_selftest_wait(gc.ctx, 0.2)
        with pytest.raises(rad.RadError) as e:
            rad.rad_check(gc.ctx)
        assert e.value.status == rad.RAD_ECUDA and "timed out" in str(e.value)
        assert 0.15 < time.time() - t0 < 5.0
        rad.rad_check(gc.ctx)                      # the word was cleared
        I = gc.to_gpu_I(w["I0"], np.arange(gc.n_ang), torch.float64)
        rad.rad_step(gc.ctx, I, gc.gas(w), 1e-3, rad.rad_opts_default())
        rad.rad_check(gc.ctx)
        with pytest.raises(rad.RadError) as e:
            rad.rad_selftest_wait(gc.ctx, 0.0)
        assert e.value.status == rad.RAD_EINVAL
    finally:
        gc.close()


def test_fp64_fma_rate_is_measured():
    """The measured FP64 FMA rate (the FP64 kernels' roofline denominator) is
    a positive rate of the order GB300's FP64 units give (nominal 1.25
    TFLOP/s), not a placeholder."""
    r = rad.rad_fp64_fma_rate(1.0)
    assert 0.1 < r < 100.0, r
