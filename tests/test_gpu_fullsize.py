"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (rad_step with the default options, then
rad_moments), on sampled outputs.

One RK2 step of a cell depends only on the cells within four of it in each
flux dimension (two stages of a stencil that reaches two cells), so the
oracle advances the 9 x 9 x 9 block around each sampled cell (cut from the
full inputs with periodic wrap where the boundary is periodic) and compares
the block's centre.  Sampled cells of the Kerr-Schild torus keep four cells
away from the radial and polar boundaries.

Tolerances: FP64 1e-12 relative (per cell, max over bins / max over bins);
the FP64 gas source 1e-11 of its own size plus 1e-13 of the cell's R^00 (it
is the change of R^0_mu over the coupling, rounded at the scale of R); FP32
transport 2e-5; moments: FP64 1e-12 of R^00, split-BF16 after the FP32
step 1.5e-4 of R^00 (1e-4 for the tensor-core contraction plus the step's
2e-5 relative error weighted by max I / mean I <= 1.25 for these inputs)."""
import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle import moments as OM
from oracle import step as OS
from oracle.angles import GeodesicGrid
from oracle.transport import Grid, Setup
from tests.harness import match_bins

pytestmark = pytest.mark.gpu

HALO = 4
NSAMPLE = 5


def _block_faces(xf, c, periodic):
    """Face coordinates of cells c-4 .. c+4 (a uniform window when periodic)."""
    if periodic:
        dx = float(xf[1] - xf[0])
        return xf[0] + dx * (np.arange(2 * HALO + 2) + c - HALO)
    return xf[c - HALO:c + HALO + 2]


def _samples(w, rng):
    n1, n2, n3 = w["n"]
    if w["kind"] == "mink_cart":
        lo = (0, 0)
        hi = (n1, n2)
    else:
        lo = (HALO, HALO)
        hi = (n1 - HALO, n2 - HALO)
    return [(int(rng.integers(0, n3)), int(rng.integers(lo[1], hi[1])), int(rng.integers(lo[0], hi[0])))
            for _ in range(NSAMPLE)]


def _oracle_block(w, ang, cell, dt):
    k, j, i = cell
    n1, n2, n3 = w["n"]
    per = [b[0] == "periodic" for b in w["bc"]]
    ii = np.arange(i - HALO, i + HALO + 1) % n1
    jj = np.arange(j - HALO, j + HALO + 1) % n2
    kk = np.arange(k - HALO, k + HALO + 1) % n3
    xf = [_block_faces(w["xf"][0], i, per[0]), _block_faces(w["xf"][1], j, per[1]),
          _block_faces(w["xf"][2], k, per[2])]
    st = Setup(Grid(w["kind"], w["spin"], xf, (("outflow", "outflow"),) * 3, 3), ang)
    cut = lambda a: torch.tensor(np.ascontiguousarray(a[np.ix_(kk, jj, ii)]))
    gas = {key: cut(w[key]) for key in ("rho", "u", "alpha_a", "alpha_s")}
    gas["eta"] = None
    I, T, src, ok = OS.rk2_step(cut(w["I0"]), cut(w["T"]), gas, dt, st, OS.Opts())
    assert bool(ok.all())
    c = (HALO, HALO, HALO)
    R = OM.moments(I[c][None, None, None], ang)[0, 0, 0]
    return I[c].numpy(), float(T[c]), src[c].numpy(), R.numpy()


@pytest.fixture(scope="module", params=["turb3d", "torus3d"])
def full(request):
    w = W.make(request.param)
    ang = GeodesicGrid(w["level"])
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, w["level"])
    gdir, _, _ = rad.rad_get_angles(ctx, na)
    rad.rad_set_metric(ctx, w["kind"], w["spin"], w["ndim"], w["xf"], w["bc"])
    dt = rad.rad_cfl_dt(ctx, w["cfl"])
    gmap = match_bins(gdir, ang.dir.numpy())
    sh = w["I0"].shape[:-1]
    Ih = np.zeros(sh + (nap,))
    Ih[..., gmap] = w["I0"]
    rng = np.random.default_rng(11)
    cells = _samples(w, rng)
    ref = {c: _oracle_block(w, ang, c, dt) for c in cells}
    yield w, ctx, na, nap, dt, gmap, Ih, cells, ref
    torch.cuda.synchronize()
    rad.rad_destroy(ctx)


def _gas(w):
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g = {key: t(w[key]) for key in ("rho", "u", "alpha_a", "alpha_s", "T")}
    g["eta"] = None
    return g


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_full_size_step_and_moments(full, prec):
    w, ctx, na, nap, dt, gmap, Ih, cells, ref = full
    f32 = prec == "f32"
    I = torch.tensor(Ih, dtype=torch.float32 if f32 else torch.float64, device="cuda")
    gas = _gas(w)
    src = torch.zeros(I.shape[:-1] + (4,), dtype=torch.float64, device="cuda")
    o = rad.rad_opts_default(precision=rad.RAD_F32 if f32 else rad.RAD_F64)
    rad.rad_step(ctx, I, gas, dt, o, src)
    R = torch.zeros(I.shape[:-1] + (10,), dtype=I.dtype, device="cuda")
    rad.rad_moments(ctx, I, rad.RAD_F32 if f32 else rad.RAD_F64, rad.RAD_FRAME_TETRAD,
                    rad.RAD_MOM_BF16X3 if f32 else rad.RAD_MOM_SIMT, gas, R)
    torch.cuda.synchronize()
    rad.rad_check(ctx)
    tol = 2e-5 if f32 else 1e-12
    rtol = 1.5e-4 if f32 else 1e-12
    for c in cells:
        I_o, T_o, src_o, R_o = ref[c]
        I_g = I[c].double().cpu().numpy()[gmap]
        assert np.abs(I_g - I_o).max() <= tol * np.abs(I_o).max(), (prec, c)
        assert abs(float(gas["T"][c]) - T_o) <= tol * abs(T_o), (prec, c)
        if not f32:
            s_g = src[c].cpu().numpy()
            # the source is a difference of radiation four-momenta before and
            # after the coupling: its rounding scale is R^00, not |src|
            assert np.abs(s_g - src_o).max() <= 1e-11 * np.abs(src_o).max() + 1e-13 * abs(R_o[0]), c
        R_g = R[c].double().cpu().numpy()
        assert np.abs(R_g - R_o).max() <= rtol * abs(R_o[0]), (prec, c)
        # padding bins are written as zero
        assert float(I[c][na:].abs().max()) == 0.0 if nap > na else True
