"""Every three-dimensional benchmark workload at its full size and its stated
number of RK2 steps, in the launch configuration bench.py times, against the
FP64 oracle's values stored by tests/golden/make_config_samples.py and
tests/golden/make_torus3d_big_subvolume.py (oracle-only scripts):

  turb3d       128^3 x 162 bins, 10 steps: 4096 sampled cells (T, gas
               source, moments) and 8192 sampled (cell, bin) intensities
  torus3d      128 x 64 x 64 x 362 bins, 5 steps: the same, the samples
               including every cell within four of the radial and polar
               boundaries in several lines
  torus3d_big  192 x 96 x 96 x 642 bins, 20 steps: the whole 24^3 subvolume
               at r ~ 10, theta = pi/2, phi = 0 (T, moments) and 8192
               sampled intensities — the precision sweep FP64 / FP32 /
               FP32 + split-BF16 moments

Each comparison reports the normwise relative error (max |d| / max |ref|)
and the largest per-element relative error (max |d| / |ref|), and asserts
the stated tolerances: FP64 1e-12 normwise (source 1e-11 of its size plus
1e-13 of R^00), FP32 after the stated steps 2e-5 normwise for I, T and the
FP32 moments, split-BF16 moments 1.5e-4 of R^00 per component."""
import json
import math
import os

import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from oracle.angles import GeodesicGrid
from tests.harness import match_bins

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RESULTS = {}


def _golden(name):
    f = os.path.join(GOLDEN, name)
    if not os.path.exists(f):
        pytest.skip(f"{name} has not been generated")
    return np.load(f)


def _run(w, prec, steps, dt, method):
    """The workload through rad_step (default options) x steps, then
    rad_moments; the initial intensity is uploaded one x3 slab at a time."""
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, w["level"])
    gdir, _, _ = rad.rad_get_angles(ctx, na)
    rad.rad_set_metric(ctx, w["kind"], w["spin"], w["ndim"], w["xf"], w["bc"])
    dt_gpu = rad.rad_cfl_dt(ctx, w["cfl"])
    assert abs(dt_gpu - dt) <= 1e-12 * dt                     # the oracle's bound
    gmap = match_bins(gdir, GeodesicGrid(w["level"]).dir.numpy())
    f32 = prec == "f32"
    tdt = torch.float32 if f32 else torch.float64
    n1, n2, n3 = w["n"]
    I = torch.zeros((n3, n2, n1, nap), dtype=tdt, device="cuda")
    for k in range(n3):
        row = np.zeros((n2, n1, nap))
        row[..., gmap] = W.intensity_rows(w, k)
        I[k] = torch.tensor(row, device="cuda").to(tdt)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    gas = {k: t(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s", "T")}
    gas["eta"] = None
    src = torch.zeros((n3, n2, n1, 4), dtype=torch.float64, device="cuda")
    o = rad.rad_opts_default(precision=rad.RAD_F32 if f32 else rad.RAD_F64)
    for _ in range(steps):
        rad.rad_step(ctx, I, gas, dt, o, src)
    R = torch.zeros((n3, n2, n1, 10), dtype=tdt, device="cuda")
    rad.rad_moments(ctx, I, rad.RAD_F32 if f32 else rad.RAD_F64, rad.RAD_FRAME_TETRAD, method, gas, R)
    torch.cuda.synchronize()
    rad.rad_check(ctx)
    rad.rad_destroy(ctx)
    return I, gas["T"], src, R, gmap


def _errs(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    return float(d.max() / np.abs(b).max()), float((d / np.maximum(np.abs(b), 1e-300)).max())


def _record(key, **v):
    RESULTS[key] = v
    out = os.environ.get("RAD_CONFIG_ERRORS")
    if out:
        with open(out, "w") as fh:
            json.dump(RESULTS, fh, indent=1)


CASES = [("f64", rad.RAD_MOM_SIMT), ("f32", rad.RAD_MOM_SIMT), ("f32", rad.RAD_MOM_BF16X3)]


@pytest.mark.parametrize("name", ["turb3d", "torus3d"])
@pytest.mark.parametrize("prec,method", CASES)
def test_config_at_stated_steps(name, prec, method):
    g = _golden(f"{name}_samples.npz")
    w = W.make(name, with_intensity=False)
    steps = int(g["steps"])
    assert steps == w["nsteps"]
    I, T, src, R, gmap = _run(w, prec, steps, float(g["dt"]), method)
    c = g["cells"]
    kc, jc, ic = (torch.tensor(c[:, q], device="cuda") for q in range(3))
    bc = g["bin_cells"]
    Ig = I[torch.tensor(bc[:, 0]), torch.tensor(bc[:, 1]), torch.tensor(bc[:, 2]),
           torch.tensor(gmap[g["bins"]])].double().cpu().numpy()
    eI = _errs(Ig, g["I"])
    eT = _errs(T[kc, jc, ic].cpu().numpy(), g["T"])
    Rg = R[kc, jc, ic].double().cpu().numpy()
    eR = float((np.abs(Rg - g["R"]) / np.abs(g["R"][:, :1])).max())
    es = _errs(src[kc, jc, ic].cpu().numpy(), g["src"])
    bf16 = method == rad.RAD_MOM_BF16X3
    _record(f"{name}/{prec}{'+bf16' if bf16 else ''}", steps=steps, I=eI, T=eT, R_over_R00=eR, src=es)
    if prec == "f64":
        assert eI[0] < 1e-12 and eT[0] < 1e-12 and eR < 1e-12, (eI, eT, eR)
        sref = g["src"]
        assert np.abs(src[kc, jc, ic].cpu().numpy() - sref).max() <= \
            1e-11 * np.abs(sref).max() + 1e-13 * np.abs(g["R"][:, 0]).max()
    else:
        assert eI[0] < 2e-5 and eT[0] < 2e-5, (eI, eT)
        assert eR < (1.5e-4 if bf16 else 2e-5), eR
    if name == "torus3d":
        # the boundary lines are among the samples
        assert (c[:, 1] < 4).any() and (c[:, 1] >= w["n"][1] - 4).any()
        assert (c[:, 2] < 4).any() and (c[:, 2] >= w["n"][0] - 4).any()


@pytest.mark.parametrize("prec,method", CASES)
def test_torus3d_big_subvolume_at_20_steps(prec, method):
    g = _golden("torus3d_big_subvolume.npz")
    w = W.make("torus3d_big", with_intensity=False)
    steps = int(g["steps"])
    assert steps == w["nsteps"] == 20
    I, T, src, R, gmap = _run(w, prec, steps, float(g["dt"]), method)
    i0, j0, k0 = (int(x) for x in g["origin"])
    S = int(g["sub"])
    n3 = w["n"][2]
    kk = torch.tensor(np.arange(k0, k0 + S) % n3, device="cuda")
    sub = lambda X: X[kk][:, j0:j0 + S, i0:i0 + S]
    eT = _errs(sub(T).cpu().numpy(), g["T"])
    Rg = sub(R).double().cpu().numpy()
    eR = float((np.abs(Rg - g["R"]) / np.abs(g["R"][..., :1])).max())
    c = g["sample_cells"]
    Is = sub(I).double().cpu().numpy()[c[:, 0], c[:, 1], c[:, 2]][np.arange(len(c)), gmap[g["sample_bins"]]]
    eI = _errs(Is, g["sample_I"])
    bf16 = method == rad.RAD_MOM_BF16X3
    _record(f"torus3d_big/{prec}{'+bf16' if bf16 else ''}", steps=steps, I=eI, T=eT, R_over_R00=eR,
            margin_diff=float(g["margin_diff"]))
    if prec == "f64":
        assert eI[0] < 1e-12 and eT[0] < 1e-12 and eR < 1e-12, (eI, eT, eR)
    else:
        assert eI[0] < 2e-5 and eT[0] < 2e-5, (eI, eT)
        assert eR < (1.5e-4 if bf16 else 2e-5), eR
