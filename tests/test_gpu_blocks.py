"""Blocks of a decomposed domain on one GPU, through the C ABI: every block
is its own context (its cells, RAD_BC_HALO on shared faces), stepped one
stage at a time with rad_step_stage after its neighbours' rad_halo_pack
layers have been copied into its halo buffers (the exchange that messages
between GPUs perform in a multi-GPU run).  The assembled result must equal
rad_step on the undivided domain bit for bit: the per-cell arithmetic does
not depend on the block; the blocks' outgoing-flux losses add up to the
undivided loss.  Also: the calls that refuse shared faces."""
import numpy as np
import pytest
import torch

import paper_2302_04283_gb300 as rad
import workloads as W
from paper_2302_04283_gb300 import blocks as B

pytestmark = pytest.mark.gpu

R = {"dc": rad.RAD_RECON_DC, "plm": rad.RAD_RECON_PLM, "ppm": rad.RAD_RECON_PPM, "mapr": rad.RAD_RECON_MAPR}


def _ctx(w, xf, bc):
    ctx = rad.rad_create(torch.cuda.current_stream())
    na, nap = rad.rad_init_angles(ctx, w["level"])
    rad.rad_set_metric(ctx, w["kind"], w["spin"], w["ndim"], xf, bc)
    return ctx, na, nap


def _gas(w, sl=None):
    t = lambda a: torch.tensor(np.ascontiguousarray(a if sl is None else a[sl]), dtype=torch.float64,
                               device="cuda")
    g = {k: t(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s", "T")}
    g["eta"] = t(w["eta"]) if w["eta"] is not None else None
    return g


def _initial(w, nap, tdt):
    I = torch.zeros(w["I0"].shape[:-1] + (nap,), dtype=tdt, device="cuda")
    I[..., :w["I0"].shape[-1]] = torch.tensor(w["I0"], device="cuda").to(tdt)
    return I


CASES = [
    # name, cells, level, parts, precision, recon, recon_ang, steps
    ("turb3d", (12, 6, 5), 2, (2, 1, 1), "f64", "plm", "dc", 2),
    ("turb3d", (9, 6, 8), 2, (3, 1, 2), "f32", "plm", "dc", 2),
    ("turb3d", (6, 6, 8), 2, (1, 2, 2), "f64", "ppm", "dc", 1),
    ("torus3d_big", (8, 8, 4), 2, (2, 2, 1), "f64", "plm", "dc", 2),
    ("torus3d_big", (8, 8, 4), 2, (2, 2, 1), "f32", "ppm", "mapr", 2),
    ("torus3d", (6, 9, 4), 2, (1, 3, 1), "f64", "dc", "mapr", 2),
    ("adjoint2d", (12, 8, 1), 2, (2, 2, 1), "f64", "plm", "dc", 2),
]


@pytest.mark.parametrize("name,n,level,parts,prec,recon,recon_ang,steps", CASES)
def test_blocks_equal_the_undivided_step(name, n, level, parts, prec, recon, recon_ang, steps):
    w = W.make(name, n=n, level=level)
    tdt = torch.float64 if prec == "f64" else torch.float32
    mode = {"thermal": rad.RAD_COUPLE_THERMAL, "emissivity": rad.RAD_COUPLE_EMISSIVITY}[w["mode"]]
    o = rad.rad_opts_default(precision=rad.RAD_F64 if prec == "f64" else rad.RAD_F32, recon=R[recon],
                             recon_ang=R[recon_ang], coupling=mode)
    # undivided
    ctx, na, nap = _ctx(w, w["xf"], w["bc"])
    dt = rad.rad_cfl_dt(ctx, w["cfl"])
    I = _initial(w, nap, tdt)
    g = _gas(w)
    src = torch.zeros(I.shape[:-1] + (4,), dtype=torch.float64, device="cuda")
    for _ in range(steps):
        rad.rad_step(ctx, I, g, dt, o, src)
    # blocks
    dec = B.Decomposition(w["n"], parts, w["bc"])
    blocks = []
    for r in range(dec.nblocks):
        b = dec.block(r)
        c, _, _ = _ctx(w, dec.faces(w["xf"], r), b["bc"])
        sl = dec.cells(r)
        dtb = rad.rad_cfl_dt(c, w["cfl"])
        send, recv = B.halo_buffers(tuple(b["size"][::-1]), b["neighbours"], nap, tdt, "cuda")
        blocks.append(dict(ctx=c, sl=sl, nb=b["neighbours"], I=_initial(w, nap, tdt)[sl].contiguous(),
                           gas=_gas(w, sl), src=torch.zeros(tuple(b["size"][::-1]) + (4,), dtype=torch.float64,
                                                             device="cuda"),
                           send=send, recv=recv, dt=dtb))
    assert min(b["dt"] for b in blocks) == dt            # the domain's bound is the blocks' minimum
    for _ in range(steps):
        for stage in (1, 2):
            for b in blocks:
                for (d, side), buf in b["send"].items():
                    rad.rad_halo_pack(b["ctx"], b["I"] if stage == 1 else None, o.precision, d, side, buf)
            for b in blocks:                               # the messages: face (d, side) -> neighbour's (d, 1 - side)
                for (d, side), peer in b["nb"].items():
                    blocks[peer]["recv"][(d, 1 - side)].copy_(b["send"][(d, side)])
            for b in blocks:
                rad.rad_step_stage(b["ctx"], stage, b["I"], b["gas"], dt, o, b["src"], b["recv"])
    torch.cuda.synchronize()
    rad.rad_check(ctx)
    for b in blocks:
        rad.rad_check(b["ctx"])
        assert torch.equal(b["I"], I[b["sl"]])
        assert torch.equal(b["gas"]["T"], g["T"][b["sl"]])
        assert torch.equal(b["src"], src[b["sl"]])
    # the domain's outgoing-flux loss: the parts of the blocks that hold the
    # outer x1 cells (their sum is what blocks.domain_loss all-reduces)
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    rad.rad_loss_outer(ctx, I, o.precision, L)
    parts_L = []
    for r, b in enumerate(blocks):
        if B.owns_outer_x1(dec, r):
            Lb = torch.zeros(1, dtype=torch.float64, device="cuda")
            rad.rad_loss_outer(b["ctx"], b["I"], o.precision, Lb)
            parts_L.append(float(Lb))
    assert abs(sum(parts_L) - float(L)) <= 1e-13 * abs(float(L))
    for b in blocks:
        rad.rad_destroy(b["ctx"])
    rad.rad_destroy(ctx)


def test_shared_faces_are_refused_where_unsupported():
    w = W.make("turb3d", n=(8, 6, 5), level=2)
    dec = B.Decomposition(w["n"], (2, 1, 1), w["bc"])
    b = dec.block(0)
    ctx, na, nap = _ctx(w, dec.faces(w["xf"], 0), b["bc"])
    try:
        I = torch.zeros(tuple(b["size"][::-1]) + (nap,), dtype=torch.float64, device="cuda")
        g = _gas(w, dec.cells(0))
        o = rad.rad_opts_default()
        with pytest.raises(rad.RadError) as e:
            rad.rad_step(ctx, I, g, 1e-3, o)
        assert e.value.status == rad.RAD_ESTATE
        with pytest.raises(rad.RadError) as e:            # halo buffers missing
            rad.rad_step_stage(ctx, 1, I, g, 1e-3, o, None, None)
        assert e.value.status == rad.RAD_EINVAL
        send, recv = B.halo_buffers(tuple(b["size"][::-1]), b["neighbours"], nap, torch.float64, "cuda")
        with pytest.raises(rad.RadError) as e:            # the weighting reads the neighbour's gas
            rad.rad_step_stage(ctx, 1, I, g, 1e-3, rad.rad_opts_default(tau_const=1.0), None, recv)
        assert e.value.status == rad.RAD_EUNSUPPORTED
        with pytest.raises(rad.RadError) as e:            # stage 2 before any stage 1
            rad.rad_step_stage(ctx, 2, I, g, 1e-3, o, None, recv)
        assert e.value.status == rad.RAD_ESTATE
        lam, lam_n = torch.zeros_like(I), torch.zeros_like(I)
        ga = torch.zeros(I.shape[:-1], dtype=torch.float64, device="cuda")
        with pytest.raises(rad.RadError) as e:
            rad.rad_step_adjoint(ctx, I, g, 1e-3, o, lam, lam_n, None, None, ga, ga.clone(), None)
        assert e.value.status == rad.RAD_EUNSUPPORTED
        rad.rad_check(ctx)
    finally:
        rad.rad_destroy(ctx)
    # a block on a polar axis that does not hold the whole phi range
    wk = W.make("torus3d", n=(6, 6, 8), level=1, with_intensity=False)
    c2 = rad.rad_create(torch.cuda.current_stream())
    try:
        rad.rad_init_angles(c2, 1)
        xf = [wk["xf"][0], wk["xf"][1], wk["xf"][2][:5]]
        with pytest.raises(rad.RadError) as e:
            rad.rad_set_metric(c2, wk["kind"], wk["spin"], 3, xf,
                               (("outflow", "outflow"), ("polar", "polar"), ("halo", "halo")))
        assert e.value.status in (rad.RAD_EUNSUPPORTED, rad.RAD_EINVAL)
    finally:
        rad.rad_destroy(c2)
