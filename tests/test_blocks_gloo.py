"""Block decomposition on CPU ranks (gloo, world size 2): two processes each
advance one block of the domain with the oracle, exchanging the ghost layers
of their shared faces before every stage through
paper_2302_04283_gb300.blocks.exchange (the same routine the GPU blocks use),
and their blocks must equal the undivided oracle run bit for bit; the
domain's time step (blocks.domain_dt, the minimum of the blocks' bounds)
must equal the undivided bound, and its outgoing-flux loss
(blocks.domain_loss over the blocks that own the outer x1 cells) the
undivided loss to rounding.  Covers a
periodic direction split in two (both faces of each block shared with the
same neighbour) and a Kerr-Schild grid split across theta (each block keeps
a polar axis and shares one face)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "turb3d_x1": dict(name="turb3d", n=(8, 6, 5), level=2, parts=(2, 1, 1), recon="plm"),
    "turb3d_x3_ppm": dict(name="turb3d", n=(5, 4, 8), level=2, parts=(1, 1, 2), recon="ppm"),
    "torus_theta": dict(name="torus3d_big", n=(6, 8, 4), level=2, parts=(1, 2, 1), recon="plm"),
}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, case, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import workloads as W
        from oracle import cfl as OCFL
        from oracle import step as OS
        from oracle import transport as TR
        from oracle.angles import GeodesicGrid
        from oracle.transport import Grid, Setup
        from paper_2302_04283_gb300 import blocks as B
        c = CASES[case]
        w = W.make(c["name"], n=c["n"], level=c["level"])
        ang = GeodesicGrid(w["level"])
        full = Setup(Grid(w["kind"], w["spin"], w["xf"], w["bc"], w["ndim"]), ang)
        dt = OCFL.cfl_dt(full, w["cfl"])
        opts = OS.Opts(recon=c["recon"])
        gas = {k: torch.tensor(w[k]) for k in ("rho", "u", "alpha_a", "alpha_s")}
        gas["eta"] = None
        # the undivided run
        If, Tf = torch.tensor(w["I0"]), torch.tensor(w["T"])
        for _ in range(2):
            If, Tf, srcf, ok = OS.rk2_step(If, Tf, gas, dt, full, opts)
        # this rank's block
        dec = B.Decomposition(w["n"], c["parts"], w["bc"])
        blk = dec.block(rank)
        cut = dec.cells(rank)
        st = Setup(Grid(w["kind"], w["spin"], dec.faces(w["xf"], rank), blk["bc"], w["ndim"]), ang)
        gb = {k: v[cut].contiguous() for k, v in gas.items() if v is not None}
        gb["eta"] = None
        I, T = torch.tensor(w["I0"])[cut].contiguous(), torch.tensor(w["T"])[cut].contiguous()
        nb = blk["neighbours"]

        def exch(Is):
            send = {f: TR.halo_pack(Is, st.grid, *f).contiguous() for f in nb}
            recv = {f: torch.empty_like(v) for f, v in send.items()}
            B.exchange(nb, send, recv)
            return recv

        for _ in range(2):
            I, T, src, ok = OS.rk2_step(I, T, gb, dt, st, opts, exchange=exch)
            assert bool(ok.all())
        same = (torch.equal(I, If[cut]), torch.equal(T, Tf[cut]), torch.equal(src, srcf[cut]))
        dif = float((I - If[cut]).abs().max() / If[cut].abs().max())
        # the domain's time step from the blocks' bounds, and its
        # outgoing-flux loss from the blocks' parts
        dt_dom = B.domain_dt(OCFL.cfl_dt(st, w["cfl"]))
        from oracle import adjoint as OA
        Lb = OA.loss_outer(I, st) if B.owns_outer_x1(dec, rank) else torch.zeros((), dtype=I.dtype)
        L = float(B.domain_loss(Lb.reshape(1).clone())[0])
        Lf = float(OA.loss_outer(If, full))
        q.put((rank, same, dif, len(nb), abs(dt_dom - dt) / dt, abs(L - Lf) / abs(Lf)))
    finally:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_split_domain_equals_undivided_oracle(case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, same, dif, nnb, ddt, dL in out:
        assert nnb >= 1
        assert all(same), (case, rank, same, dif)
        assert ddt == 0.0, ddt              # a minimum of the same per-cell bounds
        assert dL < 1e-13, dL               # the same terms summed in another order


def test_decomposition_faces_and_neighbours():
    from paper_2302_04283_gb300 import blocks as B
    per = (("periodic", "periodic"),) * 3
    dec = B.Decomposition((12, 6, 8), (3, 1, 2), per)
    assert dec.nblocks == 6 and dec.size == (4, 6, 4)
    b = dec.block(dec.rank_of((0, 0, 1)))
    assert b["offset"] == (0, 0, 4)
    assert b["bc"] == (("halo", "halo"), ("periodic", "periodic"), ("halo", "halo"))
    assert b["neighbours"] == {(0, 0): dec.rank_of((2, 0, 1)), (0, 1): dec.rank_of((1, 0, 1)),
                               (2, 0): dec.rank_of((0, 0, 0)), (2, 1): dec.rank_of((0, 0, 0))}
    ks = (("outflow", "outflow"), ("polar", "polar"), ("periodic", "periodic"))
    dec = B.Decomposition((8, 6, 4), (2, 2, 1), ks)
    b = dec.block(0)
    assert b["bc"] == (("outflow", "halo"), ("polar", "halo"), ("periodic", "periodic"))
    assert b["neighbours"] == {(0, 1): 1, (1, 1): 2}
    with pytest.raises(ValueError):
        B.Decomposition((8, 6, 4), (1, 1, 2), ks)        # a polar block must hold the whole phi range
    with pytest.raises(ValueError):
        B.Decomposition((8, 4, 4), (4, 1, 1), per)       # fewer than 3 cells across a shared face
