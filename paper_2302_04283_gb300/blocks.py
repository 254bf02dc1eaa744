"""Block decomposition of a grid and the ghost exchange between blocks.

The paper's code splits the domain into blocks and, before every stage's
fluxes, exchanges the cells next to the faces the blocks share (the task
list of Sec. 2); Sec. 5 runs one block per GPU.  Here a block is one library
context: its grid holds its own cells, with RAD_BC_HALO on every shared
face, and it steps one stage at a time (rad_step_stage), the halos coming
from its neighbours' rad_halo_pack.

`Decomposition` cuts a rectangular domain into parts[0] x parts[1] x
parts[2] blocks (rank r is block (p1, p2, p3) with r = (p3 P2 + p2) P1 + p1)
and gives each block's cells, face coordinates, boundary kinds and
neighbours.  `exchange` moves the halo buffers between ranks with
torch.distributed point-to-point messages (NCCL for device tensors, gloo for
host tensors); `step_block` is one RK2 step of a block through the C ABI;
`domain_dt` and `domain_loss` reduce the blocks' time-step bounds (minimum)
and outgoing-flux losses (sum) over the ranks.
Nothing here does arithmetic of the method."""
import torch
import torch.distributed as dist

LAYERS = 3          # ghost layers per shared face (the widest stencil, PPM, reaches three cells)


class Decomposition:
    """parts[d] blocks along dimension d of a domain of n[d] cells with
    boundary kinds bc[d] = (lo, hi) ('periodic' | 'outflow' | 'polar')."""

    def __init__(self, n, parts, bc):
        self.n, self.parts, self.bc = tuple(n), tuple(parts), tuple(tuple(b) for b in bc)
        for d in range(3):
            if parts[d] < 1 or n[d] % parts[d]:
                raise ValueError(f"{n[d]} cells do not split into {parts[d]} equal blocks")
            if parts[d] > 1 and n[d] // parts[d] < LAYERS:
                raise ValueError("a block needs at least 3 cells across a shared face")
        if parts[2] > 1 and "polar" in self.bc[1]:
            raise ValueError("a block on a polar axis must hold the whole phi range")
        self.size = tuple(n[d] // parts[d] for d in range(3))

    @property
    def nblocks(self):
        return self.parts[0] * self.parts[1] * self.parts[2]

    def coords(self, rank):
        P1, P2, _ = self.parts
        return (rank % P1, (rank // P1) % P2, rank // (P1 * P2))

    def rank_of(self, p):
        P1, P2, _ = self.parts
        return (p[2] * P2 + p[1]) * P1 + p[0]

    def block(self, rank):
        """offset (first cell per dimension), size, bc ((lo, hi) per dimension,
        'halo' on shared faces) and neighbours {(d, side): rank} of a block."""
        p = self.coords(rank)
        off = tuple(p[d] * self.size[d] for d in range(3))
        bc, nb = [], {}
        for d in range(3):
            sides = []
            for side in (0, 1):
                edge = p[d] == (0 if side == 0 else self.parts[d] - 1)
                kind = self.bc[d][side]
                if self.parts[d] > 1 and (not edge or kind == "periodic"):
                    q = list(p)
                    q[d] = (p[d] + (1 if side else -1)) % self.parts[d]
                    nb[(d, side)] = self.rank_of(q)
                    sides.append("halo")
                else:
                    sides.append(kind)
            bc.append(tuple(sides))
        return {"offset": off, "size": self.size, "bc": tuple(bc), "neighbours": nb}

    def faces(self, xf, rank):
        """The block's face coordinates, cut from the domain's xf[d]."""
        b = self.block(rank)
        return [xf[d][b["offset"][d]:b["offset"][d] + b["size"][d] + 1] for d in range(3)]

    def cells(self, rank):
        """Slices of the domain's [k][j][i] arrays that the block holds."""
        b = self.block(rank)
        o, s = b["offset"], b["size"]
        return (slice(o[2], o[2] + s[2]), slice(o[1], o[1] + s[1]), slice(o[0], o[0] + s[0]))


def exchange(neighbours, send, recv, group=None):
    """Send send[(d, side)] (this block's layers next to face (d, side)) to the
    neighbour across that face, which takes it as its halo of face
    (d, 1 - side); receive recv[(d, side)] likewise.  Messages are posted in
    one fixed order on every rank (for each d and receiving side: receive
    that halo, send the opposite face) and tagged by the receiving face, so
    that two messages between the same pair of ranks (a periodic direction
    split in two) cannot be confused."""
    ops = []
    for d in range(3):
        for side in (0, 1):
            if (d, side) in neighbours:
                ops.append(dist.P2POp(dist.irecv, recv[(d, side)], neighbours[(d, side)], group, 2 * d + side))
            face = (d, 1 - side)
            if face in neighbours:
                ops.append(dist.P2POp(dist.isend, send[face], neighbours[face], group, 2 * d + side))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def domain_dt(dt, group=None, device=None):
    """The whole domain's time step: the smallest of the blocks' CFL bounds
    (one all-reduce; every rank gets it)."""
    t = torch.tensor([float(dt)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())


def owns_outer_x1(dec, rank):
    """Whether the block holds the domain's last x1 cells, where the
    outgoing-flux loss is taken (rad_loss_outer on that block)."""
    return dec.coords(rank)[0] == dec.parts[0] - 1


def domain_loss(L, group=None):
    """The whole domain's outgoing-flux loss from each block's part (0 from a
    block that does not own the outer x1 face): an all-reduce sum, in place
    on the one-element tensor L, which is returned."""
    dist.all_reduce(L, op=dist.ReduceOp.SUM, group=group)
    return L


def halo_buffers(ctx_shape, neighbours, nap, dtype, device):
    """Send and receive buffers of the shared faces of a block of
    ctx_shape = (n3, n2, n1) cells (rad_halo_pack layout)."""
    n3, n2, n1 = ctx_shape
    shape = {0: (LAYERS, n3, n2, nap), 1: (LAYERS, n3, n1, nap), 2: (LAYERS, n2, n1, nap)}
    send = {f: torch.empty(shape[f[0]], dtype=dtype, device=device) for f in neighbours}
    recv = {f: torch.empty(shape[f[0]], dtype=dtype, device=device) for f in neighbours}
    return send, recv


def step_block(rad, ctx, I, gas, dt, opts, gas_src, neighbours, send, recv, move=None):
    """One RK2 step of a block: before each stage, pack the shared faces of
    the stage's input, exchange them (move(send, recv), by default
    `exchange` over torch.distributed) and run the stage on the received
    halos."""
    move = move or (lambda s, r: exchange(neighbours, s, r))
    for stage in (1, 2):
        for (d, side), buf in send.items():
            rad.rad_halo_pack(ctx, I if stage == 1 else None, opts.precision, d, side, buf)
        move(send, recv)
        rad.rad_step_stage(ctx, stage, I, gas, dt, opts, gas_src, recv)
