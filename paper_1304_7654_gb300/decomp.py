"""Block decomposition of one multi-block HB case over several processes.

The paper distributes the blocks of a case over MPI ranks and exchanges the
cut (block-interface) halos once per Runge-Kutta step, aggregated per pair of
ranks, with one collective of the force coefficients per step (Sec. 2-3).
Here each process (one GPU) owns a share of the blocks:

* ``partition``: longest-processing-time assignment of the blocks by their
  cost, cells x snapshots (largest block first, to the least loaded rank).
* ``make_share``: the share as a case of its own -- its blocks, the cuts
  between them, its boundary segments -- in which every cut whose source
  block lives on another rank becomes an external box (source block -1,
  ``hb.h``'s ``HB_EXTERNAL_BLOCK``), plus, per pass (direction) and peer, the
  cells this rank sends and the ghost cells it receives, enumerated over the
  cut table in the same order on both sides.
* ``DecomposedHB``: advances the share stage by stage.  Before each RK stage
  the halos of the stage input are filled pass by pass: pack the sources
  other ranks need, exchange, fill the own cuts and boundary ghosts of the
  pass, unpack the received boxes -- so block corners get exactly the values
  of the undivided case.  The stage-1 residual sums of every rank are added
  before the RMS norms are formed, and the force coefficients (sums over wall
  faces) are added over the ranks.

The arithmetic runs in the backend: the library's CUDA kernels (``LibBackend``:
hb_halo_pass, hb_rk_stage, hb_pack_halo / hb_unpack_halo, hb_forces) or, in
the tests, the oracle.  The transport moves the packed buffers:
torch.distributed point-to-point sends (NCCL between GPUs, gloo on the host)
or, for several shares driven by one process, a direct hand-over.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np

from . import cases as C


def partition(case: C.Case, world_size: int) -> list:
    """Blocks of each rank: longest processing time first, cost = cells x
    snapshots, ties to the lowest rank; each rank's list ascending."""
    cost = [b.n[0] * b.n[1] * b.n[2] * case.n_snap for b in case.blocks]
    load = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for b in sorted(range(len(cost)), key=lambda q: (-cost[q], q)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        parts[r].append(b)
        load[r] += cost[b]
    return [sorted(p) for p in parts]


def cut_pass(row, case: C.Case) -> int:
    """The pass of a cut row: the highest direction along which its box
    leaves the destination block (lower ones are corner extensions)."""
    n = case.blocks[int(row[0])].n
    p = -1
    for a in range(case.dim):
        if row[2 + a] < 0 or row[5 + a] > n[a]:
            p = a
    return p


def cut_cells(row, dim: int):
    """Destination and source cells [m, 3] of a cut row, destination box
    enumerated k, then j, then i (i fastest)."""
    lo, hi = np.array(row[2:5]), np.array(row[5:8])
    off, perm, sign = np.array(row[8:11]), np.array(row[11:14]), np.array(row[14:17])
    if dim == 2:
        lo[2], hi[2] = 0, 1
    k, j, i = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]),
                          indexing="ij")
    dst = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    src = off[None, :] + sign[None, :] * dst[:, perm]
    if dim == 2:
        src[:, 2] = 0
    return dst, src


@dataclass
class Share:
    """One rank's share of a decomposed case."""
    rank: int
    world_size: int
    blocks: list          # global block ids, ascending; local id = position
    case: C.Case          # the share as a case (external boxes have source block -1)
    sends: list           # [pass] {peer: int array [m, 4] (local block, i, j, k) of source cells}
    recvs: list           # [pass] {peer: int array [m, 4] of destination ghost cells}
    total_cells: int      # cells of the whole case (the norms' denominator)


def make_share(case: C.Case, parts: list, rank: int) -> Share:
    owner = {b: r for r, p in enumerate(parts) for b in p}
    mine = parts[rank]
    local = {b: q for q, b in enumerate(mine)}
    dim = case.dim
    cuts = []
    sends = [dict() for _ in range(dim)]
    recvs = [dict() for _ in range(dim)]
    for row in np.asarray(case.cuts).reshape(-1, C.CUT_FIELDS):
        dst, src = int(row[0]), int(row[1])
        od, osrc = owner[dst], owner[src]
        if od != rank and osrc != rank:
            continue
        p = cut_pass(row, case)
        if od == rank and osrc == rank:
            r = row.copy()
            r[0], r[1] = local[dst], local[src]
            cuts.append(r)
            continue
        dcells, scells = cut_cells(row, dim)
        if od == rank:                      # an external box of this share
            r = row.copy()
            r[0], r[1] = local[dst], -1
            cuts.append(r)
            recvs[p].setdefault(osrc, []).append(
                np.concatenate([np.full((len(dcells), 1), local[dst]), dcells], axis=1))
        else:                               # this rank's cells in a peer's box
            sends[p].setdefault(od, []).append(
                np.concatenate([np.full((len(scells), 1), local[src]), scells], axis=1))
    bcs = []
    for row in np.asarray(case.bcs).reshape(-1, C.BC_FIELDS):
        if owner[int(row[0])] == rank:
            r = row.copy()
            r[0] = local[int(row[0])]
            bcs.append(r)
    sub = dataclasses.replace(
        case, name=f"{case.name}_share{rank}of{len(parts)}", blocks=[case.blocks[b] for b in mine],
        cuts=np.array(cuts, dtype=np.int32).reshape(-1, C.CUT_FIELDS),
        bcs=np.array(bcs, dtype=np.int32).reshape(-1, C.BC_FIELDS))
    cat = lambda d: {q: np.concatenate(v).astype(np.int64) for q, v in sorted(d.items())}
    return Share(rank=rank, world_size=len(parts), blocks=list(mine), case=sub,
                 sends=[cat(d) for d in sends], recvs=[cat(d) for d in recvs], total_cells=case.n_cells)


def state_offsets(cells, layout, n_snap: int, nv: int, dim: int) -> np.ndarray:
    """State offsets of every (cell, snapshot, variable) of cells [m, 4]
    (local block, i, j, k), cell-major: layout(b) -> (offset, strides) with
    strides over (n, v, k, j, i) and two ghost layers (k only in 3D)."""
    if len(cells) == 0:
        return np.zeros(0, dtype=np.int64)
    gk = 2 if dim == 3 else 0
    out = np.empty((len(cells), n_snap, nv), dtype=np.int64)
    n = np.arange(n_snap)[:, None]
    v = np.arange(nv)[None, :]
    for b in np.unique(cells[:, 0]):
        m = cells[:, 0] == b
        off, st = layout(int(b))
        c = cells[m]
        base = off + (c[:, 3] + gk) * st[2] + (c[:, 2] + 2) * st[3] + (c[:, 1] + 2) * st[4]
        out[m] = base[:, None, None] + (n * st[0] + v * st[1])[None]
    return out.reshape(-1)


class DecomposedHB:
    """One rank's share, advanced with the halo exchange between stages.

    backend: halo_pass(U, p), stage(Uin, U0, Uout, s, sums) (sums: per
    variable, or None), pack(U, idx) -> buffer, unpack(U, idx, buf),
    new_state(), layout(b), index(np_array) -> backend index,
    sums_buffer() -> per-variable accumulator, forces(U) -> (coef, J).
    transport: exchange(pass, {peer: buffer}, {peer: n}) -> {peer: buffer},
    allreduce(x) -> sum over ranks."""

    def __init__(self, share: Share, backend, transport):
        self.share = share
        self.be = backend
        self.tr = transport
        cs = share.case
        lay = backend.layout
        self.send_idx = [{q: backend.index(state_offsets(c, lay, cs.n_snap, cs.nv, cs.dim)) for q, c in d.items()}
                         for d in share.sends]
        self.recv_idx = [{q: backend.index(state_offsets(c, lay, cs.n_snap, cs.nv, cs.dim)) for q, c in d.items()}
                         for d in share.recvs]
        self.recv_n = [{q: len(c) * cs.n_snap * cs.nv for q, c in d.items()} for d in share.recvs]

    # the steps of one pass, usable by a driver that interleaves several shares
    def pack(self, U, p):
        return {q: self.be.pack(U, idx) for q, idx in self.send_idx[p].items()}

    def unpack(self, U, p, received):
        for q, idx in self.recv_idx[p].items():
            self.be.unpack(U, idx, received[q])

    def exchange(self, U):
        """Every ghost of U filled: per pass, pack, exchange, own cuts and
        boundary ghosts, unpack."""
        for p in range(self.share.case.dim):
            got = self.tr.exchange(p, self.pack(U, p), self.recv_n[p])
            self.be.halo_pass(U, p)
            self.unpack(U, p, got)
        return U

    def rk_smooth(self, U, n_iter: int):
        """n_iter RK iterations of the share in place; returns the norms
        [n_iter][nv] of the whole case (every rank's residual sums added
        before the square root)."""
        cs = self.share.case
        A, B = self.be.new_state(), self.be.new_state()
        norms = np.zeros((n_iter, cs.nv))
        denom = float(self.share.total_cells * cs.n_snap)
        for it in range(n_iter):
            ins, outs = (U, A, B, A), (A, B, A, U)
            for s in range(4):
                self.exchange(ins[s])
                sums = self.be.sums_buffer() if s == 0 else None
                self.be.stage(ins[s], U, outs[s], s, sums)
                if s == 0:
                    norms[it] = np.sqrt(_host(self.tr.allreduce(sums)) / denom)
        return norms

    def forces(self, U):
        """Force coefficients [N_s][bodies][3] and J of the whole case."""
        self.exchange(U)
        coef, J = self.be.forces(U)
        return self.tr.allreduce(coef), self.tr.allreduce(J)


class LibBackend:
    """The library's kernels on this process's GPU (torch tensors)."""

    def __init__(self, case: C.Case, prec: str = "fp64", device="cuda"):
        from . import hb
        self.ctx = hb.HBContext(case, prec)
        self.device = device
        self.case = case

    def layout(self, b):
        off, st, _ = self.ctx.layouts[b]
        return off, st

    def index(self, a):
        import torch
        return torch.as_tensor(a, dtype=torch.int64, device=self.device)

    def new_state(self):
        return self.ctx.new_state(self.device)

    def halo_pass(self, U, p):
        self.ctx.halo_pass(U, p)

    def stage(self, Uin, U0, Uout, s, sums):
        self.ctx.rk_stage(Uin, U0, Uout, s, sums)

    def sums_buffer(self):
        import torch
        return torch.zeros(self.case.nv, dtype=torch.float64, device=self.device)

    def pack(self, U, idx):
        import torch
        return self.ctx.pack_halo(U, idx, torch.empty(idx.numel(), dtype=self.ctx.dtype, device=self.device))

    def unpack(self, U, idx, buf):
        self.ctx.unpack_halo(U, idx, buf)

    def forces(self, U):
        return self.ctx.forces(U)


class TorchTransport:
    """Point-to-point exchange of the packed buffers and sums over the ranks
    through torch.distributed (NCCL between GPUs, gloo on the host).  Buffers
    are torch tensors on the process group's device."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, p, sends, recv_n):
        import torch
        import torch.distributed as dist
        ops, got = [], {}
        like = next(iter(sends.values()), None)
        for q, buf in sorted(sends.items()):
            ops.append(dist.P2POp(dist.isend, buf.contiguous(), q, group=self.group, tag=p))
        for q, n in sorted(recv_n.items()):
            ref = like if like is not None else torch.empty(0, dtype=torch.float64)
            got[q] = torch.empty(n, dtype=ref.dtype, device=ref.device)
            ops.append(dist.P2POp(dist.irecv, got[q], q, group=self.group, tag=p))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        return got

    def allreduce(self, x):
        import torch.distributed as dist
        y = x.clone()
        dist.all_reduce(y, op=dist.ReduceOp.SUM, group=self.group)
        return y


def _host(x) -> np.ndarray:
    """A per-variable sum (torch tensor on any device, or array) on the host."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64)


def fill_local(solvers: list, states: list):
    """Fill every ghost of the states of all shares held by this process, pass
    by pass: pack, own cuts and boundary ghosts, hand-over and unpack."""
    dim = solvers[0].share.case.dim
    for p in range(dim):
        packed = [s.pack(U, p) for s, U in zip(solvers, states)]
        for s, U in zip(solvers, states):
            s.be.halo_pass(U, p)
        for r, (s, U) in enumerate(zip(solvers, states)):
            s.unpack(U, p, {q: packed[q][r] for q in s.recv_idx[p]})


def run_local(solvers: list, states: list, n_iter: int):
    """Advance every share of a decomposition held by this process (for
    example all shares on one GPU): n_iter RK iterations; returns the norms
    [n_iter][nv] of the whole case.  The same steps as DecomposedHB.rk_smooth,
    with each packed buffer handed to its destination share and the sums
    added here in rank order."""
    cs = solvers[0].share.case
    denom = float(solvers[0].share.total_cells * cs.n_snap)
    bufs = [(s.be.new_state(), s.be.new_state()) for s in solvers]
    norms = np.zeros((n_iter, cs.nv))
    for it in range(n_iter):
        for st in range(4):
            ins = [(U, A, B, A)[st] for U, (A, B) in zip(states, bufs)]
            outs = [(A, B, A, U)[st] for U, (A, B) in zip(states, bufs)]
            fill_local(solvers, ins)
            tot = None
            for s, Uin, Uout, U in zip(solvers, ins, outs, states):
                sums = s.be.sums_buffer() if st == 0 else None
                s.be.stage(Uin, U, Uout, st, sums)
                if st == 0:
                    x = _host(sums)
                    tot = x if tot is None else tot + x
            if st == 0:
                norms[it] = np.sqrt(tot / denom)
    return norms


def forces_local(solvers: list, states: list):
    """Force coefficients [N_s][bodies][3] and J of the whole case from all
    shares held by this process (sums over the shares in rank order)."""
    fill_local(solvers, states)
    coef, J = None, 0.0
    for s, U in zip(solvers, states):
        c, j = s.be.forces(U)
        c = _host(c)
        coef = c if coef is None else coef + c
        J += float(_host(j).reshape(-1)[0])
    return coef, J
