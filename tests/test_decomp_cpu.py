"""Block decomposition over processes (the paper's distribution of blocks over
MPI ranks with one cut exchange per RK step, Sec. 2-3), host side: the
longest-processing-time partition, the exchange tables of each share, and a
decomposed run on two gloo ranks on the CPU -- each rank advancing its share
with the FP64 oracle as the per-rank backend -- against the undivided case:
the state bit for bit, the norms and force coefficients to FP64 rounding."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1304_7654_gb300 import cases as C
from paper_1304_7654_gb300 import decomp as D


def _fake_case(costs):
    blocks = [C.Block(n=(c, 1, 1), nodes=None) for c in costs]
    return C.Case(name="fake", dim=2, n_harm=0, mach=0.5, omega=0.0, blocks=blocks)


def test_partition_is_longest_processing_time_first():
    # costs of blocks 0..4 = 3, 5, 3, 4, 3 on two ranks, largest first (equal
    # costs by block index): block 1 (5) -> r0, block 3 (4) -> r1, block 0
    # (3) -> r1 (7), block 2 (3) -> r0 (8), block 4 (3) -> r1 (10)
    parts = D.partition(_fake_case([3, 5, 3, 4, 3]), 2)
    assert parts == [[1, 2], [0, 3, 4]]
    # every block once; the largest load within one block of the mean
    cs = C.ns_ogrid8()
    cost = [b.n[0] * b.n[1] * cs.n_snap for b in cs.blocks]
    for w in (2, 3, 4, 8):
        parts = D.partition(cs, w)
        assert sorted(b for p in parts for b in p) == list(range(len(cs.blocks)))
        loads = [sum(cost[b] for b in p) for p in parts]
        assert max(loads) <= sum(cost) / w + max(cost)
        assert parts == D.partition(cs, w)


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_tables_match_between_ranks(world):
    cs = C.ns_ogrid8(64, 24, n_harm=1)
    parts = D.partition(cs, world)
    shares = [D.make_share(cs, parts, r) for r in range(world)]
    owner = {b: r for r, p in enumerate(parts) for b in p}
    for r, sh in enumerate(shares):
        for p in range(cs.dim):
            for q, cells in sh.recvs[p].items():
                assert q != r
                assert len(cells) == len(shares[q].sends[p][r])
    # the external boxes of each share are exactly the ghost cells whose cut
    # source block lives on another rank
    for r, sh in enumerate(shares):
        ext = sum(int(np.prod(np.maximum(row[5:7] - row[2:4], 0))) for row in sh.case.cuts if row[1] == -1)
        remote = sum(int(np.prod(np.maximum(row[5:7] - row[2:4], 0))) for row in cs.cuts
                     if owner[int(row[0])] == r and owner[int(row[1])] != r)
        assert ext == remote
        assert ext == sum(len(c) for p in range(cs.dim) for c in sh.recvs[p].values())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    return C.ns_ogrid8(64, 24, n_harm=2, viscous=True)


def _rank(rank, world, port, n_iter, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from oracle.hb_oracle import Oracle
    from decomp_oracle_backend import OracleBackend
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cs = _case()
    parts = D.partition(cs, world)
    sh = D.make_share(cs, parts, rank)
    full = Oracle(cs)
    U0 = full.init_state(C.noise(cs), 0.01)
    be = OracleBackend(sh.case)
    U = be.new_state()
    for q, b in enumerate(sh.blocks):
        be.o.interior(U, q)[...] = full.interior(U0, b)
    solver = D.DecomposedHB(sh, be, D.TorchTransport())
    norms = solver.rk_smooth(U, n_iter)
    coef, J = solver.forces(U)
    out.put((rank, sh.blocks, [be.o.interior(U, q).copy() for q in range(len(sh.blocks))], norms,
             coef.numpy(), float(J[0])))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_undivided_case(world):
    import sys
    from oracle.hb_oracle import Oracle
    n_iter = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    here = os.path.dirname(os.path.abspath(__file__))
    if here not in sys.path:
        sys.path.insert(0, here)
    os.environ["PYTHONPATH"] = os.pathsep.join([here, os.path.dirname(here), os.environ.get("PYTHONPATH", "")])
    procs = [ctx.Process(target=_rank, args=(r, world, port, n_iter, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cs = _case()
    o = Oracle(cs)
    U = o.init_state(C.noise(cs), 0.01)
    Uref, nref = o.rk_smooth(U, n_iter)
    cref, Jref = o.forces(Uref)
    for rank, blocks, states, norms, coef, J in res:
        for b, got in zip(blocks, states):
            assert np.array_equal(got, o.interior(Uref, b)), (rank, b)
        assert np.allclose(norms, nref, rtol=1e-13, atol=0), (norms, nref)
        assert np.allclose(coef, cref, rtol=0, atol=1e-14 * np.abs(cref).max())
        assert abs(J - Jref) <= 1e-14 * max(1.0, abs(Jref))


def test_one_process_holding_every_share_equals_the_undivided_case():
    """The in-process driver (run_local: every share advanced by one process,
    buffers handed over directly) on three shares."""
    import sys
    from oracle.hb_oracle import Oracle
    here = os.path.dirname(os.path.abspath(__file__))
    if here not in sys.path:
        sys.path.insert(0, here)
    from decomp_oracle_backend import OracleBackend
    cs = _case()
    o = Oracle(cs)
    U0 = o.init_state(C.noise(cs), 0.01)
    parts = D.partition(cs, 3)
    shares = [D.make_share(cs, parts, r) for r in range(3)]
    solvers, states = [], []
    for sh in shares:
        be = OracleBackend(sh.case)
        U = be.new_state()
        for q, b in enumerate(sh.blocks):
            be.o.interior(U, q)[...] = o.interior(U0, b)
        solvers.append(D.DecomposedHB(sh, be, None))
        states.append(U)
    norms = D.run_local(solvers, states, 2)
    coef, J = D.forces_local(solvers, states)
    Uref, nref = o.rk_smooth(U0, 2)
    cref, Jref = o.forces(Uref)
    for sh, s, U in zip(shares, solvers, states):
        for q, b in enumerate(sh.blocks):
            assert np.array_equal(s.be.o.interior(U, q), o.interior(Uref, b))
    assert np.allclose(norms, nref, rtol=1e-13, atol=0)
    assert np.allclose(coef, cref, rtol=0, atol=1e-14 * np.abs(cref).max())
    assert abs(J - Jref) <= 1e-14 * max(1.0, abs(Jref))
