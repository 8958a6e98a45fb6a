"""Block decomposition on the GPU (the paper's distribution of blocks over
ranks with one cut exchange per RK step, Sec. 2-3): the shares of a
decomposed case, each a library context with external boxes, advanced by
hb_halo_pass / hb_pack_halo / hb_unpack_halo / hb_rk_stage with the halo
hand-over between them (all shares on this one GPU, driven by one process),
against the undivided case advanced by hb_rk_smooth with the same halo
passes: the state bit for bit, norms and forces to FP64 rounding."""
import numpy as np
import pytest
import torch

from oracle.hb_oracle import Oracle
from paper_1304_7654_gb300 import cases as C
from paper_1304_7654_gb300 import decomp as D
from paper_1304_7654_gb300 import hb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _block_slices(cs):
    out, o = [], 0
    for b in cs.blocks:
        m = b.n[0] * b.n[1] * b.n[2] * cs.n_snap * cs.nv
        out.append((o, o + m))
        o += m
    return out


def _shares(cs, prec, flat, world):
    sl = _block_slices(cs)
    parts = D.partition(cs, world)
    solvers, states = [], []
    for r in range(world):
        sh = D.make_share(cs, parts, r)
        be = D.LibBackend(sh.case, prec)
        mine = np.concatenate([flat[sl[b][0]:sl[b][1]] for b in sh.blocks])
        states.append(be.ctx.from_compact(torch.as_tensor(mine, device="cuda")))
        solvers.append(D.DecomposedHB(sh, be, None))
    return solvers, states


def _gather(cs, solvers, states):
    """The compact interior state of the whole case from the shares."""
    sl = _block_slices(cs)
    out = np.zeros(sl[-1][1])
    for s, U in zip(solvers, states):
        got = s.be.ctx.to_compact(U).double().cpu().numpy()
        o = 0
        for b in s.share.blocks:
            m = sl[b][1] - sl[b][0]
            out[sl[b][0]:sl[b][1]] = got[o:o + m]
            o += m
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("world", [2, 3])
def test_shares_on_one_gpu_equal_the_undivided_case(prec, world):
    """2 or 3 shares against the undivided case driven by the same calls
    (one share holding every block): bit for bit."""
    cs = C.ns_ogrid8(128, 24, n_harm=3)
    o = Oracle(cs)
    flat = o.unpack(o.init_state(C.noise(cs), 0.01))
    n_iter = 4
    s1, u1 = _shares(cs, prec, flat, 1)
    n_ref = D.run_local(s1, u1, n_iter)
    c_ref, J_ref = D.forces_local(s1, u1)
    sw, uw = _shares(cs, prec, flat, world)
    norms = D.run_local(sw, uw, n_iter)
    coef, J = D.forces_local(sw, uw)
    for s in s1 + sw:
        assert s.be.ctx.sync_status() == hb.HB_OK
    ref, got = _gather(cs, s1, u1), _gather(cs, sw, uw)
    assert np.array_equal(got, ref), (prec, world, np.abs(got - ref).max())
    assert np.allclose(norms, n_ref, rtol=1e-12, atol=0)
    assert np.allclose(coef, c_ref, rtol=0, atol=1e-13 * np.abs(c_ref).max())
    assert abs(J - J_ref) <= 1e-13 * max(1.0, abs(J_ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stage_by_stage_driver_equals_rk_smooth(prec):
    """The stage-by-stage calls (hb_halo_pass, hb_rk_stage) reproduce
    hb_rk_smooth on the undivided case, and the FP64 result the oracle's."""
    cs = C.ns_ogrid8(128, 24, n_harm=3)
    o = Oracle(cs)
    U0 = o.init_state(C.noise(cs), 0.01)
    flat = o.unpack(U0)
    s1, u1 = _shares(cs, prec, flat, 1)
    norms = D.run_local(s1, u1, 3)
    full = hb.HBContext(cs, prec)
    full.set_tuning(2, 32, 8)
    Uf = full.from_compact(torch.as_tensor(flat, device="cuda"))
    n_full = full.rk_smooth(Uf, 3).cpu().numpy()
    got = _gather(cs, s1, u1)
    want = full.to_compact(Uf).double().cpu().numpy()
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    assert np.allclose(norms, n_full, rtol=1e-12 if prec == "fp64" else 1e-5, atol=0)
    if prec == "fp64":
        Uo, no = o.rk_smooth(U0, 3)
        assert np.abs(got - o.unpack(Uo)).max() < 1e-12 * np.abs(o.unpack(Uo)).max()
        assert np.allclose(norms, no, rtol=1e-10, atol=0)


def test_share_contexts_refuse_the_whole_iteration_and_pack_round_trips():
    cs = C.ns_ogrid8(64, 24, n_harm=1)
    parts = D.partition(cs, 2)
    sh = D.make_share(cs, parts, 0)
    be = D.LibBackend(sh.case, "fp64")
    U = be.new_state()
    with pytest.raises(hb.HBError) as e:
        be.ctx.rk_smooth(U, 1)
    assert e.value.status == hb.HB_ERR_UNSUPPORTED
    torch.manual_seed(0)
    U.copy_(torch.randn_like(U))
    idx = torch.randperm(U.numel(), device="cuda")[:1000]
    buf = be.pack(U, idx)
    assert torch.equal(buf, U[idx])
    V = torch.zeros_like(U)
    be.unpack(V, idx, buf)
    assert torch.equal(V[idx], U[idx])
