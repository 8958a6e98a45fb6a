"""Large snapshot counts (N_s = 17 and 31, the paper's two test cases,
Sec. 4.1): the tile kernel runs with the case's snapshot count at run time
and takes the HB source V omega D U (Sec. 1) from a separate launch.
Parity with the FP64 oracle on the residual and on RK trajectories, a batch
mixing small and large N_s, and the drivers that refuse large N_s."""
import numpy as np
import pytest
import torch

from oracle.hb_oracle import Oracle
from paper_1304_7654_gb300 import cases as C
from paper_1304_7654_gb300 import hb

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


CASES = {
    # 17 snapshots: multi-block viscous channel with a flipped block
    "channel_flip_viscous_nh8": lambda: C.channel(16, 8, n_harm=8, viscous=True, blocks=[
        C.BlockSpec((0, 0), (9, 8)), C.BlockSpec((9, 0), (16, 3), flip=True), C.BlockSpec((9, 3), (16, 8))]),
    # 31 snapshots: pitching inviscid O-grid in 4 blocks
    "ogrid_euler_nh15": lambda: C.ogrid(48, 12, n_harm=15, viscous=False, specs=[
        C.BlockSpec((0, 0), (20, 12)), C.BlockSpec((20, 0), (48, 5)), C.BlockSpec((20, 5), (48, 12))]),
    # 31 snapshots: laminar pitching O-grid (no-slip wall, farfield)
    "ns_ogrid8_nh15": lambda: C.ns_ogrid8(64, 16, n_harm=15),
}


def _setup(cs, prec):
    o = Oracle(cs)
    U = o.init_state(C.noise(cs), 0.01)
    ctx = hb.HBContext(cs, prec)
    Ug = ctx.from_compact(torch.as_tensor(o.unpack(U), device="cuda"))
    return o, U, ctx, Ug


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity_large_ns(name, prec):
    cs = CASES[name]()
    assert cs.n_snap in (17, 31)
    o, U, ctx, Ug = _setup(cs, prec)
    if prec == "fp32":
        U = o.pack(ctx.to_compact(Ug).double().cpu().numpy())
    Rref, sc = o.residual(U)
    R = ctx.to_compact(ctx.residual(Ug)).double().cpu().numpy()
    err = np.abs(R - o.unpack(Rref)) / o.unpack(sc)
    assert err.max() < TOL[prec], (name, prec, err.max())
    assert ctx.sync_status() == hb.HB_OK


@pytest.mark.parametrize("name", list(CASES))
def test_rk_trajectory_parity_large_ns(name):
    cs = CASES[name]()
    o, U, ctx, Ug = _setup(cs, "fp64")
    Uo, no = o.rk_smooth(U, 6)
    ng = ctx.rk_smooth(Ug, 6).cpu().numpy()
    assert ctx.sync_status() == hb.HB_OK
    Ugc = ctx.to_compact(Ug).cpu().numpy()
    assert np.abs(Ugc - o.unpack(Uo)).max() < 1e-12 * np.abs(o.unpack(Uo)).max()
    assert np.allclose(ng, no, rtol=1e-10, atol=0)


def test_forces_large_ns():
    cs = CASES["ns_ogrid8_nh15"]()
    o, U, ctx, Ug = _setup(cs, "fp64")
    U, _ = o.rk_smooth(U, 3)
    Ug = ctx.from_compact(torch.as_tensor(o.unpack(U), device="cuda"))
    cref, Jref = o.forces(U)
    coef, J = ctx.forces(Ug)
    coef = coef.cpu().numpy()
    scale = np.abs(cref).max()
    assert np.abs(coef - cref).max() < 1e-12 * scale, (np.abs(coef - cref).max(), scale)
    assert abs(J.item() - Jref) < 1e-12 * scale


def test_batch_mixing_small_and_large_ns_equals_cases_alone():
    cases = [C.ogrid(32, 8, n_harm=nh, viscous=False, seed=70 + nh) for nh in (1, 8, 3, 15)]
    bctx = hb.HBContext(cases, "fp32")
    assert bctx.tuning()[0] == 0                    # the persistent driver is not built for N_s > 9
    with pytest.raises(RuntimeError):
        bctx.set_tuning(1, 32, 8)
    Ub = bctx.new_state()
    bctx.init_state(Ub, torch.as_tensor(np.concatenate([C.noise(c) for c in cases]), device="cuda"), 0.01)
    nb = bctx.rk_smooth(Ub, 3).cpu().numpy()
    assert bctx.sync_status() == hb.HB_OK
    b0 = 0
    for k, c in enumerate(cases):
        ctx = hb.HBContext(c, "fp32")
        U = ctx.new_state()
        ctx.init_state(U, torch.as_tensor(C.noise(c), device="cuda"), 0.01)
        n1 = ctx.rk_smooth(U, 3).cpu().numpy()
        off0 = bctx.layouts[b0][0]
        b0 += len(c.blocks)
        end = bctx.layouts[b0][0] if b0 < len(bctx.layouts) else bctx.size
        assert torch.equal(ctx.to_compact(U), ctx.to_compact(Ub[off0:end].clone())), k
        assert np.allclose(n1, nb[:, k], rtol=1e-12, atol=0), k
