"""Time-domain dual time stepping on the HB kernels (hb_td_step): parity
with the FP64 oracle's BDF2 dual-time iterations and forces at a physical
time; and the independent check of the HB method itself -- the periodic
limit of the time-domain run reproduces the converged HB solution at the
snapshot times (Sec. 1: the HB solver stands in for the time-domain one
for periodic flows)."""
import math

import numpy as np
import pytest
import torch

from oracle.hb_oracle import Oracle
from paper_1304_7654_gb300 import cases as C
from paper_1304_7654_gb300 import hb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _td_case():
    # laminar pitching O-grid in two blocks, one snapshot
    return C.ogrid(24, 8, n_harm=0, viscous=True, pitch_deg=3.0,
                   specs=[C.BlockSpec((0, 0), (10, 8)), C.BlockSpec((10, 0), (24, 8))])


def _states(cs, o, ctx):
    Un = o.init_state(C.noise(cs, 3), 0.01)
    Unm1 = o.init_state(C.noise(cs, 4), 0.01)
    g = lambda A: ctx.from_compact(torch.as_tensor(o.unpack(A), device="cuda"))
    return Un, Unm1, g(Un), g(Unm1)


@pytest.mark.parametrize("bdf2", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_td_step_matches_oracle(prec, bdf2):
    cs = _td_case()
    o = Oracle(cs)
    ctx = hb.HBContext(cs, prec)
    Un, Unm1, gUn, gUnm1 = _states(cs, o, ctx)
    if prec == "fp32":   # the oracle starts from the FP32-rounded states
        Un = o.pack(ctx.to_compact(gUn).double().cpu().numpy())
        Unm1 = o.pack(ctx.to_compact(gUnm1).double().cpu().numpy())
    t, dt = 5.3, 0.7
    Uo, no = o.td_step(Un, Un, Unm1 if bdf2 else None, t, dt, 4)
    U = gUn.clone()
    ng = ctx.td_step(U, gUn, gUnm1 if bdf2 else None, t, dt, 4).cpu().numpy()
    assert ctx.sync_status() == hb.HB_OK
    got = ctx.to_compact(U).double().cpu().numpy()
    ref = o.unpack(Uo)
    tol = 1e-12 if prec == "fp64" else 5e-6
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), np.abs(got - ref).max()
    assert np.allclose(ng, no, rtol=1e-10 if prec == "fp64" else 2e-3, atol=0)
    # the context keeps the frame of time t: forces of the new state at t
    cref, Jref = o.td_forces(Uo if prec == "fp64" else o.pack(got), t)
    coef, J = ctx.forces(U)
    scale = np.abs(cref).max()
    assert np.abs(coef.cpu().numpy() - cref).max() <= (1e-12 if prec == "fp64" else 2e-5) * scale


def test_td_refuses_hb_and_3d_contexts():
    for cs in (C.ogrid(24, 8, n_harm=1), C.box3d(8, 8, 4, n_harm=0)):
        ctx = hb.HBContext(cs, "fp64")
        U = ctx.new_state()
        with pytest.raises(hb.HBError) as e:
            ctx.td_step(U, U, None, 1.0, 0.1, 2)
        assert e.value.status == hb.HB_ERR_UNSUPPORTED


def test_periodic_limit_of_time_domain_run_equals_hb_solution():
    """Inviscid pitching O-grid (48x12, M 0.3, 3 deg, k 0.1): lift from the
    converged HB solution (N_H = 1 and 3) against the periodic limit of a
    BDF2 dual-time run, 84 steps per period (divisible by 3 and 7, so the
    snapshot times are steps), 6 periods from freestream, 120 inner
    iterations.  Measured: 0.4% (N_H = 1) and 0.9% (N_H = 3) of the lift
    amplitude; the run is periodic to 4e-9."""
    make = lambda nh: C.ogrid(48, 12, n_harm=nh, viscous=False, pitch_deg=3.0)
    zero = lambda cs: torch.as_tensor(np.zeros(C.interior_count(cs)), device="cuda")
    cs = make(0)
    T = 2 * math.pi / cs.omega
    steps, periods = 84, 6
    dt = T / steps
    ctx = hb.HBContext(cs, "fp64")
    Un = ctx.new_state()
    ctx.init_state(Un, zero(cs), 0.0)
    Unm1, cl = None, []
    for k in range(1, periods * steps + 1):
        U = Un.clone()
        ctx.td_step(U, Un, Unm1, k * dt, dt, 120, norms=False)
        Unm1, Un = Un, U
        cl.append(float(ctx.forces(Un)[0][0, 0, 0]))
    assert ctx.sync_status() == hb.HB_OK
    cl = np.array(cl)
    last = cl[-steps:]
    assert np.abs(last - cl[-2 * steps:-steps]).max() < 1e-6
    amp = np.abs(last - last.mean()).max()
    for nh in (1, 3):
        hcs = make(nh)
        hctx = hb.HBContext(hcs, "fp64")
        Uh = hctx.new_state()
        hctx.init_state(Uh, zero(hcs), 0.0)
        hctx.rk_smooth(Uh, 6000, norms=False)
        hb_cl = hctx.forces(Uh)[0][:, 0, 0].cpu().numpy()
        ns = hcs.n_snap
        # snapshot m at t = (periods - 1) T + m T / ns, i.e. step index (periods - 1) steps + m steps / ns
        td_cl = np.array([cl[(periods - 1) * steps + m * steps // ns - 1] for m in range(ns)])
        assert np.abs(td_cl - hb_cl).max() <= 0.02 * amp, (nh, td_cl, hb_cl, amp)
