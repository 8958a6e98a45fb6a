"""Restart files (hb_save_state / hb_load_state, the paper's restart file of
Sec. 3.1): a run saved after n iterations and resumed in a fresh context
equals the uninterrupted run bit for bit and the FP64 oracle's n + m
iterations; the file's payload is the oracle's state after n iterations;
files of another context, precision or format, and truncated files, are
refused."""
import os

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


def _start(cs, prec):
    ctx = hb.HBContext(cs, prec)
    U = ctx.new_state()
    if isinstance(cs, list):
        z = np.concatenate([C.noise(c) for c in cs])
    else:
        z = C.noise(cs)
    ctx.init_state(U, torch.as_tensor(z, device="cuda"), 0.01)
    return ctx, U


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("make", [lambda: C.ns_ogrid8(128, 24, n_harm=2),
                                  lambda: C.ogrid(48, 12, n_harm=15, viscous=False),
                                  lambda: C.batch_cases(n_cases=3, seed=5, scale=(1.0, 3.0))])
def test_resume_is_bitwise(make, prec, tmp_path):
    cs = make()
    path = str(tmp_path / "state.hbr")
    ctx, U = _start(cs, prec)
    ctx.rk_smooth(U, 4)
    ctx.save_state(U, path, iteration=4)
    n_ref = ctx.rk_smooth(U, 3)
    assert ctx.sync_status() == hb.HB_OK
    ctx2 = hb.HBContext(cs, prec)
    V = ctx2.new_state()
    assert ctx2.load_state(V, path) == 4
    n_res = ctx2.rk_smooth(V, 3)
    assert ctx2.sync_status() == hb.HB_OK
    assert torch.equal(ctx.to_compact(U), ctx2.to_compact(V))
    assert torch.equal(n_ref, n_res)


@pytest.mark.parametrize("make", [lambda: C.ns_ogrid8(128, 24, n_harm=2),
                                  lambda: C.ogrid(48, 12, n_harm=15, viscous=False)],
                         ids=["ns_ogrid8_128x24_nh2", "ogrid_48x12_nh15"])
def test_resumed_run_equals_the_oracle(make, tmp_path):
    """FP64: 4 iterations, save, load into a fresh context, 3 more.  The file's
    payload (compact interior order [block][snapshot][variable][k][j][i], the
    last values of the file) equals the oracle's state after 4 iterations, and
    the resumed state and its norms equal the oracle's 7 iterations, within
    1e-12 of max|U| (the FP64 trajectory tolerance of the parity tests)."""
    cs = make()
    o = Oracle(cs)
    U0 = o.init_state(C.noise(cs), 0.01)
    ctx = hb.HBContext(cs, "fp64")
    Ug = ctx.from_compact(torch.as_tensor(o.unpack(U0), device="cuda"))
    ctx.rk_smooth(Ug, 4)
    path = str(tmp_path / "state.hbr")
    ctx.save_state(Ug, path, iteration=4)
    assert ctx.sync_status() == hb.HB_OK
    U4, n4 = o.rk_smooth(U0, 4)
    count = C.interior_count(cs)
    payload = np.frombuffer(open(path, "rb").read()[-8 * count:], dtype=np.float64)
    ref4 = o.unpack(U4)
    scale = np.abs(ref4).max()
    assert np.abs(payload - ref4).max() < 1e-12 * scale
    ctx2 = hb.HBContext(cs, "fp64")
    V = ctx2.new_state()
    assert ctx2.load_state(V, path) == 4
    n_res = ctx2.rk_smooth(V, 3).cpu().numpy()
    assert ctx2.sync_status() == hb.HB_OK
    U7, n7 = o.rk_smooth(U4, 3)
    got = ctx2.to_compact(V).cpu().numpy()
    ref7 = o.unpack(U7)
    assert np.abs(got - ref7).max() < 1e-12 * np.abs(ref7).max()
    assert np.allclose(n_res, n7, rtol=1e-10, atol=0)


def test_foreign_and_broken_files_are_refused(tmp_path):
    cs = C.ns_ogrid8(128, 24, n_harm=2)
    ctx, U = _start(cs, "fp64")
    path = str(tmp_path / "a.hbr")
    ctx.save_state(U, path, iteration=7)
    # another grid, another harmonic count, another precision
    for other, prec in ((C.ns_ogrid8(136, 24, n_harm=2), "fp64"), (C.ns_ogrid8(128, 24, n_harm=3), "fp64"),
                        (cs, "fp32")):
        o = hb.HBContext(other, prec)
        with pytest.raises(hb.HBError) as e:
            o.load_state(o.new_state(), path)
        assert e.value.status == hb.HB_ERR_INVALID_ARG
    # truncated and missing files
    data = open(path, "rb").read()
    with open(str(tmp_path / "t.hbr"), "wb") as f:
        f.write(data[: len(data) // 2])
    for bad in (str(tmp_path / "t.hbr"), str(tmp_path / "missing.hbr")):
        with pytest.raises(hb.HBError):
            ctx.load_state(U, bad)
    # the intact file still loads
    assert ctx.load_state(U, path) == 7
    assert os.path.getsize(path) > 0
