"""The allocation-free norm entry point against the library's own RK norms.

hb_residual_norms_noalloc serves callers that cannot allocate device memory
(inside a graph capture, under a fixed memory pool); its scratch is a static
device array shared by every call.  This file is collected last so that a
failure here does not hide the other tests, and it must pass both alone in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest
import torch

from oracle.hb_oracle import Oracle
from paper_1304_7654_gb300 import cases as C
from paper_1304_7654_gb300 import hb

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_norms_match_rk_norms_on_two_calls(prec):
    import __graft_entry__ as g
    g.build()
    cs = C.ns_ogrid8(128, 24, n_harm=3)
    o = Oracle(cs)
    ctx = hb.HBContext(cs, prec)
    U = ctx.new_state()
    ctx.init_state(U, torch.as_tensor(C.noise(cs), device="cuda"), 0.01)
    # existing entry point: first-stage norms of one RK iteration
    ref = ctx.rk_smooth(U.clone(), 1)[0]
    # residual of the same state, rearranged to [n][v][cells] with volumes
    R = ctx.to_compact(ctx.residual(U))
    parts, vols, o_ = [], [], 0
    for b, blk in enumerate(cs.blocks):
        nc = blk.n[0] * blk.n[1]
        parts.append(R[o_:o_ + nc * cs.n_snap * cs.nv].reshape(cs.n_snap, cs.nv, nc))
        o_ += nc * cs.n_snap * cs.nv
        vol, _, _ = o.geometry(b)
        vols.append(vol[0, 2:-2, 2:-2].reshape(-1))
    Rn = torch.cat(parts, dim=2).contiguous()
    V = torch.as_tensor(np.concatenate(vols), device="cuda", dtype=Rn.dtype)
    ncells = V.numel()
    out1 = torch.full((cs.nv,), -1.0, dtype=torch.float64, device="cuda")
    out2 = torch.full((cs.nv,), -2.0, dtype=torch.float64, device="cuda")
    hb.residual_norms_noalloc(Rn, V, ncells, cs.n_snap, cs.nv, out1)
    hb.residual_norms_noalloc(Rn, V, ncells, cs.n_snap, cs.nv, out2)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert torch.allclose(out1, ref, rtol=tol, atol=0), (out1, ref)
    assert torch.equal(out1, out2)
    with pytest.raises(hb.HBError):          # nv above HB_NOALLOC_MAX_VARS (8)
        hb.residual_norms_noalloc(Rn, V, ncells, cs.n_snap, 9, out1)
