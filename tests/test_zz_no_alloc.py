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
    # nv above HB_NOALLOC_MAX_VARS (8): refused by the library before any launch
    import ctypes as ct
    st = hb.load().hb_residual_norms_noalloc(
        ct.c_void_p(Rn.data_ptr()), ct.c_void_p(V.data_ptr()), hb.HB_FP32 if prec == "fp32" else hb.HB_FP64,
        ncells, cs.n_snap, 9, ct.c_void_p(out1.data_ptr()), ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == hb.HB_ERR_UNSUPPORTED


def test_noalloc_grid_stride_and_limits():
    """More cells than the fixed scratch has CTAs x threads (2048 x 256), so
    the grid-stride loop and the CTA clamp run: norms of a seeded 600,000-cell
    field against an FP64 reduction on the host, two calls in a row; sizes
    beyond the limits are refused before any launch."""
    import ctypes as ct
    import __graft_entry__ as g
    g.build()
    ncells, ns, nv = 600_000, 3, 4
    rng = np.random.default_rng(21)
    Rh = rng.normal(size=(ns, nv, ncells))
    Vh = rng.uniform(0.5, 2.0, size=ncells)
    ref = np.sqrt(((Rh / Vh) ** 2).sum(axis=(0, 2)) / (ncells * ns))
    R = torch.as_tensor(Rh, device="cuda")
    V = torch.as_tensor(Vh, device="cuda")
    out = torch.zeros(nv, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        hb.residual_norms_noalloc(R, V, ncells, ns, nv, out)
        torch.cuda.synchronize()
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0), (out, ref)
    # limits: checked on the host before any launch (valid pointers passed)
    lib = hb.load()
    s = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (ct.c_void_p(R.data_ptr()), ct.c_void_p(V.data_ptr()), hb.HB_FP64)
    assert lib.hb_residual_norms_noalloc(*args, (1 << 31) + 1, 1, 1, ct.c_void_p(out.data_ptr()), s) \
        == hb.HB_ERR_UNSUPPORTED
    assert lib.hb_residual_norms_noalloc(*args, (1 << 31) - 1, 1 << 10, 8, ct.c_void_p(out.data_ptr()), s) \
        == hb.HB_ERR_UNSUPPORTED
    # the binding refuses undersized or mismatched tensors before the call
    with pytest.raises(ValueError):
        hb.residual_norms_noalloc(R, V, ncells + 1, ns, nv, out)
    with pytest.raises(ValueError):
        hb.residual_norms_noalloc(R, V.float(), ncells, ns, nv, out)
    with pytest.raises(ValueError):
        hb.residual_norms_noalloc(R, V, ncells, ns, nv, out[:2])
