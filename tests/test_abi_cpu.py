"""The C-ABI library loads and exports every declared symbol; descriptor
validation runs on the host and rejects malformed inputs before any CUDA call."""
import ctypes as ct

import numpy as np
import pytest

from paper_1304_7654_gb300 import build as hbuild
from paper_1304_7654_gb300 import cases as C
from paper_1304_7654_gb300 import hb


@pytest.fixture(scope="module")
def lib():
    hbuild.build()
    return hb.load()


def test_exports_every_declared_function(lib):
    names = hb.declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def _create(case, prec=hb.HB_FP64):
    d, keep = hb._desc(case, prec)
    h = ct.c_void_p()
    st = hb.load().hb_create(ct.byref(d), ct.byref(h))
    if h.value:
        hb.load().hb_destroy(h)
    return st


def test_rejects_harmonics_above_maximum(lib):
    # 2D up to N_H = 15 (the paper's 31 snapshots); 3D up to N_H = 4
    cs = C.channel(8, 4, n_harm=16)
    assert _create(cs) == hb.HB_ERR_UNSUPPORTED
    assert _create(C.box3d(4, 4, 4, n_harm=5)) == hb.HB_ERR_UNSUPPORTED


def test_rejects_cut_outside_ghost_layers(lib):
    cs = C.ogrid(16, 8, n_harm=1)
    bad = cs.cuts.copy()
    bad[0, 2:5] = [0, 0, 0]          # box starting inside the block
    cs.cuts = bad
    assert _create(cs) == hb.HB_ERR_INVALID_ARG


def test_rejects_cut_source_out_of_range(lib):
    cs = C.ogrid(16, 8, n_harm=1)
    bad = cs.cuts.copy()
    bad[0, 9] += 50                  # source j beyond the block
    cs.cuts = bad
    assert _create(cs) == hb.HB_ERR_INVALID_ARG


def test_rejects_missing_ghost_coverage(lib):
    cs = C.channel(8, 4)
    cs.bcs = cs.bcs[1:]              # drop one boundary segment
    assert _create(cs) == hb.HB_ERR_INVALID_ARG


def test_rejects_double_fill_and_bad_types(lib):
    cs = C.channel(8, 4)
    cs.bcs = np.concatenate([cs.bcs, cs.bcs[:1]])
    assert _create(cs) == hb.HB_ERR_INVALID_ARG
    cs = C.channel(8, 4)
    bad = cs.bcs.copy()
    bad[0, 8] = 9
    cs.bcs = bad
    assert _create(cs) == hb.HB_ERR_INVALID_ARG


def test_rejects_bad_block_id_and_left_handed_block(lib):
    cs = C.ogrid(16, 8, n_harm=1)
    bad = cs.cuts.copy()
    bad[0, 1] = 7
    cs.cuts = bad
    assert _create(cs) == hb.HB_ERR_INVALID_ARG
    cs = C.channel(8, 4)
    cs.blocks[0].nodes = np.ascontiguousarray(cs.blocks[0].nodes[:, ::-1])   # mirrored: left-handed
    assert _create(cs) == hb.HB_ERR_INVALID_ARG


def test_null_arguments(lib):
    h = ct.c_void_p()
    assert lib.hb_create(None, ct.byref(h)) == hb.HB_ERR_INVALID_ARG
    assert lib.hb_destroy(None) == hb.HB_ERR_INVALID_ARG
    assert lib.hb_state_size(None) == -1
