"""Batched persistent driver: many independent HB cases (different grids,
N_H, Mach, pitch) in one persistent cooperative launch per chunk of
iterations, against the same cases run alone and against the FP64 oracle;
bounded-barrier timeout (injected on the host: one CTA is told not to arrive);
autotuner."""
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


def _small_batch(n=6, seed=9):
    return C.batch_cases(n_cases=n, seed=seed, scale=(1.0, 4.0))


def _batch_state(ctx, cases):
    U = ctx.new_state()
    noise = torch.as_tensor(np.concatenate([C.noise(c) for c in cases]), device="cuda")
    ctx.init_state(U, noise, 0.01)
    return U


def _case_slices(ctx, cases):
    out, b0 = [], 0
    for c in cases:
        off0 = ctx.layouts[b0][0]
        b0 += len(c.blocks)
        end = ctx.layouts[b0][0] if b0 < len(ctx.layouts) else ctx.size
        out.append((off0, end))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_cases_run_alone(prec):
    cases = _small_batch()
    bctx = hb.HBContext(cases, prec)
    bctx.set_tuning(1, 32, 8)                      # persistent driver
    Ub = _batch_state(bctx, cases)
    nb = bctx.rk_smooth(Ub, 3)
    assert bctx.sync_status() == hb.HB_OK
    assert nb.shape == (3, len(cases), cases[0].nv)
    for k, (c, (a, e)) in enumerate(zip(cases, _case_slices(bctx, cases))):
        for mode in (1, 0):
            ctx = hb.HBContext(c, prec)
            ctx.set_tuning(mode, 32, 8)
            U = ctx.new_state()
            ctx.init_state(U, torch.as_tensor(C.noise(c), device="cuda"), 0.01)
            n1 = ctx.rk_smooth(U, 3)
            same = torch.equal(ctx.to_compact(U), ctx.to_compact(Ub[a:e].clone()))
            if mode == 1:
                assert same, (k, mode)           # same kernel: bitwise
                # the norms sum FP64 per-tile partials; the batch and the lone
                # case split their last wave into different row strips, so
                # the partials group differently: equal to FP64 rounding
                assert np.allclose(n1.cpu().numpy(), nb[:, k].cpu().numpy(), rtol=1e-12, atol=0), k
            else:   # a separately compiled kernel: equal to rounding
                a_, b_ = ctx.to_compact(U), ctx.to_compact(Ub[a:e].clone())
                assert (a_ - b_).abs().max() <= 2e-6 * b_.abs().max(), (k, (a_ - b_).abs().max())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_per_phase_batch_equals_cases_run_alone(prec):
    """Per-phase launches (one per case and stage): each case of the batch is
    bitwise the case advanced alone with the same driver and tile shape, also
    the N_s = 7 and 9 cases whose tiles park their balances in per-case slices
    of the stage scratch (the slices of different cases do not overlap)."""
    cases = _small_batch(8, seed=20)
    assert {7, 9} <= {c.n_snap for c in cases}
    bctx = hb.HBContext(cases, prec)
    bctx.set_tuning(0, 32, 8)
    Ub = _batch_state(bctx, cases)
    bctx.rk_smooth(Ub, 3, norms=False)
    assert bctx.sync_status() == hb.HB_OK
    for k, (c, (a, e)) in enumerate(zip(cases, _case_slices(bctx, cases))):
        ctx = hb.HBContext(c, prec)
        ctx.set_tuning(0, 32, 8)
        U = ctx.new_state()
        ctx.init_state(U, torch.as_tensor(C.noise(c), device="cuda"), 0.01)
        ctx.rk_smooth(U, 3, norms=False)
        assert torch.equal(ctx.to_compact(U), ctx.to_compact(Ub[a:e].clone())), (k, c.n_snap)


def test_batch_fp64_matches_oracle_per_case():
    cases = _small_batch(4, seed=19)
    bctx = hb.HBContext(cases, "fp64")
    bctx.set_tuning(1, 32, 8)
    Ub = _batch_state(bctx, cases)
    nb = bctx.rk_smooth(Ub, 2).cpu().numpy()
    for k, (c, (a, e)) in enumerate(zip(cases, _case_slices(bctx, cases))):
        o = Oracle(c)
        U = o.init_state(C.noise(c), 0.01)
        Uo, no = o.rk_smooth(U, 2)
        ctx = hb.HBContext(c, "fp64")
        got = ctx.to_compact(Ub[a:e].clone()).cpu().numpy()
        assert np.abs(got - o.unpack(Uo)).max() < 1e-12 * np.abs(o.unpack(Uo)).max(), k
        assert np.allclose(nb[:, k], no, rtol=1e-10), k


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_runs_as_one_persistent_launch_replayed_from_a_graph(prec):
    """The batched form: every chunk of the batch's RK iterations is one
    persistent cooperative launch, captured once into a CUDA graph and
    replayed (hb_graph_info), and the replayed chunks give the same state as
    direct launches of the same kernel (bitwise)."""
    cases = _small_batch(8, seed=29)
    bctx = hb.HBContext(cases, prec)
    bctx.set_tuning(1, 32, 8)
    Ub = _batch_state(bctx, cases)
    U2 = Ub.clone()
    bctx.rk_smooth(Ub, 5)
    bctx.rk_smooth(Ub, 5)
    assert bctx.sync_status() == hb.HB_OK
    cap, replays, persist_replays, direct = bctx.graph_info()
    assert cap == 1, "persistent chunk was not captured into a graph"
    assert persist_replays == 2 and replays == 2 and direct == 0
    # the same iterations without graphs (timing brackets single launches)
    bctx.set_timing(True)
    bctx.rk_smooth(U2, 5)
    bctx.rk_smooth(U2, 5)
    bctx.set_timing(False)
    assert bctx.sync_status() == hb.HB_OK
    assert bctx.graph_info()[3] == 2
    assert torch.equal(Ub, U2)


def test_tile_shape_and_driver_do_not_change_the_state():
    # each face is computed once from the same inputs whatever the tile shape
    # or row-strip split: a rerun is bitwise equal; other tile shapes and the
    # other driver are separately compiled kernels (the compiler may fuse a
    # multiply-add in one and not the other) and agree to FP32 rounding
    c = C.ns_ogrid8(128, 24, n_harm=2)
    ref = None
    for mode, TI, TJ in [(0, 32, 8), (0, 32, 4), (0, 16, 8), (1, 32, 8), (1, 32, 4), (1, 16, 8)]:
        runs = []
        for _ in range(2):
            ctx = hb.HBContext(c, "fp32")
            ctx.set_tuning(mode, TI, TJ)
            U = ctx.new_state()
            ctx.init_state(U, torch.as_tensor(C.noise(c), device="cuda"), 0.01)
            ctx.rk_smooth(U, 3)
            runs.append(U)
        assert torch.equal(runs[0], runs[1]), (mode, TI, TJ)
        if ref is None:
            ref = runs[0]
        assert (runs[0] - ref).abs().max() <= 2e-6 * ref.abs().max(), (mode, TI, TJ)


def test_barrier_timeout_is_reported_and_context_recovers():
    cases = _small_batch(3)
    os.environ["HB_TEST_SKIP_BARRIER_CTA"] = "0"
    os.environ["HB_BARRIER_TIMEOUT_MS"] = "200"
    try:
        bad = hb.HBContext(cases, "fp32")
    finally:
        del os.environ["HB_TEST_SKIP_BARRIER_CTA"]
        del os.environ["HB_BARRIER_TIMEOUT_MS"]
    bad.set_tuning(1, 32, 8)
    U = _batch_state(bad, cases)
    bad.rk_smooth(U, 1)
    assert bad.sync_status() == hb.HB_ERR_TIMEOUT
    # the GPU and a fresh context still work
    good = hb.HBContext(cases, "fp32")
    good.set_tuning(1, 32, 8)
    U2 = _batch_state(good, cases)
    good.rk_smooth(U2, 2)
    assert good.sync_status() == hb.HB_OK
    assert torch.isfinite(U2).all()


def test_autotuner_picks_a_built_configuration(tmp_path):
    os.environ["HB_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    try:
        cases = _small_batch(4)
        ctx = hb.HBContext(cases, "fp32")
        U = _batch_state(ctx, cases)
        U0 = U.clone()
        mode, TI, TJ = ctx.autotune(U, iters=2)
        assert torch.equal(U, U0)                       # U untouched
        assert (TI, TJ) in [(32, 8), (32, 4), (16, 8)] and mode in (0, 1)
        txt = (tmp_path / "tune.txt").read_text()
        assert f" {mode} {TI} {TJ}" in txt
        again = hb.HBContext(cases, "fp32")             # the cache is read at creation
        assert again.tuning() == (mode, TI, TJ)
    finally:
        del os.environ["HB_TUNE_CACHE"]
