"""Pins of the FP64 oracle to facts fixed by the mathematics, not by the oracle.

Every test here runs on the CPU.  Each one checks the oracle against a closed
form, an invariant of the discretisation, brute force, or an independent
restatement of a *definition* (the physical Euler flux, the Taylor polynomial
of the Runge-Kutta scheme, the exact divergence of a smooth field), chosen so
that a dropped term, a wrong sign or index, or a transposed operand anywhere in
the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_1304_7654_gb300 import cases as C
from oracle.hb_oracle import Oracle, d_matrix, roe_flux, van_albada

G = 1.4


# ------------------------------------------------------------------ helpers --
def euler_flux(W, S, vg=(0.0, 0.0, 0.0)):
    """Physical ALE Euler flux through area vector S (definition, 5 comps)."""
    rho, u, v, w, p = W
    S = np.asarray(list(S) + [0.0] * (3 - len(S)))
    vel = np.array([u, v, w])
    q = vel @ S
    qg = np.asarray(list(vg) + [0.0] * (3 - len(vg))) @ S
    rE = p / (G - 1) + 0.5 * rho * vel @ vel
    return np.array([rho * (q - qg), *(rho * vel * (q - qg) + p * S), rE * (q - qg) + p * q])


def cons5(W):
    rho, u, v, w, p = W
    return np.array([rho, rho * u, rho * v, rho * w, p / (G - 1) + 0.5 * rho * (u * u + v * v + w * w)])


def rand_state(rng, dim=2):
    W = np.array([rng.uniform(0.7, 1.3), rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6),
                  rng.uniform(-0.6, 0.6) if dim == 3 else 0.0, rng.uniform(0.5, 1.0)])
    return W


def interior_blocks(o, A):
    return [o.interior(A, b) for b in range(len(o.blocks))]


# ------------------------------------------------------------ D matrix (A1) --
@pytest.mark.parametrize("nh", list(range(0, 16)))
def test_d_matrix_differentiates_harmonics_exactly(nh):
    ns = 2 * nh + 1
    D = d_matrix(ns)
    th = 2 * np.pi * np.arange(ns) / ns
    for k in range(0, nh + 1):
        assert np.allclose(D @ np.cos(k * th), -k * np.sin(k * th), atol=1e-12 * max(1, ns))
        assert np.allclose(D @ np.sin(k * th), k * np.cos(k * th), atol=1e-12 * max(1, ns))
    # antisymmetric, zero row sums, spectrum i*k for k = -nh..nh
    assert np.allclose(D, -D.T, atol=0)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-12 * ns)
    ev = np.sort(np.linalg.eigvals(D).imag)
    assert np.allclose(ev, np.arange(-nh, nh + 1), atol=1e-9 * ns)


@pytest.mark.parametrize("nh", [1, 3, 8])
def test_d_matrix_aliases_above_nh(nh):
    ns = 2 * nh + 1
    D = d_matrix(ns)
    th = 2 * np.pi * np.arange(ns) / ns
    k = nh + 1            # aliases to -(nh): derivative is not recovered
    assert not np.allclose(D @ np.sin(k * th), k * np.cos(k * th), atol=1e-6)


def test_d_matrix_three_snapshots_closed_form():
    # 3-point trigonometric differentiation: D = (1/sqrt 3) [[0,1,-1],[-1,0,1],[1,-1,0]]
    r = 1 / math.sqrt(3.0)
    ref = r * np.array([[0, 1, -1], [-1, 0, 1], [1, -1, 0]], dtype=float)
    assert np.allclose(d_matrix(3), ref, atol=1e-15)


# ---------------------------------------------------------- van Albada (A4) --
def test_van_albada_properties():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = rng.normal(size=2)
        assert van_albada(a, a) == pytest.approx(a, rel=1e-14)
        assert abs(van_albada(a, -a)) < 1e-15
        assert van_albada(a, b) == pytest.approx(van_albada(b, a), rel=1e-14)
        if a * b > 0:   # same sign: limited slope lies between the two differences
            v = van_albada(a, b)
            assert min(a, b) - 1e-14 <= v <= max(a, b) + 1e-14
    assert van_albada(0.0, 0.0) == 0.0


# ------------------------------------------------------------------ Roe (A5) --
@pytest.mark.parametrize("dim", [2, 3])
def test_roe_consistency(dim):
    rng = np.random.default_rng(1)
    for _ in range(50):
        W = rand_state(rng, dim)
        S = rng.normal(size=dim)
        vg = rng.normal(size=dim) * 0.2
        F = roe_flux(W, W, S, vg, dim=dim)
        assert np.allclose(F, euler_flux(W, S, vg), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_roe_property_and_eigenvector_completeness(dim):
    rng = np.random.default_rng(2)
    for _ in range(50):
        WL, WR = rand_state(rng, dim), rand_state(rng, dim)
        S = rng.normal(size=dim)
        n = S / np.linalg.norm(S)
        vg = rng.normal(size=dim) * 0.2
        # sum_k lambda_k alpha_k r_k = F_R - F_L (per unit area, relative frame)
        lam = roe_flux(WL, WR, n, vg, dim=dim, mode=1)
        dF = euler_flux(WR, n, vg) - euler_flux(WL, n, vg)
        assert np.allclose(lam, dF, rtol=1e-12, atol=1e-12)
        # sum_k alpha_k r_k = U_R - U_L
        ar = roe_flux(WL, WR, n, vg, dim=dim, mode=2)
        assert np.allclose(ar, cons5(WR) - cons5(WL), rtol=1e-12, atol=1e-12)


def test_roe_supersonic_upwinding_and_rotation():
    rng = np.random.default_rng(3)
    S = np.array([0.7, -0.4])
    n = S / np.linalg.norm(S)
    for _ in range(20):
        WL = rand_state(rng)
        WR = rand_state(rng)
        c = math.sqrt(G * WL[4] / WL[0])
        WL[1:3] = 2.5 * c * n          # supersonic towards R
        WR[1:3] = 2.5 * c * n * 1.05
        F = roe_flux(WL, WR, S)
        assert np.allclose(F, euler_flux(WL, S), rtol=1e-12, atol=1e-12)
    # rotating states and face together rotates the momentum flux only
    for _ in range(20):
        WL, WR = rand_state(rng), rand_state(rng)
        S = rng.normal(size=2)
        phi = rng.uniform(0, 2 * np.pi)
        R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
        rot = lambda W: np.array([W[0], *(R @ W[1:3]), 0.0, W[4]])
        F = roe_flux(WL, WR, S)
        Fr = roe_flux(rot(WL), rot(WR), R @ S)
        assert np.allclose(Fr[[0, 4]], F[[0, 4]], rtol=1e-12, atol=1e-13)
        assert np.allclose(Fr[1:3], R @ F[1:3], rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------- geometry (A12) --
@pytest.mark.parametrize("make", [
    lambda: C.channel(12, 6),
    lambda: C.ns_ogrid8(64, 24, n_harm=1),
    lambda: C.periodic_box2d(10, 8),
    lambda: C.box3d(8, 6, 4, n_harm=1),
])
def test_geometry_closed_cells_and_positive_volumes(make):
    cs = make()
    o = Oracle(cs)
    for b, blk in enumerate(cs.blocks):
        vol, xc, S = o.geometry(b)
        _, p, g = o.blocks[b]
        n = blk.n
        assert vol.min() > 0
        # sum of outward face vectors of every cell away from the last ghost layer
        tot = np.zeros_like(xc)
        for d in range(cs.dim):
            ax = 2 - d
            lo = S[d]
            hi = np.roll(S[d], -1, axis=ax)
            tot += hi - lo
        sl = tuple(slice(g[2 - a], g[2 - a] + n[2 - a]) for a in range(3))
        assert np.abs(tot[sl]).max() < 1e-12 * max(1.0, np.abs(S).max())


@pytest.mark.parametrize("make", [
    lambda: C.ns_ogrid8(),
    lambda: C.adjoint_ogrid4(),
    lambda: C.paper_tc1(),
    lambda: C.paper_tc2(1024, 256),
    lambda: C.channel(),
    lambda: C.box3d(),
], ids=["ns_ogrid8", "adjoint_ogrid4", "paper_tc1", "paper_tc2_1024x256", "channel", "box3d"])
def test_every_padded_cell_has_positive_volume_at_full_size(make):
    """Reading A12 (point-reflected ghost nodes) needs ghost cells that are
    cells: every padded cell of every benchmark workload, ghosts included, has
    a positive volume.  The sharp trailing edge of the O-grids is where this
    can fail (neighbouring grid lines meeting inside the body)."""
    cs = make()
    o = Oracle(cs)
    for b in range(len(cs.blocks)):
        vol, _, _ = o.geometry(b)
        _, p, g = o.blocks[b]
        n = cs.blocks[b].n
        inner = vol[tuple(slice(g[2 - a], g[2 - a] + n[2 - a]) for a in range(3))]
        assert vol.min() > 0.5 * inner.min(), (b, vol.min(), inner.min())


def test_every_padded_cell_of_the_batch_has_positive_volume():
    for cs in C.batch_cases():
        o = Oracle(cs)
        vol, _, _ = o.geometry(0)
        assert vol.min() > 0, cs.name


def test_volumes_fill_the_domain():
    cs = C.channel(20, 10)
    o = Oracle(cs)
    vol, _, _ = o.geometry(0)
    assert vol[0, 2:-2, 2:-2].sum() == pytest.approx(2.0, rel=1e-13)
    cs = C.box3d(8, 6, 4, n_harm=1)
    o = Oracle(cs)
    vol, _, _ = o.geometry(0)
    assert vol[2:-2, 2:-2, 2:-2].sum() == pytest.approx(4.0, rel=1e-12)


# --------------------------------------------------- freestream preservation --
def _freestream(cs):
    o = Oracle(cs)
    U = o.init_state(np.zeros(C.interior_count(cs)), 0.0)
    R, sc = o.residual(U)
    return o, R, sc


def test_freestream_channel_all_cells():
    cs = C.channel(16, 8)
    cs.ubc_amp = 0.0
    o, R, sc = _freestream(cs)
    assert np.max(np.abs(R) / np.maximum(sc, 1e-300)) < 1e-14


@pytest.mark.parametrize("viscous", [False, True])
def test_freestream_pitching_ogrid_away_from_wall(viscous):
    cs = C.ns_ogrid8(64, 24, n_harm=2, viscous=viscous)
    o, R, sc = _freestream(cs)
    for b, blk in enumerate(cs.blocks):
        r = o.interior(R, b)
        s = o.interior(sc, b)
        j0 = 3 if b < 4 else 0          # inner-ring blocks touch the wall
        j1 = blk.n[1] - (3 if b >= 4 else 0)
        assert np.max(np.abs(r[:, :, :, j0:j1]) / s[:, :, :, j0:j1]) < 1e-13


def test_freestream_box3d():
    cs = C.box3d(8, 8, 4, n_harm=1, gust=0.0)
    o, R, sc = _freestream(cs)
    r = o.interior(R, 0)[:, :, :, 3:, :]
    s = o.interior(sc, 0)[:, :, :, 3:, :]
    assert np.max(np.abs(r) / s) < 1e-13


# ---------------------------------------------- HB source, steady special case --
def test_hb_source_vanishes_for_identical_snapshots():
    steady = C.channel(12, 6, n_harm=0)
    steady.ubc_amp = 0.0
    hb = C.channel(12, 6, n_harm=2)
    hb.ubc_amp = 0.0
    os_, oh = Oracle(steady), Oracle(hb)
    rng = np.random.default_rng(4)
    Us = os_.init_state(rng.uniform(-1, 1, C.interior_count(steady)), 0.01)
    Is = os_.unpack(Us).reshape(1, -1)
    Uh = oh.pack(np.repeat(Is, hb.n_snap, axis=0).reshape(-1))
    Rs = os_.unpack(os_.residual(Us, with_scale=False)).reshape(1, -1)
    Rh = oh.unpack(oh.residual(Uh, with_scale=False)).reshape(hb.n_snap, -1)
    for n in range(hb.n_snap):
        assert np.allclose(Rh[n], Rs[0], rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------- conservation --
def _periodic_multiblock(ni=16, nj=12, **kw):
    specs = [C.BlockSpec((0, 0), (10, 7)), C.BlockSpec((10, 0), (16, 7)),
             C.BlockSpec((0, 7), (5, 12)), C.BlockSpec((5, 7), (16, 12), flip=True)]
    return C.periodic_box2d(ni, nj, specs=specs, **kw)


@pytest.mark.parametrize("viscous", [False, True])
def test_discrete_conservation_periodic(viscous):
    cs = _periodic_multiblock(viscous=viscous, n_harm=2)
    o = Oracle(cs)
    U = o.init_state(C.noise(cs, 12), 0.05)
    R, sc = o.residual(U)
    D = d_matrix(cs.n_snap)
    tot = np.zeros((cs.n_snap, cs.nv))
    hb = np.zeros((cs.n_snap, cs.nv))
    scale = 0.0
    for b in range(len(cs.blocks)):
        vol, _, _ = o.geometry(b)
        _, p, g = o.blocks[b]
        n = cs.blocks[b].n
        V = vol[:, g[1]:g[1] + n[1], g[0]:g[0] + n[0]]
        r = o.interior(R, b)
        u = o.interior(U, b)
        tot += r.sum(axis=(2, 3, 4))
        hb += cs.omega * np.einsum("nm,mvkji,kji->nv", D, u, V)
        scale = max(scale, o.interior(sc, b).sum())
    # interior fluxes telescope; the HB term sums to zero over snapshots
    assert np.abs(tot.sum(axis=0)).max() < 1e-13 * scale
    assert np.abs(tot - hb).max() < 1e-13 * scale


# ---------------------------------------------------- cut transparency (A6) --
def _global_to_blocks(I, specs, blocks):
    parts = []
    for sp, blk in zip(specs, blocks):
        a = I[..., sp.lo[1]:sp.hi[1], sp.lo[0]:sp.hi[0]]
        if sp.flip:
            a = a[..., ::-1, ::-1]
        parts.append(np.ascontiguousarray(a).reshape(-1))
    return np.concatenate(parts)


@pytest.mark.parametrize("kind", ["ogrid8", "channel_flip", "periodic"])
def test_multiblock_equals_single_block(kind):
    if kind == "ogrid8":
        ni, nj = 64, 24
        one = C.ogrid(ni, nj, n_harm=1, viscous=True)
        specs = C.ogrid8_specs(ni, nj)
        many = C.ns_ogrid8(ni, nj, n_harm=1, viscous=True)
    elif kind == "channel_flip":
        ni, nj = 16, 8
        one = C.channel(ni, nj, viscous=True)
        specs = [C.BlockSpec((0, 0), (9, 8)), C.BlockSpec((9, 0), (16, 3), flip=True),
                 C.BlockSpec((9, 3), (16, 8))]
        many = C.channel(ni, nj, blocks=specs, viscous=True)
    else:
        ni, nj = 16, 12
        one = C.periodic_box2d(ni, nj, viscous=True)
        many = _periodic_multiblock(viscous=True)
        specs = [C.BlockSpec((0, 0), (10, 7)), C.BlockSpec((10, 0), (16, 7)),
                 C.BlockSpec((0, 7), (5, 12)), C.BlockSpec((5, 7), (16, 12), flip=True)]
    o1, om = Oracle(one), Oracle(many)
    U1 = o1.init_state(C.noise(one, 3), 0.02)
    I1 = o1.unpack(U1).reshape(one.n_snap, one.nv, nj, ni)
    Um = om.pack(_global_to_blocks(I1, specs, many.blocks))
    R1, S1 = o1.residual(U1)
    Rm = om.residual(Um, with_scale=False)
    G1 = _global_to_blocks(o1.unpack(R1).reshape(one.n_snap, one.nv, nj, ni), specs, many.blocks)
    GS = _global_to_blocks(o1.unpack(S1).reshape(one.n_snap, one.nv, nj, ni), specs, many.blocks)
    assert np.max(np.abs(om.unpack(Rm) - G1) / GS) < 1e-14


# --------------------------------------------------------- rotation invariance --
def test_rotation_invariance_channel():
    # the limiter acts on Cartesian velocity components; it is odd and
    # symmetric, so the discrete residual is covariant under quarter turns
    phi = 0.5 * math.pi
    cs = C.channel(12, 6, viscous=True)
    rc = C.channel(12, 6, viscous=True)
    R2 = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
    for blk in rc.blocks:
        blk.nodes = np.ascontiguousarray(blk.nodes @ R2.T)
    rc.alpha0_deg = math.degrees(phi)
    o, orr = Oracle(cs), Oracle(rc)
    U = o.init_state(C.noise(cs, 5), 0.02)
    Ur = U.copy()
    v = orr.block_view(Ur, 0)
    m = o.block_view(U, 0)
    v[:, 1] = R2[0, 0] * m[:, 1] + R2[0, 1] * m[:, 2]
    v[:, 2] = R2[1, 0] * m[:, 1] + R2[1, 1] * m[:, 2]
    R, sc = o.residual(U)
    Rr = orr.residual(Ur, with_scale=False)
    a, b = o.block_view(R, 0), orr.block_view(Rr, 0)
    s = o.block_view(sc, 0)
    exp = a.copy()
    exp[:, 1] = R2[0, 0] * a[:, 1] + R2[0, 1] * a[:, 2]
    exp[:, 2] = R2[1, 0] * a[:, 1] + R2[1, 1] * a[:, 2]
    ss = np.maximum(s, s[:, 1:3].max(axis=1, keepdims=True) * (np.arange(4) >= 0)[None, :, None, None, None])
    assert np.max(np.abs(b - exp) / np.maximum(ss, 1e-300)) < 1e-13
    # local time steps are rotation invariant too
    assert np.allclose(o.time_step(U), orr.time_step(Ur), rtol=1e-13)


# ------------------------------------------------ Runge-Kutta scheme (A9) --
def test_rk_amplification_is_fourth_order_taylor():
    # uniform periodic grid: every cell has the same time step, so a state that
    # is uniform in space stays uniform and only the HB source acts
    cs = C.periodic_box2d(6, 5, n_harm=2, perturb=0.0)
    o = Oracle(cs)
    ns, nv = cs.n_snap, cs.nv
    rng = np.random.default_rng(6)
    base = np.array([1.0, 0.3, 0.1, 1 / (G - 1) / G + 0.05])
    snap = base[None, :] * (1 + 0.05 * rng.uniform(-1, 1, size=(ns, nv)))
    I = np.broadcast_to(snap[:, :, None, None, None], (ns, nv, 1, 5, 6))
    U = o.pack(I.reshape(-1))
    dt = o.interior(o.time_step(U), 0)[:, 0, 0]          # [n][j][i]
    vol, _, _ = o.geometry(0)
    U1, _ = o.rk_smooth(U, 1)
    out = o.interior(U1, 0)
    D = d_matrix(ns)
    for (j, i) in [(0, 0), (2, 3), (4, 5)]:
        Z = -np.diag(dt[:, j, i]) @ (cs.omega * D)        # dU/dtau = -(1/V) R = -omega D U
        P = np.eye(ns) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
        exp = P @ snap
        assert np.allclose(out[:, :, 0, j, i], exp, rtol=1e-12, atol=1e-13)


def test_rk_norms_are_rms_of_first_stage_residual():
    cs = C.channel(12, 6, n_harm=1)
    o = Oracle(cs)
    U = o.init_state(C.noise(cs), 0.01)
    R = o.residual(U, with_scale=False)
    vol, _, _ = o.geometry(0)
    r = o.interior(R, 0) / vol[None, None, 0:1, 2:-2, 2:-2]
    exp = np.sqrt(np.mean(r ** 2, axis=(0, 2, 3, 4)))
    _, norms = o.rk_smooth(U, 1)
    assert np.allclose(norms[0], exp, rtol=1e-13)


# --------------------------------------- manufactured-solution order (A18) --
def _mms_prim(x, y, t):
    s = 1 + 0.05 * np.sin(t)
    rho = (1 + 0.1 * x + 0.05 * np.exp(0.5 * y)) * s
    u = 0.3 + 0.1 * y + 0.05 * np.exp(0.3 * x)
    v = 0.1 + 0.05 * x + 0.1 * y * y
    p = 1 / G * (1 + 0.1 * x + 0.05 * y + 0.02 * np.exp(0.2 * y)) * s
    return rho, u, v, p


def _fd(f, x, h=1e-3):
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


def _mms_flux(x, y, t, nx, ny, mu, kap):
    rho, u, v, p = _mms_prim(x, y, t)
    q = u * nx + v * ny
    E = p / (G - 1) / rho + 0.5 * (u * u + v * v)
    F = np.array([rho * q, rho * u * q + p * nx, rho * v * q + p * ny, (rho * E + p) * q])
    if mu == 0.0:
        return F
    T = lambda xx, yy: G * _mms_prim(xx, yy, t)[3] / _mms_prim(xx, yy, t)[0]
    ux = _fd(lambda a: _mms_prim(a, y, t)[1], x)
    uy = _fd(lambda a: _mms_prim(x, a, t)[1], y)
    vx = _fd(lambda a: _mms_prim(a, y, t)[2], x)
    vy = _fd(lambda a: _mms_prim(x, a, t)[2], y)
    Tx, Ty = _fd(lambda a: T(a, y), x), _fd(lambda a: T(x, a), y)
    div = ux + vy
    txx, tyy, txy = mu * (2 * ux - 2 / 3 * div), mu * (2 * vy - 2 / 3 * div), mu * (uy + vx)
    Fv = np.array([0 * x, txx * nx + txy * ny, txy * nx + tyy * ny,
                   u * (txx * nx + txy * ny) + v * (txy * nx + tyy * ny) + kap * (Tx * nx + Ty * ny)])
    return F - Fv


@pytest.mark.parametrize("viscous", [False, True])
def test_manufactured_solution_truncation_order(viscous):
    """R_h/V approaches div F(U) + dU/dt at cell centroids at second order (or
    better) on a smoothly perturbed grid; the time part (one harmonic <= N_H)
    is exact, so only the spatial error remains."""
    mach, re = 0.5, 50.0
    mu = mach / re if viscous else 0.0
    kap = mu / ((G - 1) * 0.72)
    errs = []
    for n in (16, 32, 64):
        cs = C.channel(n, n // 2, n_harm=1, viscous=viscous)
        cs.reynolds = re
        cs.ubc_amp = 0.0
        o = Oracle(cs)
        vol, xc, _ = o.geometry(0)
        X, Y = xc[0, :, :, 0], xc[0, :, :, 1]
        U = np.zeros(o.size)
        bv = o.block_view(U, 0)
        ts = 2 * np.pi * np.arange(3) / 3
        for k in range(3):
            rho, u, v, p = _mms_prim(X, Y, ts[k])
            bv[k] = np.array([rho, rho * u, rho * v, p / (G - 1) + 0.5 * rho * (u * u + v * v)])[:, None]
        R = o.residual(U, with_scale=False)
        e = []
        for k in range(3):
            div = (_fd(lambda a: _mms_flux(a, Y, ts[k], 1, 0, mu, kap), X)
                   + _fd(lambda a: _mms_flux(X, a, ts[k], 0, 1, mu, kap), Y))
            rho_t = lambda tt: np.array([
                _mms_prim(X, Y, tt)[0], _mms_prim(X, Y, tt)[0] * _mms_prim(X, Y, tt)[1],
                _mms_prim(X, Y, tt)[0] * _mms_prim(X, Y, tt)[2],
                _mms_prim(X, Y, tt)[3] / (G - 1) + 0.5 * _mms_prim(X, Y, tt)[0]
                * (_mms_prim(X, Y, tt)[1] ** 2 + _mms_prim(X, Y, tt)[2] ** 2)])
            dudt = _fd(rho_t, ts[k]) * cs.omega
            err = o.block_view(R, 0)[k, :, 0] / vol[0] - div - dudt
            e.append(err[:, 4:-4, 4:-4])
        errs.append(np.sqrt(np.mean(np.array(e) ** 2, axis=(0, 2, 3))))
    errs = np.array(errs)
    order = np.log2(errs[:-1] / errs[1:])
    assert (order >= 1.9).all(), order


# ----------------------------------------------------------------- forces --
def test_uniform_pressure_on_closed_body_gives_no_force():
    cs = C.ogrid(48, 12, n_harm=1, viscous=False, pitch_deg=3.0)
    o = Oracle(cs)
    U = np.zeros(o.size)
    for b in range(len(cs.blocks)):
        v = o.interior(U, b)
        v[:, 0] = 1.3
        v[:, 1:3] = 0.0
        v[:, 3] = 2.0 / G / (G - 1)           # p = 2 p_inf, fluid at rest
    coef, J = o.forces(U)
    assert np.abs(coef[:, :, :2]).max() < 1e-13


def test_symmetric_airfoil_at_zero_incidence_has_zero_lift():
    cs = C.ogrid(48, 16, n_harm=0, viscous=True, pitch_deg=0.0)
    o = Oracle(cs)
    U = o.init_state(np.zeros(C.interior_count(cs)), 0.0)
    U, _ = o.rk_smooth(U, 30)
    coef, J = o.forces(U)
    assert abs(coef[0, 0, 0]) < 1e-10 * abs(coef[0, 0, 1])
    assert abs(J) < 1e-10 * abs(coef[0, 0, 1])


# ---------------------------------------------------------- adjoint columns --
def test_adjoint_columns_dual_match_central_differences():
    cs = C.adjoint_ogrid4(64, 16, n_harm=1)
    o = Oracle(cs)
    U = o.init_state(C.noise(cs), 0.01)
    U, _ = o.rk_smooth(U, 3)
    rng = np.random.default_rng(11)
    psi = rng.normal(size=o.size)
    cells = C.sample_cells(cs, 6, 11)
    cols = np.array([[*c, v, n] for c in cells for v in range(cs.nv) for n in (0, cs.n_snap - 1)])
    exact = o.adjoint_columns(U, psi, 0.7, cols, mode=0)
    # central differences carry an O(h^2) truncation error (measured: x100 per
    # decade of h); h = 1e-7 keeps it near 1e-8 relative, above FP64 rounding
    fd = o.adjoint_columns(U, psi, 0.7, cols, mode=1, h=1e-7)
    scale = np.abs(exact).max()
    assert np.max(np.abs(exact - fd)) < 1e-6 * scale
    # wall-adjacent cells see the functional
    wall = np.array([[0, 3, 0, 0, v, 0] for v in range(cs.nv)])
    ej = o.adjoint_columns(U, psi * 0, 1.0, wall, mode=0)
    fj = o.adjoint_columns(U, psi * 0, 1.0, wall, mode=1, h=1e-7)
    assert np.abs(ej).max() > 0
    assert np.max(np.abs(ej - fj)) < 1e-6 * np.abs(ej).max()


def test_multiblock_equals_single_block_3d():
    ni, nj, nk = 8, 6, 6
    one = C.box3d(ni, nj, nk, n_harm=1)
    specs = [C.BlockSpec((0, 0, 0), (5, 6, 3)), C.BlockSpec((5, 0, 0), (8, 6, 3)),
             C.BlockSpec((0, 0, 3), (8, 4, 6)), C.BlockSpec((0, 4, 3), (8, 6, 6))]
    many = C.box3d(ni, nj, nk, n_harm=1, specs=specs)
    o1, om = Oracle(one), Oracle(many)
    U1 = o1.init_state(C.noise(one, 3), 0.02)
    I1 = o1.unpack(U1).reshape(one.n_snap, one.nv, nk, nj, ni)

    def split(A):
        return np.concatenate([np.ascontiguousarray(
            A[..., s.lo[2]:s.hi[2], s.lo[1]:s.hi[1], s.lo[0]:s.hi[0]]).reshape(-1) for s in specs])

    R1, S1 = o1.residual(U1)
    Rm = om.residual(om.pack(split(I1)), with_scale=False)
    shp = (one.n_snap, one.nv, nk, nj, ni)
    ref = split(o1.unpack(R1).reshape(shp))
    sc = split(o1.unpack(S1).reshape(shp))
    assert np.max(np.abs(om.unpack(Rm) - ref) / sc) < 1e-14


# ------------------------------------------- time-domain dual time stepping --
def test_td_bdf2_term_is_exact_for_quadratics_in_time():
    # on a doubly periodic grid a spatially uniform state has zero flux
    # balance (closed cells), so R* / V is the time term alone; BDF2 is exact
    # for states quadratic in t: R*/V = dU/dt = B + 2 C t at t_(k+1)
    cs = C.periodic_box2d(8, 6, n_harm=0)
    o = Oracle(cs)
    A = np.array([1.0, 0.3, -0.1, 0.8])
    B = np.array([0.02, -0.01, 0.03, 0.05])
    Cq = np.array([0.004, 0.002, -0.003, 0.001])
    t1, dt = 0.7, 0.05
    at = lambda t: A + B * t + Cq * t * t

    def state(t):   # conservative variables uniform in space
        flat = np.concatenate([np.repeat(at(t)[:, None], b.n[0] * b.n[1], axis=1).ravel() for b in cs.blocks])
        return o.pack(flat)

    vols = [o.geometry(b)[0][0, 2:-2, 2:-2].ravel() for b in range(len(cs.blocks))]

    def per_var(R):
        out, k = [], 0
        for b, blk in enumerate(cs.blocks):
            m = blk.n[0] * blk.n[1]
            for v in range(4):
                out.append((v, R[k:k + m] / vols[b]))
                k += m
        return out

    U, Un, Unm1 = state(t1), state(t1 - dt), state(t1 - 2 * dt)
    for v, got in per_var(o.unpack(o.td_residual(U, Un, Unm1, t1, dt))):
        assert np.allclose(got, B[v] + 2 * Cq[v] * t1, rtol=0, atol=1e-11), v
    # the first step (no U^(n-1)) is backward Euler: (U - U^n) / dt
    for v, got in per_var(o.unpack(o.td_residual(U, Un, None, t1, dt))):
        assert np.allclose(got, (at(t1)[v] - at(t1 - dt)[v]) / dt, rtol=0, atol=1e-11), v


def test_td_residual_at_rest_in_time_is_the_steady_residual():
    # U = U^n = U^(n-1): the time term vanishes; at t = 0 the frame is the one
    # of the single HB snapshot, so R* equals the N_H = 0 residual
    cs = C.ogrid(24, 8, n_harm=0, viscous=True, pitch_deg=3.0)
    o = Oracle(cs)
    U = o.init_state(C.noise(cs), 0.01)
    R0 = o.residual(U, with_scale=False)
    Rt = o.td_residual(U, U, U, 0.0, 0.1)
    # (3/2 - 2 + 1/2) U is zero up to the rounding of the BDF combination
    assert np.abs(o.unpack(Rt) - o.unpack(R0)).max() <= 1e-12 * np.abs(o.unpack(R0)).max()


# ------------------------------------- viscous flux, linear velocity field --
def _affine_channel(ni, nj, viscous):
    """Single-block channel on a skewed affine grid (every cell the same
    parallelogram), steady (N_H = 0)."""
    xi = np.linspace(0.0, 2.0, ni + 1)
    eta = np.linspace(0.0, 1.0, nj + 1)
    X, Y = np.meshgrid(xi, eta)
    gn = np.stack([X + 0.3 * Y, 0.1 * X + Y], axis=-1)
    ext = C.extend_ghost_nodes(gn, 2, (False, False))
    side_bc = {(0, 0): (C.BC_FARFIELD, -1), (0, 1): (C.BC_FARFIELD, -1),
               (1, 0): (C.BC_SLIP, -1), (1, 1): (C.BC_SLIP, -1)}
    bl, cuts, bcs = C.split_blocks(ext, 2, (ni, nj), (False, False), side_bc,
                                   [C.BlockSpec((0, 0), (ni, nj))])
    return C.Case(name="affine_channel", dim=2, n_harm=0, mach=0.5, omega=0.1, viscous=viscous,
                  blocks=bl, cuts=cuts, bcs=bcs, n_bodies=0, seed=1)


def test_viscous_flux_of_a_linear_velocity_field_is_exact_on_an_affine_grid():
    """Reading A6 (Green-Gauss cell gradients from face means, face gradient =
    mean + edge-normal correction, Stokes stress, Fourier heat flux) with the
    constant viscosity of A17.  For uniform density and pressure and a linear
    velocity u = u0 + A x on a grid of equal parallelograms, every gradient is
    exact, the stress tau = mu (A + A^T - 2/3 tr(A) I) is constant and T is
    uniform, so the viscous part of each interior residual (viscous run minus
    inviscid run) is, by the divergence theorem, zero in mass and momentum
    and -V tau : A in energy.  A wrong gradient factor, stress coefficient or
    sign, or a dropped -2/3 div term, breaks it."""
    ni, nj = 24, 16
    A = np.array([[0.03, -0.02], [0.05, 0.01]])          # A[i][j] = d u_i / d x_j
    u0 = np.array([0.5, 0.0])
    on, off = Oracle(_affine_channel(ni, nj, True)), Oracle(_affine_channel(ni, nj, False))
    vol, xc, _ = on.geometry(0)
    U = np.zeros(on.size)
    blk = on.block_view(U, 0)
    vel = u0[:, None, None, None] + np.einsum("ab,kjib->akji", A, xc[..., :2])
    p = 1.0 / G
    blk[0, 0] = 1.0
    blk[0, 1] = vel[0]
    blk[0, 2] = vel[1]
    blk[0, 3] = p / (G - 1) + 0.5 * (vel[0] ** 2 + vel[1] ** 2)
    Rv = on.interior(on.residual(U, with_scale=False), 0) - off.interior(off.residual(U, with_scale=False), 0)
    mu = 0.5 / 5.0e3
    tau = mu * (A + A.T - 2.0 / 3.0 * np.trace(A) * np.eye(2))
    phi = float(np.sum(tau * A))
    _, _, g = on.blocks[0]
    V = vol[:, g[1]:g[1] + nj, g[0]:g[0] + ni]
    inner = (slice(None), slice(3, nj - 3), slice(3, ni - 3))   # cells whose stencils see no ghost
    scale = mu * np.abs(A).max() * 2.2                          # |tau| |S| with |S| ~ 0.1
    r = Rv[0]
    assert np.abs(r[0][inner]).max() < 1e-12 * scale
    assert np.abs(r[1][inner]).max() < 1e-9 * scale
    assert np.abs(r[2][inner]).max() < 1e-9 * scale
    np.testing.assert_allclose(r[3][inner], -V[inner] * phi, rtol=1e-8, atol=1e-9 * scale)


# ----------------------------------------------- viscous wall traction, Couette --
def _couette_case(ni, nj, L, H):
    """Uniform grid on [0, L] x [0, H], periodic in x; no-slip wall at y = 0
    (body 0, at rest), slip wall at y = H; steady, laminar."""
    X, Y = np.meshgrid(np.linspace(0.0, L, ni + 1), np.linspace(0.0, H, nj + 1))
    ext = C.extend_ghost_nodes(np.stack([X, Y], axis=-1), 2, (True, False),
                               period_shift=[np.array([L, 0.0]), np.zeros(2)])
    side_bc = {(1, 0): (C.BC_NOSLIP, 0), (1, 1): (C.BC_SLIP, -1)}
    bl, cuts, bcs = C.split_blocks(ext, 2, (ni, nj), (True, False), side_bc,
                                   [C.BlockSpec((0, 0), (ni, nj))])
    return C.Case(name="couette", dim=2, n_harm=0, mach=0.4, omega=0.1, viscous=True,
                  blocks=bl, cuts=cuts, bcs=bcs, n_bodies=1, seed=1)


def test_couette_wall_shear_gives_the_exact_skin_friction_force():
    """Force reading (A14: wall pressure p_0, traction tau_w . S from the face
    gradient, coefficients over 1/2 rho_inf U_inf^2 c with c = 1) and the
    no-slip ghost u_g = -u: plane Couette flow u = U0 y / H over the wall at
    rest, uniform density and pressure.  The mirrored ghosts continue the
    linear profile, so the wall gradient is exact and the fluid pulls the
    wall downstream with tau_xy = mu U0 / H over its length L: cd = mu U0 L /
    (H q_inf), cl = 0 (no pressure excess, tau_yy = 0), cm = 0 (the force acts
    on the line y = 0 through the pivot's height)."""
    ni, nj, L, H, U0 = 16, 8, 1.0, 0.5, 0.3
    cs = _couette_case(ni, nj, L, H)
    o = Oracle(cs)
    _, xc, _ = o.geometry(0)
    U = np.zeros(o.size)
    blk = o.block_view(U, 0)
    u = U0 * xc[..., 1] / H
    p = 1.0 / G
    blk[0, 0] = 1.0
    blk[0, 1] = u
    blk[0, 2] = 0.0
    blk[0, 3] = p / (G - 1) + 0.5 * u * u
    coef, J = o.forces(U)
    mu = cs.mach / cs.reynolds
    qinf = 0.5 * cs.mach ** 2
    cd = mu * U0 * L / (H * qinf)
    cl_, cd_, cm_ = coef[0, 0]
    assert abs(cd_ - cd) < 1e-12 * cd, (cd_, cd)
    assert abs(cl_) < 1e-12 * cd and abs(cm_) < 1e-12 * cd, (cl_, cm_)
    assert J == cl_


# ------------------------------------------- farfield characteristic ghosts --
def test_farfield_ghosts_carry_the_characteristic_invariants():
    """Reading of the farfield condition (1D characteristics normal to the
    face): the ghost state carries the outgoing Riemann invariant
    R+ = q_n + 2c/(gamma-1) of the first interior cell and the incoming
    R- = q_n - 2c/(gamma-1) of the freestream; entropy p / rho^gamma and the
    tangential velocity come from the interior on outflow and from the
    freestream on inflow; both ghost layers hold it.  Checked on the straight
    inlet (x = 0) and outlet (x = 2) of the channel, steady, from a random
    subsonic state around the freestream (M = 0.5, zero incidence)."""
    cs = C.channel(24, 8, n_harm=0)
    o = Oracle(cs)
    rng = np.random.default_rng(3)
    _, p_, g = o.blocks[0]
    ni, nj = cs.blocks[0].n[0], cs.blocks[0].n[1]
    U = np.zeros(o.size)
    blk = o.block_view(U, 0)
    sh = blk[0, 0].shape
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, sh)
    u = 0.5 + 0.05 * rng.uniform(-1, 1, sh)
    v = 0.05 * rng.uniform(-1, 1, sh)
    p = (1.0 / G) * (1.0 + 0.05 * rng.uniform(-1, 1, sh))
    blk[0, 0], blk[0, 1], blk[0, 2] = rho, rho * u, rho * v
    blk[0, 3] = p / (G - 1) + 0.5 * rho * (u * u + v * v)
    F = o.block_view(o.fill_ghosts(U), 0)[0, :, 0]           # [v][j][i], padded

    def prim(i, j):
        r = F[0, j, i]
        uu, vv = F[1, j, i] / r, F[2, j, i] / r
        pp = (G - 1) * (F[3, j, i] - 0.5 * r * (uu * uu + vv * vv))
        return r, uu, vv, pp

    Wf = (1.0, 0.5, 0.0, 1.0 / G)
    for j in range(g[1], g[1] + nj):
        for side, nx in ((0, -1.0), (1, 1.0)):                   # inlet: outward -x, outlet: +x
            i_in = g[0] if side == 0 else g[0] + ni - 1
            ghosts = (g[0] - 1, g[0] - 2) if side == 0 else (g[0] + ni, g[0] + ni + 1)
            ri, ui, vi, pi = prim(i_in, j)
            ci = math.sqrt(G * pi / ri)
            cf = math.sqrt(G * Wf[3] / Wf[0])
            Rp = nx * ui + 2 * ci / (G - 1)
            Rm = nx * Wf[1] - 2 * cf / (G - 1)
            src = (ri, ui, vi, pi) if side == 1 else Wf              # outflow at the outlet
            for ig in ghosts:
                rg, ug, vg, pg = prim(ig, j)
                cg = math.sqrt(G * pg / rg)
                assert abs(nx * ug + 2 * cg / (G - 1) - Rp) < 1e-12
                assert abs(nx * ug - 2 * cg / (G - 1) - Rm) < 1e-12
                assert abs(pg / rg ** G - src[3] / src[0] ** G) < 1e-12
                assert abs(vg - src[2]) < 1e-12


# ------------------------------------------------ moving wall ghost kinematics --
@pytest.mark.parametrize("viscous", [False, True])
def test_pitching_wall_ghosts_satisfy_the_wall_condition(viscous):
    """Wall readings (slip: relative normal velocity reflected; no-slip:
    u_g = 2 v_wall - u) on a rigidly pitching O-grid.  Each ghost layer and
    its mirror cell average to the wall's own velocity: the normal component
    (slip) or the whole vector (no-slip) equals the velocity of the rotated
    face midpoint, taken here as a central difference in time of the rigid
    rotation x(t) = pivot + R(A sin(omega t)) (x - pivot), independent of the
    oracle's grid-velocity formula; the slip wall keeps the tangential
    velocity.  Every snapshot of N_H = 2, at each of which the pitch rate is
    nonzero."""
    cs = C.ogrid(32, 8, n_harm=2, viscous=viscous, pitch_deg=3.0, radius=5.0)
    o = Oracle(cs)
    rng = np.random.default_rng(4)
    U = np.zeros(o.size)
    blk = o.block_view(U, 0)
    sh = blk[:, 0].shape
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, sh)
    u = cs.mach + 0.05 * rng.uniform(-1, 1, sh)
    v = 0.05 * rng.uniform(-1, 1, sh)
    p = (1.0 / G) * (1.0 + 0.05 * rng.uniform(-1, 1, sh))
    blk[:, 0], blk[:, 1], blk[:, 2] = rho, rho * u, rho * v
    blk[:, 3] = p / (G - 1) + 0.5 * rho * (u * u + v * v)
    Fv = o.block_view(o.fill_ghosts(U), 0)[:, :, 0]            # [n][v][j][i], padded
    _, _, g = o.blocks[0]
    nodes = cs.blocks[0].nodes                                   # [j][i][2], 2 ghost layers
    A, w, ns = math.radians(cs.pitch_amp_deg), cs.omega, cs.n_snap
    piv = np.array(cs.pivot)

    def place(x, t):
        th = A * math.sin(w * t)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        return piv + R @ (x - piv)

    def vel(n, i, j):
        return Fv[n, 1:3, j, i] / Fv[n, 0, j, i]

    h = 1e-5
    for n in range(ns):
        t = 2 * math.pi * n / (ns * w)
        for i in range(cs.blocks[0].n[0]):
            x0, x1 = nodes[2, 2 + i], nodes[2, 3 + i]
            xm = 0.5 * (x0 + x1)
            vw = (place(xm, t + h) - place(xm, t - h)) / (2 * h)
            e = place(x1, t) - place(x0, t)
            nrm = np.array([e[1], -e[0]]) / np.linalg.norm(e)
            tan = e / np.linalg.norm(e)
            for layer in (1, 2):                                  # ghost g1-layer mirrors cell g1+layer-1
                ug = vel(n, g[0] + i, g[1] - layer)
                ui = vel(n, g[0] + i, g[1] + layer - 1)
                mean = 0.5 * (ug + ui)
                assert abs((mean - vw) @ nrm) < 1e-9, (n, i, layer)
                if viscous:
                    assert np.abs(mean - vw).max() < 1e-9, (n, i, layer)
                else:
                    assert abs((ug - ui) @ tan) < 1e-12, (n, i, layer)


def test_viscous_flux_of_a_linear_velocity_field_is_exact_on_an_affine_grid_3d():
    """The 3D form of the linear-field pin above: parallelepiped cells (an
    affine map of a uniform lattice, ghosts point-reflected), u = u0 + A x
    with a full 3x3 A, uniform density and pressure: the viscous part of each
    interior residual is zero in mass and momentum and -V tau : A in energy,
    tau = mu (A + A^T - 2/3 tr(A) I)."""
    ni, nj, nk = 10, 9, 8
    Z, Y, X = np.meshgrid(np.linspace(0, 1, nk + 1), np.linspace(0, 1, nj + 1), np.linspace(0, 1.2, ni + 1),
                          indexing="ij")
    M = np.array([[1.0, 0.2, 0.1], [0.05, 1.0, 0.15], [0.1, -0.1, 1.0]])
    gn = np.einsum("ab,kjib->kjia", M, np.stack([X, Y, Z], axis=-1))
    ext = C.extend_ghost_nodes(gn, 3, (False, False, False))
    side_bc = {(d, s): (C.BC_FARFIELD, -1) for d in range(3) for s in range(2)}

    def case(viscous):
        bl, cuts, bcs = C.split_blocks(ext, 3, (ni, nj, nk), (False, False, False), side_bc,
                                       [C.BlockSpec((0, 0, 0), (ni, nj, nk))])
        return C.Case(name="affine_box", dim=3, n_harm=0, mach=0.3, omega=0.1, viscous=viscous,
                      blocks=bl, cuts=cuts, bcs=bcs, n_bodies=0, seed=1)

    A = np.array([[0.03, -0.02, 0.01], [0.05, 0.01, -0.04], [-0.02, 0.03, 0.02]])
    u0 = np.array([0.3, 0.0, 0.0])
    on, off = Oracle(case(True)), Oracle(case(False))
    vol, xc, _ = on.geometry(0)
    U = np.zeros(on.size)
    blk = on.block_view(U, 0)
    vel = u0[:, None, None, None] + np.einsum("ab,kjib->akji", A, xc)
    p = 1.0 / G
    blk[0, 0] = 1.0
    blk[0, 1:4] = vel
    blk[0, 4] = p / (G - 1) + 0.5 * (vel ** 2).sum(axis=0)
    Rv = on.interior(on.residual(U, with_scale=False), 0) - off.interior(off.residual(U, with_scale=False), 0)
    mu = 0.3 / 5.0e3
    tau = mu * (A + A.T - 2.0 / 3.0 * np.trace(A) * np.eye(3))
    phi = float(np.sum(tau * A))
    _, _, g = on.blocks[0]
    V = vol[g[2]:g[2] + nk, g[1]:g[1] + nj, g[0]:g[0] + ni]
    inner = (slice(3, nk - 3), slice(3, nj - 3), slice(3, ni - 3))
    scale = mu * np.abs(A).max() * 0.03                          # |tau| |S|, |S| ~ 0.015
    r = Rv[0]
    for q in range(4):
        assert np.abs(r[q][inner]).max() < 1e-9 * scale, q
    np.testing.assert_allclose(r[4][inner], -V[inner] * phi, rtol=1e-8, atol=1e-9 * scale)


# ------------------------------------- unsteady farfield: inlet angle and gust --
def _ff_ghost_checks(Wg, Wi, Winf, nrm):
    """Deviations of a farfield ghost from the characteristic reading, as a
    vector: [R+ of the ghost - R+ of the interior cell, R- of the ghost - R- of
    the freestream, entropy - upwind entropy, tangential velocity - upwind
    tangential velocity (3 comps)].  The upwind side is chosen by the sign of
    the ghost's own normal velocity (outflow: interior, inflow: freestream)."""
    def inv(W):
        rho, vel, p = W[0], np.asarray(W[1:4]), W[4]
        q = vel @ nrm
        c = math.sqrt(G * p / rho)
        return q + 2 * c / (G - 1), q - 2 * c / (G - 1), p / rho ** G, vel - q * nrm
    gp, gm, gs, gt = inv(Wg)
    ip, _, is_, it = inv(Wi)
    _, fm, fs, ft = inv(Winf)
    up_s, up_t = (is_, it) if (np.asarray(Wg[1:4]) @ nrm) > 0 else (fs, ft)
    return np.concatenate([[gp - ip, gm - fm, gs - up_s], gt - up_t])


def _prim5(Uc, dim):
    rho = Uc[0]
    vel = np.zeros(3)
    vel[:dim] = Uc[1:1 + dim] / rho
    p = (G - 1) * (Uc[dim + 1] - 0.5 * rho * vel @ vel)
    return np.array([rho, *vel, p])


def _random_state_around(o, cs, rng, u0, amp=0.05):
    U = np.zeros(o.size)
    for b in range(len(cs.blocks)):
        blk = o.block_view(U, b)
        sh = blk[:, 0].shape
        rho = 1.0 + amp * rng.uniform(-1, 1, sh)
        vel = [u0[a] + amp * rng.uniform(-1, 1, sh) for a in range(cs.dim)]
        p = (1.0 / G) * (1.0 + amp * rng.uniform(-1, 1, sh))
        blk[:, 0] = rho
        for a in range(cs.dim):
            blk[:, 1 + a] = rho * vel[a]
        blk[:, cs.dim + 1] = p / (G - 1) + 0.5 * rho * sum(v * v for v in vel)
    return U


def _channel_inflow_freestream(cs, n, mutation=None):
    """Freestream of snapshot n of the 2D channel workload, written from the
    workload's statement: inlet angle alpha(t) = 2 deg * sin(omega t) with
    omega from reduced frequency 0.1 on the unit height (omega = 0.2 M),
    t_n = 2 pi n / (N_s omega); rho = 1, c = 1, |u| = M."""
    M = cs.mach
    w = 0.2 * M
    t = 2 * math.pi * n / (cs.n_snap * w)
    amp = math.radians(2.0)
    if mutation == "deg_as_rad":
        amp = 2.0
    elif mutation == "amplitude":
        amp = math.radians(2.0) * 1.5
    elif mutation == "phase_sign":
        t = -t
    a = amp * math.sin(w * t)
    return np.array([1.0, M * math.cos(a), M * math.sin(a), 0.0, 1.0 / G])


def _channel_farfield_deviation(mutation=None):
    cs = C.channel(24, 8, n_harm=2)
    o = Oracle(cs)
    U = _random_state_around(o, cs, np.random.default_rng(13), (cs.mach, 0.0))
    F = o.block_view(o.fill_ghosts(U), 0)[:, :, 0]              # [n][v][j][i], padded
    _, _, g = o.blocks[0]
    ni, nj = cs.blocks[0].n[0], cs.blocks[0].n[1]
    worst = 0.0
    for n in range(cs.n_snap):
        Winf = _channel_inflow_freestream(cs, n, mutation)
        for j in range(g[1], g[1] + nj):
            for side, nx in ((0, -1.0), (1, 1.0)):                 # x = 0 and x = 2 are straight
                i_in = g[0] if side == 0 else g[0] + ni - 1
                ghosts = (g[0] - 1, g[0] - 2) if side == 0 else (g[0] + ni, g[0] + ni + 1)
                Wi = _prim5(F[n, :, j, i_in], 2)
                for ig in ghosts:
                    dev = _ff_ghost_checks(_prim5(F[n, :, j, ig], 2), Wi, Winf, np.array([nx, 0.0, 0.0]))
                    worst = max(worst, np.abs(dev).max())
    return worst


def test_unsteady_inlet_angle_farfield_ghosts():
    """Channel workload (inlet angle 2 deg sin(omega t), Mach 0.5, reduced
    frequency 0.1 on the height): at every snapshot of N_H = 2 the farfield
    ghosts at inlet and outlet carry the freestream's incoming invariant, and
    on inflow its entropy and tangential velocity, of the inflow angle of that
    snapshot.  The expected freestream is computed here from the workload's
    statement, not by the oracle."""
    assert _channel_farfield_deviation() < 1e-12


@pytest.mark.parametrize("mutation", ["deg_as_rad", "amplitude", "phase_sign"])
def test_unsteady_inlet_angle_pin_detects_planted_mistakes(mutation):
    """The same check against a freestream carrying a plausible mistake (the
    2 deg amplitude read as radians, a wrong amplitude, the time phase with
    the wrong sign) fails by far: the pin separates them from the reading."""
    assert _channel_farfield_deviation(mutation) > 1e-4


def _box_gust_freestream(cs, n, xf, mutation=None):
    """Freestream of snapshot n of the 3D box workload at a point with
    x-coordinate xf: a convected vertical gust v' = 0.02 M sin(omega t -
    omega x / M) on the uniform stream (M, 0, 0); omega = 0.2 M."""
    M = cs.mach
    w = 0.2 * M
    t = 2 * math.pi * n / (cs.n_snap * w)
    amp = 0.02 * M
    ph = w * t - w * xf / M
    if mutation == "amplitude":
        amp = 0.02
    elif mutation == "phase_sign":
        ph = w * t + w * xf / M
    elif mutation == "deg_as_rad":
        ph = math.radians(ph)
    return np.array([1.0, M, amp * math.sin(ph), 0.0, 1.0 / G])


def _box_farfield_deviation(mutation=None):
    cs = C.box3d(8, 6, 4, n_harm=2)
    o = Oracle(cs)
    U = _random_state_around(o, cs, np.random.default_rng(14), (cs.mach, 0.0, 0.0), amp=0.004)
    F = o.block_view(o.fill_ghosts(U), 0)                       # [n][v][k][j][i], padded
    _, _, g = o.blocks[0]
    ni, nj, nk = cs.blocks[0].n
    X = cs.blocks[0].nodes                                       # [k][j][i][3], 2 ghost layers
    worst = 0.0
    for n in range(cs.n_snap):
        for k in range(nk):
            kk = g[2] + k
            # x-min and x-max faces (straight planes x = 0 and x = 4)
            for j in range(nj):
                jj = g[1] + j
                for side, nx in ((0, -1.0), (1, 1.0)):
                    a = 2 if side == 0 else 2 + ni                 # node index of the face plane
                    xf = X[2 + k:4 + k, 2 + j:4 + j, a, 0].mean()
                    Winf = _box_gust_freestream(cs, n, xf, mutation)
                    i_in = g[0] if side == 0 else g[0] + ni - 1
                    Wi = _prim5(F[n, :, kk, jj, i_in], 3)
                    for ig in ((g[0] - 1, g[0] - 2) if side == 0 else (g[0] + ni, g[0] + ni + 1)):
                        dev = _ff_ghost_checks(_prim5(F[n, :, kk, jj, ig], 3), Wi, Winf,
                                               np.array([nx, 0.0, 0.0]))
                        worst = max(worst, np.abs(dev).max())
            # y-max face (the plane y = 1), normal +y: the gust is the normal velocity
            for i in range(ni):
                ii = g[0] + i
                xf = X[2 + k:4 + k, 2 + nj, 2 + i:4 + i, 0].mean()
                Winf = _box_gust_freestream(cs, n, xf, mutation)
                Wi = _prim5(F[n, :, kk, g[1] + nj - 1, ii], 3)
                for jg in (g[1] + nj, g[1] + nj + 1):
                    dev = _ff_ghost_checks(_prim5(F[n, :, kk, jg, ii], 3), Wi, Winf, np.array([0.0, 1.0, 0.0]))
                    worst = max(worst, np.abs(dev).max())
    return worst


def test_convected_gust_farfield_ghosts():
    """3D box workload (vertical gust 0.02 M sin(omega t - omega x / M) at the
    farfield, Mach 0.3, omega = 0.2 M): at every snapshot of N_H = 2 the
    ghosts at x = 0, x = 4 and y = 1 carry the incoming invariant of the gusty
    freestream at the face centroid, and on inflow its entropy and tangential
    velocity; expected values from the workload's statement."""
    assert _box_farfield_deviation() < 1e-12


@pytest.mark.parametrize("mutation", ["deg_as_rad", "amplitude", "phase_sign"])
def test_convected_gust_pin_detects_planted_mistakes(mutation):
    """Gust amplitude without the factor M, the convective phase with the
    wrong sign, and the phase taken as degrees each fail the check."""
    assert _box_farfield_deviation(mutation) > 1e-5
