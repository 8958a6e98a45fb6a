"""Seeded synthetic workloads for the harmonic-balance (HB) residual.

This module generates the *inputs* of the method and nothing else: structured
grids (node coordinates including two ghost-node layers), their split into
blocks, the cut (block-interface) and boundary-condition tables, the flow
parameters of each workload, and seeded random numbers.  It holds none of the
method's arithmetic (no state, flux, source or time-step formula), so both the
FP64 CPU oracle and the CUDA library consume it without sharing any numerics.

Conventions
-----------
* Index directions d = 0, 1, 2 are (i, j, k).  2D grids have nk = 1 and no k
  ghost layers.
* Arrays are stored with i fastest: node arrays are ``[j, i, comp]`` in 2D and
  ``[k, j, i, comp]`` in 3D; a block of ``ni x nj (x nk)`` cells carries
  ``(ni+5) x (nj+5) (x (nk+5))`` nodes, local node ``a`` in ``[-2, n+3)``.
* A cut row (17 ints) fills the ghost box ``[lo, hi)`` of ``dst_blk`` from
  ``src_blk``: ``src[a] = off[a] + sign[a] * dst[perm[a]]``.  The box lies in
  the ghost layers of exactly one direction ``p`` (its *pass*); along
  directions ``q < p`` it may cover ghost cells (corners), along ``q > p`` it
  stays in the interior.  Sources are interior cells or ghost cells of an
  earlier pass, so filling pass 0, then 1, then 2 gives block corners the
  values a single-block grid would have (the paper's per-RK-step cut
  exchange, Sec. 3.1 "MPI Optimisations").
* A BC row (10 ints): ``blk, face, lo[3], hi[3], type, body``; ``face`` is
  ``2*p + side`` (side 0 = low, 1 = high) and ``lo/hi`` give the tangential
  cell range (ghost-extended along earlier passes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_FARFIELD, BC_SLIP, BC_NOSLIP = 1, 2, 3
UBC_NONE, UBC_INLET_ANGLE, UBC_GUST = 0, 1, 2
MOTION_NONE, MOTION_PITCH = 0, 1

CUT_FIELDS = 17
BC_FIELDS = 10


@dataclass
class Block:
    n: tuple            # (ni, nj, nk); nk = 1 in 2D
    nodes: np.ndarray   # float64, [j, i, 2] (2D) or [k, j, i, 3] (3D), incl. 2 ghost layers


@dataclass
class Case:
    """One HB workload: flow parameters, blocks, cut and BC tables."""
    name: str
    dim: int
    n_harm: int
    mach: float
    omega: float
    viscous: bool = False
    reynolds: float = 5.0e3
    prandtl: float = 0.72
    gamma: float = 1.4
    alpha0_deg: float = 0.0
    cfl: float = 1.5
    lim_eps: float = 1.0e-12
    entropy_frac: float = 0.1
    entropy_fix: bool = True
    motion: int = MOTION_NONE
    pitch_amp_deg: float = 0.0
    pivot: tuple = (0.25, 0.0)
    ubc: int = UBC_NONE
    ubc_amp: float = 0.0
    blocks: list = field(default_factory=list)
    cuts: np.ndarray = None      # int32 [n_cuts, 17]
    bcs: np.ndarray = None       # int32 [n_bcs, 10]
    n_bodies: int = 0
    functag: int = 3
    seed: int = 0

    @property
    def n_snap(self) -> int:
        return 2 * self.n_harm + 1

    @property
    def nv(self) -> int:
        return self.dim + 2

    @property
    def n_cells(self) -> int:
        return int(sum(b.n[0] * b.n[1] * b.n[2] for b in self.blocks))


# --------------------------------------------------------------------------
# ghost-node extension and block split
# --------------------------------------------------------------------------

def _axis(dim: int, d: int) -> int:
    return dim - 1 - d


def extend_ghost_nodes(gn: np.ndarray, dim: int, periodic, period_shift=None) -> np.ndarray:
    """Add two ghost-node layers per direction, direction 0 first.

    Periodic directions wrap (node N is node 0 shifted by ``period_shift[d]``);
    the others point-reflect along the grid line, x(-m) = 2 x(0) - x(m).
    """
    out = np.asarray(gn, dtype=np.float64)
    for d in range(dim):
        ax = _axis(dim, d)
        n = out.shape[ax] - 1
        take = lambda idx: np.take(out, idx, axis=ax)
        if periodic[d]:
            shift = np.zeros(out.shape[-1]) if period_shift is None else np.asarray(period_shift[d], float)
            lo = np.concatenate([take([n - 2]) - shift, take([n - 1]) - shift], axis=ax)
            hi = np.concatenate([take([1]) + shift, take([2]) + shift], axis=ax)
        else:
            x0, xn = take([0]), take([n])
            lo = np.concatenate([2 * x0 - take([2]), 2 * x0 - take([1])], axis=ax)
            hi = np.concatenate([2 * xn - take([n - 1]), 2 * xn - take([n - 2])], axis=ax)
        out = np.concatenate([lo, out, hi], axis=ax)
    return out


@dataclass
class BlockSpec:
    lo: tuple           # global cell origin (I0, J0, K0)
    hi: tuple           # global cell end (exclusive)
    flip: bool = False  # store the block with i and j both reversed


def split_blocks(gn_ext: np.ndarray, dim: int, ncell: tuple, periodic, side_bc: dict,
                 specs: list):
    """Cut a ghost-extended global grid into blocks; build cut and BC tables.

    ``side_bc[(d, side)] = (type, body)`` for every non-periodic global side.
    Returns (blocks, cuts, bcs).
    """
    ncell = tuple(ncell) + (1,) * (3 - len(ncell))
    periodic = tuple(periodic) + (False,) * (3 - len(periodic))
    ng = [2, 2, 2 if dim == 3 else 0]
    owner = -np.ones(ncell[::-1], dtype=np.int64)        # [K, J, I]
    for b, s in enumerate(specs):
        lo = tuple(s.lo) + (0,) * (3 - len(s.lo))
        hi = tuple(s.hi) + (1,) * (3 - len(s.hi))
        sl = owner[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        if (sl >= 0).any():
            raise ValueError("blocks overlap")
        sl[...] = b
    if (owner < 0).any():
        raise ValueError("blocks do not cover the grid")

    los, his, flips, ns = [], [], [], []
    blocks = []
    for s in specs:
        lo = np.array(tuple(s.lo) + (0,) * (3 - len(s.lo)))
        hi = np.array(tuple(s.hi) + (1,) * (3 - len(s.hi)))
        los.append(lo); his.append(hi); flips.append(bool(s.flip)); ns.append(hi - lo)
        sl = [slice(None)] * gn_ext.ndim
        for d in range(dim):
            ax = _axis(dim, d)
            sl[ax] = slice(int(lo[d]), int(hi[d]) + 5)
        nodes = gn_ext[tuple(sl)]
        if s.flip:
            nodes = np.flip(nodes, axis=(_axis(dim, 0), _axis(dim, 1)))
        blocks.append(Block(n=tuple(int(v) for v in (hi - lo)), nodes=np.ascontiguousarray(nodes)))

    def to_global(b, c):                 # c: [m, 3] local cells
        g = c + los[b]
        if flips[b]:
            g = g.copy()
            g[:, 0] = his[b][0] - 1 - c[:, 0]
            g[:, 1] = his[b][1] - 1 - c[:, 1]
        return g

    def to_local(o, g):
        c = g - los[o]
        if flips[o]:
            c = c.copy()
            c[:, 0] = his[o][0] - 1 - g[:, 0]
            c[:, 1] = his[o][1] - 1 - g[:, 1]
        return c

    cuts, bcs = [], []
    for b in range(len(specs)):
        n = ns[b]
        for p in range(dim):
            for side in (0, 1):
                rng = []
                for d in range(3):
                    if d == p:
                        rng.append(np.arange(-2, 0) if side == 0 else np.arange(n[d], n[d] + 2))
                    elif d < p:
                        rng.append(np.arange(-ng[d], n[d] + ng[d]))
                    else:
                        rng.append(np.arange(0, n[d]))
                cc = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
                g = to_global(b, cc)
                out_p = (g[:, p] < 0) | (g[:, p] >= ncell[p])
                if out_p.any() and not periodic[p]:
                    if not out_p.all():
                        raise ValueError("ghost box straddles the domain edge")
                    gside = 0 if g[0, p] < 0 else 1
                    btype, body = side_bc[(p, gside)]
                    lo3, hi3 = cc.min(axis=0), cc.max(axis=0) + 1
                    bcs.append([b, 2 * p + side, *lo3, *hi3, btype, body])
                    continue
                g = g.copy()
                for d in range(3):
                    if periodic[d]:
                        g[:, d] = np.mod(g[:, d], ncell[d])
                gc = g.copy()
                for d in range(p):
                    gc[:, d] = np.clip(gc[:, d], 0, ncell[d] - 1)
                own = owner[gc[:, 2], gc[:, 1], gc[:, 0]]
                for o in np.unique(own):
                    m = own == o
                    dst = cc[m]
                    src = to_local(int(o), g[m])
                    sign = np.array([1 if flips[b] == flips[o] else -1] * 2 + [1])
                    off = src - sign * dst
                    keys, inv = np.unique(off, axis=0, return_inverse=True)
                    for kk in range(len(keys)):
                        dd = dst[inv.reshape(-1) == kk]
                        lo3, hi3 = dd.min(axis=0), dd.max(axis=0) + 1
                        if np.prod(hi3 - lo3) != len(dd):
                            raise ValueError("cut group is not a box")
                        cuts.append([b, int(o), *lo3, *hi3, *keys[kk], 0, 1, 2, *sign])
    return (blocks,
            np.array(cuts, dtype=np.int32).reshape(-1, CUT_FIELDS),
            np.array(bcs, dtype=np.int32).reshape(-1, BC_FIELDS))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def _geometric(n: int, first: float) -> np.ndarray:
    """n+1 points on [0,1] whose spacings grow geometrically from ``first``."""
    if first * n >= 1.0:
        return np.linspace(0.0, 1.0, n + 1)
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        r = 0.5 * (lo + hi)
        s = first * (r ** n - 1.0) / (r - 1.0)
        lo, hi = (r, hi) if s < 1.0 else (lo, r)
    h = first * r ** np.arange(n)
    x = np.concatenate([[0.0], np.cumsum(h)])
    return x / x[-1]


def channel(ni=64, nj=32, n_harm=1, mach=0.5, seed=7, blocks=None, viscous=False,
            name="euler_channel"):
    """2D channel [0,2]x[0,1] on a sinusoidally perturbed grid (amplitude 0.05 of
    the height, seeded phases); farfield inlet/outlet, slip walls; inlet angle
    2 deg * sin(omega t) with reduced frequency 0.1 on the channel height."""
    rng = np.random.default_rng(seed)
    ph1, ph2 = rng.uniform(0.0, 2.0 * np.pi, size=2)
    xi = np.linspace(0.0, 2.0, ni + 1)
    eta = np.linspace(0.0, 1.0, nj + 1)
    X, Y = np.meshgrid(xi, eta)            # [j, i]
    bump = 0.05 * np.sin(np.pi * X / 2.0) * np.sin(np.pi * Y)
    x = X + bump * np.sin(2.0 * np.pi * 2.0 * X / 2.0 + ph1)
    y = Y + bump * np.sin(2.0 * np.pi * 2.0 * Y + ph2)
    gn = np.stack([x, y], axis=-1)
    ext = extend_ghost_nodes(gn, 2, (False, False))
    specs = blocks or [BlockSpec((0, 0), (ni, nj))]
    side_bc = {(0, 0): (BC_FARFIELD, -1), (0, 1): (BC_FARFIELD, -1),
               (1, 0): (BC_SLIP, -1), (1, 1): (BC_SLIP, -1)}
    bl, cuts, bcs = split_blocks(ext, 2, (ni, nj), (False, False), side_bc, specs)
    omega = 2.0 * 0.1 * mach / 1.0
    return Case(name=name, dim=2, n_harm=n_harm, mach=mach, omega=omega, viscous=viscous,
                ubc=UBC_INLET_ANGLE, ubc_amp=2.0, blocks=bl, cuts=cuts, bcs=bcs,
                n_bodies=0, seed=seed)


def naca0012_closed(x):
    """NACA 0012 half-thickness with the closed-trailing-edge coefficient."""
    x = np.clip(x, 0.0, 1.0)
    t = 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)
    return np.maximum(t, 0.0)


def ogrid_nodes(ni: int, nj: int, radius=20.0, first=1.0e-3):
    """O-grid nodes [j, i, 2] around a closed-TE NACA-0012-thickness body.

    i runs clockwise from the trailing edge (lower surface first) so that
    (i, j-outward) is right-handed; node column ni repeats column 0.  Surface
    nodes sit at x = 1 - |sin(beta/2)|: clustered at the leading edge and
    evenly spaced (dx ~ dbeta/2) at the sharp trailing edge.  With that
    spacing the straight grid lines of neighbouring trailing-edge nodes meet
    only ~0.07 c inside the body, so the point-reflected ghost cells (two
    layers of ~1e-3 c) keep positive volumes; a cosine distribution, clustered
    at both ends, makes them meet within 2e-4 c and inverts the ghost cells
    at the trailing edge."""
    beta = -2.0 * np.pi * np.arange(ni + 1) / ni
    xs = 1.0 - np.abs(np.sin(0.5 * beta))
    ys = np.sign(np.sin(beta)) * naca0012_closed(xs)
    xo = 0.5 + radius * np.cos(beta)
    yo = radius * np.sin(beta)
    f = _geometric(nj, first / radius)
    x = xs[None, :] + f[:, None] * (xo - xs)[None, :]
    y = ys[None, :] + f[:, None] * (yo - ys)[None, :]
    x[:, -1] = x[:, 0]
    y[:, -1] = y[:, 0]
    return np.stack([x, y], axis=-1)


def ogrid(ni=1280, nj=192, n_harm=3, mach=0.3, viscous=True, reynolds=5.0e3,
          pitch_deg=3.0, k_red=0.1, specs=None, name="ns_ogrid", seed=8,
          radius=20.0, first=1.0e-3):
    """Pitching O-grid case: no-slip (or slip) wall at j=0, farfield at j=nj,
    periodic wrap in i; rigid pitch about the quarter chord."""
    gn = ogrid_nodes(ni, nj, radius=radius, first=first)
    ext = extend_ghost_nodes(gn, 2, (True, False))
    wall = BC_NOSLIP if viscous else BC_SLIP
    side_bc = {(1, 0): (wall, 0), (1, 1): (BC_FARFIELD, -1)}
    specs = specs or [BlockSpec((0, 0), (ni, nj))]
    bl, cuts, bcs = split_blocks(ext, 2, (ni, nj), (True, False), side_bc, specs)
    omega = 2.0 * k_red * mach
    # pseudo-time CFL 1.0: with 1.5 the explicit scheme diverges on these
    # O-grids, inviscid within ~50-600 iterations and viscous (8 blocks,
    # 1280x192) at iteration 68, identically in FP32 and FP64
    return Case(name=name, dim=2, n_harm=n_harm, mach=mach, omega=omega, viscous=viscous,
                cfl=1.0,
                reynolds=reynolds, motion=MOTION_PITCH if pitch_deg else MOTION_NONE,
                pitch_amp_deg=pitch_deg, blocks=bl, cuts=cuts, bcs=bcs, n_bodies=1, seed=seed)


def ogrid8_specs(ni: int, nj: int):
    """Eight uneven blocks with T-junctions: inner ring (lower 2/3 of j) split
    384/256/384/256 of 1280, outer ring 128/384/384/384 of 1280."""
    inner = [384, 256, 384, 256]
    outer = [128, 384, 384, 384]
    jm = (nj * 2) // 3
    specs = []
    for widths, (j0, j1) in ((inner, (0, jm)), (outer, (jm, nj))):
        cuts = np.round(np.cumsum([0] + widths) * ni / 1280).astype(int)
        for a, b in zip(cuts[:-1], cuts[1:]):
            specs.append(BlockSpec((int(a), j0), (int(b), j1)))
    return specs


def ns_ogrid8(ni=1280, nj=192, n_harm=3, viscous=True, **kw):
    """Multi-block laminar NS pitching-airfoil workload (8 uneven blocks,
    245,760 cells at full size, N_H = 3)."""
    return ogrid(ni=ni, nj=nj, n_harm=n_harm, viscous=viscous,
                 specs=ogrid8_specs(ni, nj), name="ns_ogrid8", **kw)


def block_lattice(ni: int, nj: int, bi: int, bj: int):
    """ni x nj cells cut into a lattice of bi x bj blocks."""
    return [BlockSpec((i, j), (i + bi, j + bj)) for j in range(0, nj, bj) for i in range(0, ni, bi)]


def paper_tc1(ni=1024, nj=256, n_harm=15, **kw):
    """Shape of the paper's first test case (Sec. 4.1): 512 blocks of 32x16
    cells (262,144 cells), 31 snapshots; a pitching wing section, inviscid
    (the synthetic stand-in for the heaving and pitching energy-extraction
    wing, whose grid is not available)."""
    return ogrid(ni=ni, nj=nj, n_harm=n_harm, viscous=False, specs=block_lattice(ni, nj, ni // 32, nj // 16),
                 name="paper_tc1", seed=41, **kw)


def paper_tc2(ni=4096, nj=1024, n_harm=8, **kw):
    """Shape of the paper's second test case (Sec. 4.1): 2048 blocks of
    64x32 cells (4,194,304 cells), 17 snapshots; an inviscid wing section in a
    periodically yawing stream (the synthetic stand-in for the wind-turbine
    blade section in yawed wind: fixed grid, inflow angle varying at the
    fundamental frequency)."""
    cs = ogrid(ni=ni, nj=nj, n_harm=n_harm, viscous=False, pitch_deg=0.0,
               specs=block_lattice(ni, nj, ni // 64, nj // 32), name="paper_tc2", seed=42, **kw)
    cs.ubc, cs.ubc_amp = UBC_INLET_ANGLE, 2.0
    return cs


def adjoint_ogrid4(ni=512, nj=256, n_harm=4, **kw):
    """Adjoint workload: 4 blocks 96/160/128/128 of 512 in i, laminar, N_H = 4."""
    widths = np.round(np.cumsum([0, 96, 160, 128, 128]) * ni / 512).astype(int)
    specs = [BlockSpec((int(a), 0), (int(b), nj)) for a, b in zip(widths[:-1], widths[1:])]
    return ogrid(ni=ni, nj=nj, n_harm=n_harm, viscous=True, specs=specs,
                 name="adjoint_ogrid4", seed=11, **kw)


def batch_cases(n_cases=64, seed=9, scale=(1.0, 16.0), base=(32, 16)):
    """Independent single-block inviscid pitching O-grids: cell counts
    (32s)x(16s), s log-uniform, rounded to multiples of 8; N_H uniform in
    {1..4}; Mach U[0.3,0.7]; pitch amplitude U[1,5] deg; k = 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cases):
        s = math.exp(rng.uniform(math.log(scale[0]), math.log(scale[1])))
        ni = max(8, int(round(base[0] * s / 8.0)) * 8)
        nj = max(8, int(round(base[1] * s / 8.0)) * 8)
        nh = int(rng.integers(1, 5))
        mach = float(rng.uniform(0.3, 0.7))
        amp = float(rng.uniform(1.0, 5.0))
        first = min(1.0e-3 * 16.0 / nj * 8.0, 0.05)
        cs = ogrid(ni=ni, nj=nj, n_harm=nh, mach=mach, viscous=False, pitch_deg=amp,
                   name=f"batch{c:02d}", seed=seed * 1000 + c, first=first)
        out.append(cs)
    return out


def box3d(ni=256, nj=128, nk=64, n_harm=2, mach=0.3, reynolds=5.0e3, ratio=1.05,
          seed=10, gust=0.02, name="ns_box3d", specs=None):
    """3D box [0,4]x[0,1]x[0,1], geometric stretching towards the y=0 no-slip
    wall, smooth seeded interior node perturbation, farfield with a convected
    vertical gust at x-min, x-max and y-max, periodic in z."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(0.0, 4.0, ni + 1)
    h0 = (ratio - 1.0) / (ratio ** nj - 1.0)
    ys = np.concatenate([[0.0], np.cumsum(h0 * ratio ** np.arange(nj))])
    ys /= ys[-1]
    zs = np.linspace(0.0, 1.0, nk + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")    # [k, j, i]
    ph = rng.uniform(0.0, 2.0 * np.pi, size=3)
    env = np.sin(np.pi * X / 4.0) * np.sin(np.pi * Y)
    dy = np.gradient(ys)[None, :, None] * np.ones_like(Y)
    amp = 0.15 * np.minimum(np.minimum(dy, 4.0 / ni), 1.0 / nk)
    x = X + amp * env * np.sin(2 * np.pi * Y + ph[0])
    y = Y + amp * env * np.sin(2 * np.pi * X / 4.0 + ph[1])
    z = Z + amp * env * np.sin(2 * np.pi * X / 4.0 + 2 * np.pi * Y + ph[2])
    gn = np.stack([x, y, z], axis=-1)
    shift = [None, None, np.array([0.0, 0.0, 1.0])]
    ext = extend_ghost_nodes(gn, 3, (False, False, True), period_shift=shift)
    side_bc = {(0, 0): (BC_FARFIELD, -1), (0, 1): (BC_FARFIELD, -1),
               (1, 0): (BC_NOSLIP, -1), (1, 1): (BC_FARFIELD, -1)}
    specs = specs or [BlockSpec((0, 0, 0), (ni, nj, nk))]
    bl, cuts, bcs = split_blocks(ext, 3, (ni, nj, nk), (False, False, True), side_bc, specs)
    return Case(name=name, dim=3, n_harm=n_harm, mach=mach, omega=2.0 * 0.1 * mach,
                viscous=True, reynolds=reynolds, ubc=UBC_GUST, ubc_amp=gust,
                blocks=bl, cuts=cuts, bcs=bcs, n_bodies=0, seed=seed)


def periodic_box2d(ni=16, nj=12, n_harm=1, mach=0.4, viscous=False, seed=5, specs=None,
                   name="periodic_box2d", perturb=0.04):
    """Doubly periodic unit square with a smooth seeded node perturbation that
    vanishes on the period boundaries: a domain without physical boundaries."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=2)
    X, Y = np.meshgrid(np.linspace(0.0, 1.0, ni + 1), np.linspace(0.0, 1.0, nj + 1))
    env = perturb * np.sin(np.pi * X) * np.sin(np.pi * Y)
    gn = np.stack([X + env * np.sin(2 * np.pi * Y + ph[0]), Y + env * np.sin(2 * np.pi * X + ph[1])], -1)
    ext = extend_ghost_nodes(gn, 2, (True, True), period_shift=[np.array([1.0, 0.0]), np.array([0.0, 1.0])])
    specs = specs or [BlockSpec((0, 0), (ni, nj))]
    bl, cuts, bcs = split_blocks(ext, 2, (ni, nj), (True, True), {}, specs)
    return Case(name=name, dim=2, n_harm=n_harm, mach=mach, omega=2.0 * 0.1 * mach,
                viscous=viscous, reynolds=200.0, blocks=bl, cuts=cuts, bcs=bcs, n_bodies=0, seed=seed)


def noise(case: Case, seed: int | None = None) -> np.ndarray:
    """Uniform [-1, 1] numbers, one per interior (block, snapshot, var, cell),
    packed block after block as [n][v][k][j][i] (i fastest)."""
    rng = np.random.default_rng(case.seed if seed is None else seed)
    total = case.n_cells * case.n_snap * case.nv
    return rng.uniform(-1.0, 1.0, size=total)


def interior_count(case: Case) -> int:
    return case.n_cells * case.n_snap * case.nv


def sample_cells(case: Case, count: int, seed: int) -> np.ndarray:
    """Seeded interior cells [count, 4] = (block, i, j, k)."""
    rng = np.random.default_rng(seed)
    w = np.array([b.n[0] * b.n[1] * b.n[2] for b in case.blocks], dtype=float)
    out = []
    for _ in range(count):
        b = int(rng.choice(len(w), p=w / w.sum()))
        n = case.blocks[b].n
        out.append([b, int(rng.integers(n[0])), int(rng.integers(n[1])), int(rng.integers(n[2]))])
    return np.array(out, dtype=np.int32)


CONFIGS = {
    "euler_channel": lambda: channel(),
    "ns_ogrid8": lambda: ns_ogrid8(),
    "ns_box3d": lambda: box3d(),
    "adjoint_ogrid4": lambda: adjoint_ogrid4(),
}
