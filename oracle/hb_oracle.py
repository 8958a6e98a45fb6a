"""ctypes marshalling for the C++ FP64 oracle (``hb_oracle.cpp``).

Test infrastructure only (see the package docstring).  Every function here
converts a :class:`paper_1304_7654_gb300.cases.Case` or numpy arrays into the
oracle's flat C arguments; all arithmetic happens in ``hb_oracle.cpp``.

State layout of the oracle: per block ``[n][v][k][j][i]`` over the padded cell
range (two ghost layers per in-plane direction, none along k in 2D), blocks one
after another.  ``unpack``/``pack`` convert to and from the compact interior
layout ``[block][n][v][k][j][i]`` used by the tests.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hb_oracle.cpp")
_LIB = os.path.join(_HERE, "libhb_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libhb_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


def _compile(lib: str, extra, force: bool) -> str:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", *extra,
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no GPU, no CUDA)."""
    return _compile(_LIB, [], force)


def build_openmp(force: bool = False) -> str:
    """Compile the same source with OpenMP (libhb_oracle_omp.so), used only to
    time the oracle on all host cores; its results equal the plain build's
    bit for bit."""
    return _compile(_LIB_OMP, ["-fopenmp"], force)


def _load(openmp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if openmp else _lib) is None:
            lib = ct.CDLL(build_openmp() if openmp else build())
            lib.orc_create.restype = ct.c_void_p
            lib.orc_create.argtypes = [ct.c_int, ct.c_int, _dp, ct.c_int, _ip, _dp, ct.c_int, _ip,
                                       ct.c_int, _ip]
            lib.orc_destroy.argtypes = [ct.c_void_p]
            lib.orc_state_size.restype = ct.c_int64
            lib.orc_state_size.argtypes = [ct.c_void_p]
            lib.orc_block_info.argtypes = [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int64), _ip, _ip]
            lib.orc_geometry.argtypes = [ct.c_void_p, ct.c_int, _dp, _dp, _dp]
            lib.orc_init_state.argtypes = [ct.c_void_p, _dp, ct.c_double, _dp]
            lib.orc_fill_ghosts.argtypes = [ct.c_void_p, _dp]
            lib.orc_residual.argtypes = [ct.c_void_p, _dp, _dp, _dp]
            lib.orc_residual_cells.argtypes = [ct.c_void_p, _dp, ct.c_int, _ip, _dp, _dp]
            lib.orc_time_step.argtypes = [ct.c_void_p, _dp, _dp]
            lib.orc_rk_smooth.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp]
            lib.orc_rk_smooth_threads.argtypes = [ct.c_void_p, _dp, ct.c_int, _dp, ct.c_int]
            lib.orc_halo_pass.argtypes = [ct.c_void_p, _dp, ct.c_int]
            lib.orc_rk_stage.argtypes = [ct.c_void_p, _dp, _dp, _dp, ct.c_int, _dp]
            lib.orc_openmp_threads.restype = ct.c_int
            lib.orc_forces.argtypes = [ct.c_void_p, _dp, _dp, _dp]
            lib.orc_td_residual.argtypes = [ct.c_void_p, _dp, _dp, _dp, ct.c_double, ct.c_double, _dp]
            lib.orc_td_step.argtypes = [ct.c_void_p, _dp, _dp, _dp, ct.c_double, ct.c_double, ct.c_int, _dp]
            lib.orc_td_forces.argtypes = [ct.c_void_p, _dp, ct.c_double, _dp, _dp]
            lib.orc_adjoint_columns.argtypes = [ct.c_void_p, _dp, _dp, ct.c_double, ct.c_int, _ip,
                                                _dp, ct.c_int, ct.c_double]
            lib.orc_d_matrix.argtypes = [ct.c_int, _dp]
            lib.orc_van_albada.restype = ct.c_double
            lib.orc_van_albada.argtypes = [ct.c_double, ct.c_double, ct.c_double]
            lib.orc_roe_flux.argtypes = [ct.c_int, _dp, _dp, _dp, _dp, _dp, ct.c_int, _dp]
            if openmp:
                _lib_omp = lib
            else:
                _lib = lib
    return _lib_omp if openmp else _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def d_matrix(ns: int) -> np.ndarray:
    D = np.zeros((ns, ns))
    _load().orc_d_matrix(ns, _d(D))
    return D


def van_albada(a: float, b: float, eps: float = 1e-12) -> float:
    return _load().orc_van_albada(float(a), float(b), float(eps))


def roe_flux(WL, WR, S, vg=(0.0, 0.0, 0.0), dim=2, gamma=1.4, entropy_fix=True,
             entropy_frac=0.1, mode=0) -> np.ndarray:
    """5-component (mass, mx, my, mz, energy) Roe flux through area vector S."""
    prm = _f64([gamma, 1.0 if entropy_fix else 0.0, entropy_frac])
    F = np.zeros(5)
    wl, wr = _f64(WL), _f64(WR)
    s3 = _f64(list(S) + [0.0] * (3 - len(S)))
    v3 = _f64(list(vg) + [0.0] * (3 - len(vg)))
    _load().orc_roe_flux(dim, _d(prm), _d(wl), _d(wr), _d(s3), _d(v3), int(mode), _d(F))
    return F


def case_params(case) -> np.ndarray:
    return _f64([case.gamma, case.prandtl, case.mach, case.reynolds, case.alpha0_deg, case.omega,
                 case.cfl, case.lim_eps, case.entropy_frac, 1.0 if case.viscous else 0.0,
                 1.0 if case.entropy_fix else 0.0, case.motion, case.pitch_amp_deg,
                 case.pivot[0], case.pivot[1], case.ubc, case.ubc_amp, case.n_bodies,
                 case.functag, 0.0])


class Oracle:
    """One case loaded into the oracle."""

    def __init__(self, case, openmp: bool = False):
        """openmp=True loads the OpenMP build (for timing on all host cores)."""
        lib = _load(openmp)
        self.case = case
        self.lib = lib
        dims = np.array([b.n for b in case.blocks], dtype=np.int32).reshape(-1)
        nodes = np.concatenate([_f64(b.nodes).reshape(-1) for b in case.blocks])
        cuts = np.ascontiguousarray(case.cuts, dtype=np.int32).reshape(-1)
        bcs = np.ascontiguousarray(case.bcs, dtype=np.int32).reshape(-1)
        if cuts.size == 0:
            cuts = np.zeros(17, dtype=np.int32)
        if bcs.size == 0:
            bcs = np.zeros(10, dtype=np.int32)
        self._keep = (dims, nodes, cuts, bcs)
        self.h = lib.orc_create(case.dim, case.n_harm, _d(case_params(case)), len(case.blocks),
                                _i(dims), _d(nodes), len(case.cuts), _i(cuts), len(case.bcs),
                                _i(bcs))
        self.size = int(lib.orc_state_size(self.h))
        self.ns, self.nv = case.n_snap, case.nv
        self.blocks = []
        for b in range(len(case.blocks)):
            off = ct.c_int64()
            p = np.zeros(3, dtype=np.int32)
            g = np.zeros(3, dtype=np.int32)
            lib.orc_block_info(self.h, b, ct.byref(off), _i(p), _i(g))
            self.blocks.append((int(off.value), tuple(int(x) for x in p), tuple(int(x) for x in g)))

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # ---- layout helpers -------------------------------------------------
    def block_view(self, U, b):
        """[n][v][k][j][i] view of block b over its padded cells."""
        off, p, _ = self.blocks[b]
        size = self.ns * self.nv * p[0] * p[1] * p[2]
        return U[off:off + size].reshape(self.ns, self.nv, p[2], p[1], p[0])

    def interior(self, U, b):
        _, p, g = self.blocks[b]
        n = self.case.blocks[b].n
        v = self.block_view(U, b)
        return v[:, :, g[2]:g[2] + n[2], g[1]:g[1] + n[1], g[0]:g[0] + n[0]]

    def unpack(self, U) -> np.ndarray:
        """Compact interior layout [block][n][v][k][j][i], flattened."""
        return np.concatenate([self.interior(U, b).reshape(-1) for b in range(len(self.blocks))])

    def pack(self, flat) -> np.ndarray:
        U = np.zeros(self.size)
        o = 0
        for b in range(len(self.blocks)):
            t = self.interior(U, b)
            t[...] = np.asarray(flat[o:o + t.size]).reshape(t.shape)
            o += t.size
        return U

    # ---- method steps ---------------------------------------------------
    def geometry(self, b):
        _, p, _ = self.blocks[b]
        nc = p[0] * p[1] * p[2]
        vol, xc, S = np.zeros(nc), np.zeros(3 * nc), np.zeros(9 * nc)
        self.lib.orc_geometry(self.h, b, _d(vol), _d(xc), _d(S))
        sh = (p[2], p[1], p[0])
        return vol.reshape(sh), xc.reshape(sh + (3,)), S.reshape((3,) + sh + (3,))

    def init_state(self, noise, amp=0.01) -> np.ndarray:
        U = np.zeros(self.size)
        z = _f64(noise)
        self.lib.orc_init_state(self.h, _d(z), float(amp), _d(U))
        return U

    def fill_ghosts(self, U) -> np.ndarray:
        U = _f64(U).copy()
        self.lib.orc_fill_ghosts(self.h, _d(U))
        return U

    def residual(self, U, with_scale=True):
        U = _f64(U)
        R = np.zeros(self.size)
        sc = np.zeros(self.size) if with_scale else None
        self.lib.orc_residual(self.h, _d(U), _d(R), _d(sc) if with_scale else None)
        return (R, sc) if with_scale else R

    def residual_cells(self, U, cells):
        U = _f64(U)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        m = len(cells)
        R = np.zeros((m, self.ns, self.nv))
        sc = np.zeros((m, self.ns, self.nv))
        self.lib.orc_residual_cells(self.h, _d(U), m, _i(cells), _d(R), _d(sc))
        return R, sc

    def time_step(self, U) -> np.ndarray:
        U = _f64(U)
        dt = np.zeros(self.size)
        self.lib.orc_time_step(self.h, _d(U), _d(dt))
        return dt

    def rk_smooth(self, U, n_iter):
        U = _f64(U).copy()
        norms = np.zeros((max(n_iter, 1), self.nv))
        self.lib.orc_rk_smooth(self.h, _d(U), int(n_iter), _d(norms))
        return U, norms[:n_iter]

    def rk_smooth_threads(self, U, n_iter, threads):
        """rk_smooth with the residual sweeps on `threads` threads (OpenMP build
        only; bit for bit the single-thread result)."""
        U = _f64(U).copy()
        norms = np.zeros((max(n_iter, 1), self.nv))
        self.lib.orc_rk_smooth_threads(self.h, _d(U), int(n_iter), _d(norms), int(threads))
        return U, norms[:n_iter]

    def halo_pass(self, U, p):
        """One pass of the ghost fill in place on U (float64 array of the
        oracle layout); cuts with source block -1 are left alone."""
        assert U.dtype == np.float64 and U.flags.c_contiguous and U.size == self.size
        self.lib.orc_halo_pass(self.h, _d(U), int(p))

    def rk_stage(self, Uin, U0, Uout, stage, sums=None):
        """One RK stage out of place, Uin's ghosts as given; at stage 0 the
        sums of (R/V)^2 per variable into sums (nv doubles) if given."""
        for a in (Uin, U0, Uout):
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.size
        self.lib.orc_rk_stage(self.h, _d(Uin), _d(U0), _d(Uout), int(stage),
                              _d(sums) if sums is not None else None)

    def openmp_threads(self) -> int:
        return int(self.lib.orc_openmp_threads())

    def forces(self, U):
        U = _f64(U)
        nb = max(self.case.n_bodies, 1)
        coef = np.zeros((self.ns, nb, 3))
        J = ct.c_double()
        self.lib.orc_forces(self.h, _d(U), _d(coef), ct.byref(J))
        return coef[:, :self.case.n_bodies], float(J.value)

    # ---- time-domain dual time stepping (cases with n_harm = 0)
    def td_residual(self, U, Un, Unm1, t, dt):
        """R*(U) = R(U; t) + V (a0 U + a1 U^n + a2 U^(n-1)) / dt (BDF2, or BDF1
        when Unm1 is None), interior entries."""
        assert self.ns == 1, "time-domain stepping needs a one-snapshot case"
        U, Un = _f64(U), _f64(Un)
        R = np.zeros(self.size)
        self.lib.orc_td_residual(self.h, _d(U), _d(Un), None if Unm1 is None else _d(_f64(Unm1)),
                                 float(t), float(dt), _d(R))
        return R

    def td_step(self, U, Un, Unm1, t, dt, n_inner):
        """n_inner pseudo-time RK iterations of R*(U) = 0 at time t."""
        assert self.ns == 1, "time-domain stepping needs a one-snapshot case"
        U = _f64(U).copy()
        norms = np.zeros((max(n_inner, 1), self.nv))
        self.lib.orc_td_step(self.h, _d(U), _d(_f64(Un)), None if Unm1 is None else _d(_f64(Unm1)),
                             float(t), float(dt), int(n_inner), _d(norms))
        return U, norms[:n_inner]

    def td_forces(self, U, t):
        U = _f64(U)
        nb = max(self.case.n_bodies, 1)
        coef = np.zeros((1, nb, 3))
        J = ct.c_double()
        self.lib.orc_td_forces(self.h, _d(U), float(t), _d(coef), ct.byref(J))
        return coef[:, :self.case.n_bodies], float(J.value)

    def adjoint_columns(self, U, psi, J_seed, cols, mode=0, h=1e-7) -> np.ndarray:
        """d/dU_col [psi . R(U) + J_seed * J(U)] for cols (b, i, j, k, v, n)."""
        U, psi = _f64(U), _f64(psi)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.zeros(len(cols))
        self.lib.orc_adjoint_columns(self.h, _d(U), _d(psi), float(J_seed), len(cols), _i(cols),
                                     _d(out), int(mode), float(h))
        return out
