"""Thin Python binding of libhb.so (include/hb.h): argument marshalling only.

PyTorch supplies device memory and the current stream; every step of the
residual path runs in the library's CUDA kernels.  There is no fallback: if
``libhb.so`` is missing or CUDA is unavailable the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "hb.h")

HB_OK, HB_ERR_INVALID_ARG, HB_ERR_UNSUPPORTED, HB_ERR_CUDA = 0, 1, 2, 3
HB_ERR_NONFINITE, HB_ERR_TIMEOUT, HB_ERR_OOM = 4, 5, 6
HB_FP64, HB_FP32 = 0, 1
STATUS_NAMES = {0: "HB_OK", 1: "HB_ERR_INVALID_ARG", 2: "HB_ERR_UNSUPPORTED", 3: "HB_ERR_CUDA",
                4: "HB_ERR_NONFINITE", 5: "HB_ERR_TIMEOUT", 6: "HB_ERR_OOM"}


class HBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class HbBlockDesc(ct.Structure):
    _fields_ = [("ni", ct.c_int), ("nj", ct.c_int), ("nk", ct.c_int),
                ("nodes", ct.POINTER(ct.c_double))]


class HbCutDesc(ct.Structure):
    _fields_ = [("dst_blk", ct.c_int), ("src_blk", ct.c_int), ("lo", ct.c_int * 3),
                ("hi", ct.c_int * 3), ("off", ct.c_int * 3), ("perm", ct.c_int * 3),
                ("sign", ct.c_int * 3)]


class HbBcDesc(ct.Structure):
    _fields_ = [("blk", ct.c_int), ("face", ct.c_int), ("lo", ct.c_int * 3), ("hi", ct.c_int * 3),
                ("type", ct.c_int), ("body", ct.c_int)]


class HbCaseDesc(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("n_harm", ct.c_int),
                ("mach", ct.c_double), ("reynolds", ct.c_double), ("prandtl", ct.c_double),
                ("gamma", ct.c_double), ("alpha0_deg", ct.c_double), ("omega", ct.c_double),
                ("cfl", ct.c_double), ("lim_eps", ct.c_double), ("entropy_frac", ct.c_double),
                ("viscous", ct.c_int), ("entropy_fix", ct.c_int),
                ("motion", ct.c_int), ("pitch_amp_deg", ct.c_double), ("pivot", ct.c_double * 2),
                ("ubc", ct.c_int), ("ubc_amp", ct.c_double),
                ("n_blocks", ct.c_int), ("blocks", ct.POINTER(HbBlockDesc)),
                ("n_cuts", ct.c_int), ("cuts", ct.POINTER(HbCutDesc)),
                ("n_bcs", ct.c_int), ("bcs", ct.POINTER(HbBcDesc)),
                ("n_bodies", ct.c_int), ("functag", ct.c_int), ("prec", ct.c_int)]


_lib = None
_vp = ct.c_void_p
_dp = ct.POINTER(ct.c_double)


def declared_functions():
    """Names of the functions declared in include/hb.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hb_[a-z_0-9]+)\s*\(", txt)))


def load(path: str | None = None):
    """Load libhb.so; raise if it is not built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libhb.so not found at {p}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ct.CDLL(p)
    lib.hb_create.argtypes = [ct.POINTER(HbCaseDesc), ct.POINTER(_vp)]
    lib.hb_create_batch.argtypes = [ct.POINTER(HbCaseDesc), ct.c_int, ct.POINTER(_vp)]
    lib.hb_destroy.argtypes = [_vp]
    lib.hb_state_size.restype = ct.c_int64
    lib.hb_state_size.argtypes = [_vp]
    lib.hb_state_layout.argtypes = [_vp, ct.c_int, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                    ct.POINTER(ct.c_int)]
    lib.hb_init_state.argtypes = [_vp, _vp, _vp, ct.c_double, _vp]
    lib.hb_exchange_halos.argtypes = [_vp, _vp, _vp]
    lib.hb_residual.argtypes = [_vp, _vp, _vp, _vp]
    lib.hb_rk_smooth.argtypes = [_vp, _vp, ct.c_int, _vp, _vp]
    lib.hb_forces.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.hb_adjoint_residual.argtypes = [_vp, _vp, _vp, ct.c_double, _vp, _vp, _vp]
    lib.hb_sync_status.argtypes = [_vp, _vp]
    lib.hb_set_timing.argtypes = [_vp, ct.c_int]
    lib.hb_autotune.argtypes = [_vp, _vp, ct.c_int, _vp]
    lib.hb_set_tuning.argtypes = [_vp, ct.c_int, ct.c_int, ct.c_int]
    lib.hb_get_tuning.argtypes = [_vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    lib.hb_kernel_stats.argtypes = [_vp, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64),
                                    ct.c_int]
    lib.hb_residual_norms_noalloc.argtypes = [_vp, _vp, ct.c_int, ct.c_int64, ct.c_int, ct.c_int,
                                              _vp, _vp]
    lib.hb_graph_info.argtypes = [_vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int64)]
    lib.hb_halo_pass.argtypes = [_vp, _vp, ct.c_int, _vp]
    lib.hb_rk_stage.argtypes = [_vp, _vp, _vp, _vp, ct.c_int, _vp, _vp]
    lib.hb_pack_halo.argtypes = [_vp, _vp, _vp, ct.c_int64, _vp, _vp]
    lib.hb_unpack_halo.argtypes = [_vp, _vp, _vp, ct.c_int64, _vp, _vp]
    lib.hb_td_step.argtypes = [_vp, _vp, _vp, _vp, ct.c_double, ct.c_double, ct.c_int, _vp, _vp]
    lib.hb_defect_correction.argtypes = [_vp, _vp, _vp, ct.c_int, ct.c_int, ct.c_double, _vp, _vp]
    lib.hb_save_state.argtypes = [_vp, _vp, ct.c_char_p, ct.c_int64, _vp]
    lib.hb_load_state.argtypes = [_vp, _vp, ct.c_char_p, ct.POINTER(ct.c_int64), _vp]
    lib.hb_last_error.restype = ct.c_char_p
    lib.hb_last_error.argtypes = [_vp]
    _lib = lib
    return lib


def _desc(case, prec):
    """Marshal a cases.Case into an HbCaseDesc; returns (desc, keepalive)."""
    keep = []
    nb = len(case.blocks)
    blocks = (HbBlockDesc * nb)()
    for b, blk in enumerate(case.blocks):
        nodes = np.ascontiguousarray(blk.nodes, dtype=np.float64)
        keep.append(nodes)
        blocks[b].ni, blocks[b].nj, blocks[b].nk = blk.n
        blocks[b].nodes = nodes.ctypes.data_as(_dp)
    cuts = (HbCutDesc * max(1, len(case.cuts)))()
    for q, r in enumerate(np.asarray(case.cuts).reshape(-1, 17)):
        c = cuts[q]
        c.dst_blk, c.src_blk = int(r[0]), int(r[1])
        for a in range(3):
            c.lo[a], c.hi[a], c.off[a] = int(r[2 + a]), int(r[5 + a]), int(r[8 + a])
            c.perm[a], c.sign[a] = int(r[11 + a]), int(r[14 + a])
    bcs = (HbBcDesc * max(1, len(case.bcs)))()
    for q, r in enumerate(np.asarray(case.bcs).reshape(-1, 10)):
        c = bcs[q]
        c.blk, c.face = int(r[0]), int(r[1])
        for a in range(3):
            c.lo[a], c.hi[a] = int(r[2 + a]), int(r[5 + a])
        c.type, c.body = int(r[8]), int(r[9])
    d = HbCaseDesc()
    d.dim, d.n_harm = case.dim, case.n_harm
    d.mach, d.reynolds, d.prandtl, d.gamma = case.mach, case.reynolds, case.prandtl, case.gamma
    d.alpha0_deg, d.omega, d.cfl = case.alpha0_deg, case.omega, case.cfl
    d.lim_eps, d.entropy_frac = case.lim_eps, case.entropy_frac
    d.viscous, d.entropy_fix = int(case.viscous), int(case.entropy_fix)
    d.motion, d.pitch_amp_deg = int(case.motion), case.pitch_amp_deg
    d.pivot[0], d.pivot[1] = case.pivot
    d.ubc, d.ubc_amp = int(case.ubc), case.ubc_amp
    d.n_blocks, d.blocks = nb, blocks
    d.n_cuts, d.cuts = len(case.cuts), cuts
    d.n_bcs, d.bcs = len(case.bcs), bcs
    d.n_bodies, d.functag, d.prec = case.n_bodies, case.functag, prec
    keep += [blocks, cuts, bcs]
    return d, keep


def _stream():
    import torch
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ct.c_void_p(0 if t is None else t.data_ptr())


class HBContext:
    """A library context for one case (or a batch of cases)."""

    def __init__(self, case, prec: str = "fp64"):
        lib = load()
        self.lib = lib
        self.prec = HB_FP32 if prec in ("fp32", HB_FP32) else HB_FP64
        cases = case if isinstance(case, (list, tuple)) else [case]
        self.cases = list(cases)
        self.is_batch = isinstance(case, (list, tuple))
        descs, keep = [], []
        for c in cases:
            d, k = _desc(c, self.prec)
            descs.append(d)
            keep.append(k)
        arr = (HbCaseDesc * len(descs))(*descs)
        h = _vp()
        if isinstance(case, (list, tuple)):
            st = lib.hb_create_batch(arr, len(descs), ct.byref(h))
        else:
            st = lib.hb_create(arr, ct.byref(h))
        if st != HB_OK:
            raise HBError(st, "hb_create failed (see stderr)")
        self.h = h
        self.size = int(lib.hb_state_size(h))
        self.nv = cases[0].nv
        self.layouts = []
        nblocks = sum(len(c.blocks) for c in cases)
        for b in range(nblocks):
            off = ct.c_int64()
            st_ = (ct.c_int64 * 5)()
            ext = (ct.c_int * 3)()
            self._check(lib.hb_state_layout(h, b, ct.byref(off), st_, ext))
            self.layouts.append((int(off.value), tuple(int(x) for x in st_), tuple(int(x) for x in ext)))
        self._gather = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.hb_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _check(self, st):
        if st != HB_OK:
            msg = self.lib.hb_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise HBError(st, msg)

    @property
    def dtype(self):
        import torch
        return torch.float32 if self.prec == HB_FP32 else torch.float64

    def new_state(self, device="cuda"):
        import torch
        return torch.zeros(self.size, dtype=self.dtype, device=device)

    # ---- layout marshalling (compact interior order [block][n][v][k][j][i])
    def gather_index(self):
        if self._gather is None:
            idx = []
            b = 0
            for c in self.cases:
                for blk in c.blocks:
                    off, st, _ = self.layouts[b]
                    ni, nj, nk = blk.n
                    gk = 2 if c.dim == 3 else 0
                    n = np.arange(c.n_snap)[:, None, None, None, None]
                    v = np.arange(c.nv)[None, :, None, None, None]
                    k = np.arange(nk)[None, None, :, None, None]
                    j = np.arange(nj)[None, None, None, :, None]
                    i = np.arange(ni)[None, None, None, None, :]
                    e = off + n * st[0] + v * st[1] + (k + gk) * st[2] + (j + 2) * st[3] + (i + 2) * st[4]
                    idx.append(e.reshape(-1))
                    b += 1
            self._gather = np.concatenate(idx).astype(np.int64)
        return self._gather

    def to_compact(self, U):
        import torch
        gi = torch.as_tensor(self.gather_index(), device=U.device)
        return U[gi]

    def from_compact(self, flat, U=None):
        import torch
        gi = torch.as_tensor(self.gather_index(), device=flat.device)
        if U is None:
            U = torch.zeros(self.size, dtype=self.dtype, device=flat.device)
        U[gi] = flat.to(self.dtype)
        return U

    # ---- library calls
    def init_state(self, U, noise=None, amp=0.0):
        self._check(self.lib.hb_init_state(self.h, _ptr(U), _ptr(noise), float(amp), _stream()))
        return U

    def exchange_halos(self, U):
        self._check(self.lib.hb_exchange_halos(self.h, _ptr(U), _stream()))
        return U

    def residual(self, U, R=None):
        if R is None:
            R = self.new_state(U.device)
        self._check(self.lib.hb_residual(self.h, _ptr(U), _ptr(R), _stream()))
        return R

    def rk_smooth(self, U, n_iter, norms=True):
        """n_iter RK iterations in place; returns FP64 norms [n_iter][nv]
        (single case) or [n_iter][n_cases][nv] (batch)."""
        import torch
        nc = len(self.cases)
        out = (torch.zeros((max(n_iter, 1), nc, self.nv), dtype=torch.float64, device=U.device)
               if norms else None)
        self._check(self.lib.hb_rk_smooth(self.h, _ptr(U), int(n_iter), _ptr(out), _stream()))
        if not norms:
            return None
        out = out[:n_iter]
        return out[:, 0] if nc == 1 and not self.is_batch else out

    def autotune(self, U, iters=3):
        self._check(self.lib.hb_autotune(self.h, _ptr(U), int(iters), _stream()))
        return self.tuning()

    def set_tuning(self, mode, TI=32, TJ=8):
        self._check(self.lib.hb_set_tuning(self.h, int(mode), int(TI), int(TJ)))

    def tuning(self):
        m, a, b = ct.c_int(), ct.c_int(), ct.c_int()
        self._check(self.lib.hb_get_tuning(self.h, ct.byref(m), ct.byref(a), ct.byref(b)))
        return int(m.value), int(a.value), int(b.value)

    def rk_smooth_into(self, U, n_iter, norms=None):
        """hb_rk_smooth with a caller-provided FP64 [n_iter][nv] norms tensor (or None)."""
        self._check(self.lib.hb_rk_smooth(self.h, _ptr(U), int(n_iter), _ptr(norms), _stream()))

    def forces_into(self, U, coef=None, J=None):
        self._check(self.lib.hb_forces(self.h, _ptr(U), _ptr(coef), _ptr(J), _stream()))

    def forces(self, U):
        import torch
        c = self.cases[0]
        coef = torch.zeros((c.n_snap, max(c.n_bodies, 1), 3), dtype=torch.float64, device=U.device)
        J = torch.zeros(1, dtype=torch.float64, device=U.device)
        self._check(self.lib.hb_forces(self.h, _ptr(U), _ptr(coef), _ptr(J), _stream()))
        return coef[:, :c.n_bodies], J

    def adjoint_residual(self, U, psi, J_seed=0.0, r_adj=None):
        import torch
        if r_adj is None:
            r_adj = self.new_state(U.device)
        J = torch.zeros(1, dtype=torch.float64, device=U.device)
        self._check(self.lib.hb_adjoint_residual(self.h, _ptr(U), _ptr(psi), float(J_seed),
                                                 _ptr(r_adj), _ptr(J), _stream()))
        return r_adj, J

    def set_timing(self, enable=True):
        self._check(self.lib.hb_set_timing(self.h, int(bool(enable))))

    def kernel_stats(self, which, reset=False):
        """(ms, launches) of kernel class `which` (0 tile, 1 halo, 2 all: count only)."""
        ms, n = ct.c_double(), ct.c_int64()
        self._check(self.lib.hb_kernel_stats(self.h, int(which), ct.byref(ms), ct.byref(n), int(reset)))
        return float(ms.value), int(n.value)

    # ---- block decomposition (a share of a multi-block case with external boxes)
    def halo_pass(self, U, p):
        """hb_halo_pass: this context's cuts and boundary ghosts of pass p."""
        self._check(self.lib.hb_halo_pass(self.h, _ptr(U), int(p), _stream()))

    def rk_stage(self, Uin, U0, Uout, stage, sums=None):
        """hb_rk_stage: Uout = U0 - alpha dtau/V R(Uin); at stage 0 the FP64
        sums of (R/V)^2 per case and variable into sums ([n_cases][nv])."""
        self._check(self.lib.hb_rk_stage(self.h, _ptr(Uin), _ptr(U0), _ptr(Uout), int(stage), _ptr(sums),
                                         _stream()))

    def pack_halo(self, U, idx, buf):
        """hb_pack_halo: buf[e] = U[idx[e]] (idx: int64 device tensor)."""
        self._check(self.lib.hb_pack_halo(self.h, _ptr(U), _ptr(idx), int(idx.numel()), _ptr(buf), _stream()))
        return buf

    def unpack_halo(self, U, idx, buf):
        """hb_unpack_halo: U[idx[e]] = buf[e]."""
        self._check(self.lib.hb_unpack_halo(self.h, _ptr(U), _ptr(idx), int(idx.numel()), _ptr(buf), _stream()))
        return U

    def graph_info(self):
        """hb_graph_info: (persist_captured, graph replays, persistent replays,
        direct persistent launches); persist_captured is -1 (no persistent
        chunk yet), 0 (capture refused) or 1 (captured)."""
        cap = ct.c_int()
        counts = (ct.c_int64 * 3)()
        self._check(self.lib.hb_graph_info(self.h, ct.byref(cap), counts))
        return int(cap.value), int(counts[0]), int(counts[1]), int(counts[2])

    def td_step(self, U, U_n, U_nm1, t, dt, n_inner, norms=True):
        """hb_td_step: n_inner dual-time iterations of the physical step to t
        (BDF2; backward Euler when U_nm1 is None); returns FP64 norms
        [n_inner][nv] (single case) or [n_inner][n_cases][nv]."""
        import torch
        nc = len(self.cases)
        out = (torch.zeros((max(n_inner, 1), nc, self.nv), dtype=torch.float64, device=U.device)
               if norms else None)
        self._check(self.lib.hb_td_step(self.h, _ptr(U), _ptr(U_n), _ptr(U_nm1), float(t), float(dt),
                                        int(n_inner), _ptr(out), _stream()))
        if not norms:
            return None
        out = out[:n_inner]
        return out[:, 0] if nc == 1 and not self.is_batch else out

    def defect_correction(self, ctx64, U64, n_outer, n_inner, sigma=1.0, norms=True):
        """hb_defect_correction with this FP32 context and the FP64 context
        ctx64 of the same case(s): U64 (FP64 state) refined in place; returns
        the FP64 defect norms [n_outer][nv] (single case) or [n_outer][n_cases][nv]."""
        import torch
        nc = len(self.cases)
        out = (torch.zeros((max(n_outer, 1), nc, self.nv), dtype=torch.float64, device=U64.device)
               if norms else None)
        self._check(self.lib.hb_defect_correction(self.h, ctx64.h, _ptr(U64), int(n_outer), int(n_inner),
                                                  float(sigma), _ptr(out), _stream()))
        if not norms:
            return None
        out = out[:n_outer]
        return out[:, 0] if nc == 1 and not self.is_batch else out

    def save_state(self, U, path, iteration=0):
        """hb_save_state: restart file of U's interior cells with `iteration`."""
        self._check(self.lib.hb_save_state(self.h, _ptr(U), os.fsencode(path), int(iteration), _stream()))

    def load_state(self, U, path):
        """hb_load_state into U; returns the stored iteration."""
        it = ct.c_int64(0)
        self._check(self.lib.hb_load_state(self.h, _ptr(U), os.fsencode(path), ct.byref(it), _stream()))
        return int(it.value)

    def sync_status(self):
        return int(self.lib.hb_sync_status(self.h, _stream()))


def residual_norms_noalloc(R, vol, ncells, n_snap, nv, norms):
    """Binding of hb_residual_norms_noalloc: R [n_snap][nv][ncells] and vol
    [ncells] (both float32 or both float64 CUDA tensors), norms FP64 [nv]."""
    import torch
    if R.dtype not in (torch.float32, torch.float64) or vol.dtype != R.dtype:
        raise ValueError("R and vol must both be float32 or both float64")
    if norms.dtype != torch.float64:
        raise ValueError("norms must be float64")
    for name, t in (("R", R), ("vol", vol), ("norms", norms)):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if R.device != vol.device or R.device != norms.device:
        raise ValueError("R, vol and norms must be on one device")
    if int(ncells) < 1 or int(n_snap) < 1 or int(nv) < 1:
        raise ValueError("ncells, n_snap and nv must be positive")
    if R.numel() < int(n_snap) * int(nv) * int(ncells) or vol.numel() < int(ncells) or norms.numel() < int(nv):
        raise ValueError("R, vol or norms is smaller than n_snap * nv * ncells, ncells or nv")
    prec = HB_FP32 if R.dtype == torch.float32 else HB_FP64
    st = load().hb_residual_norms_noalloc(_ptr(R), _ptr(vol), prec, int(ncells), int(n_snap), int(nv),
                                          _ptr(norms), _stream())
    if st != HB_OK:
        raise HBError(st, "hb_residual_norms_noalloc")
    return norms
