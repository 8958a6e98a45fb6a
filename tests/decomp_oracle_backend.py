"""The FP64 oracle as the per-rank backend of paper_1304_7654_gb300.decomp
(test infrastructure: lets the block decomposition's host logic -- partition,
exchange tables, pass order, sums over ranks -- run on CPU ranks)."""
import numpy as np
import torch

from oracle.hb_oracle import Oracle


class OracleBackend:
    def __init__(self, case):
        self.o = Oracle(case)
        self.case = case

    def layout(self, b):
        off, p, g = self.o.blocks[b]
        plane = p[0] * p[1] * p[2]
        return off, (self.case.nv * plane, plane, p[0] * p[1], p[0], 1)

    def index(self, a):
        return np.asarray(a, dtype=np.int64)

    def new_state(self):
        return np.zeros(self.o.size)

    def halo_pass(self, U, p):
        self.o.halo_pass(U, p)

    def stage(self, Uin, U0, Uout, s, sums):
        self.o.rk_stage(Uin, U0, Uout, s, None if sums is None else sums.numpy())

    def sums_buffer(self):
        return torch.zeros(self.case.nv, dtype=torch.float64)

    def pack(self, U, idx):
        return torch.as_tensor(U[idx].copy())

    def unpack(self, U, idx, buf):
        U[idx] = np.asarray(buf)

    def forces(self, U):
        coef, J = self.o.forces(U)
        return torch.as_tensor(np.ascontiguousarray(coef)), torch.as_tensor([J], dtype=torch.float64)
