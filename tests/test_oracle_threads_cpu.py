"""The OpenMP build of the oracle (used only to time it on all host cores)
gives the single-thread oracle's RK iterations bit for bit."""
import numpy as np

from oracle.hb_oracle import Oracle
from paper_1304_7654_gb300 import cases as C


def test_openmp_oracle_equals_single_thread_bitwise():
    cs = C.ns_ogrid8(64, 24, n_harm=2)
    o, oo = Oracle(cs), Oracle(cs, openmp=True)
    U = o.init_state(C.noise(cs), 0.01)
    U1, n1 = o.rk_smooth(U, 2)
    for threads in (1, 3):
        U2, n2 = oo.rk_smooth_threads(U, 2, threads)
        assert np.array_equal(U1, U2) and np.array_equal(n1, n2), threads
