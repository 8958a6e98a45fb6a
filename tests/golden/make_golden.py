"""Write the stored expected values of tests/golden/ from the FP64 oracle alone.

The paper prints no worked example or solution values, so the fixtures here
are regression values of the oracle itself (which is pinned to the
mathematics by tests/test_oracle_pins.py): a change to the oracle's arithmetic
shows up as a changed fixture, and its commit has to name the passage or the
reading that justifies it.  Only oracle/ and the seeded input generators are
called.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.hb_oracle import Oracle  # noqa: E402
from paper_1304_7654_gb300 import cases as C  # noqa: E402

N_SAMPLE = 64


def golden_cases():
    """(name, case) pairs of the fixtures: small, seeded members of the
    benchmark families (2D inviscid channel, 2D laminar pitching O-grid with
    two blocks and a wall, 3D laminar box)."""
    return [
        ("channel_12x6_nh1", C.channel(12, 6, n_harm=1)),
        ("ogrid_24x8_nh2_two_blocks", C.ogrid(24, 8, n_harm=2, viscous=True, pitch_deg=3.0, radius=5.0,
                                              specs=[C.BlockSpec((0, 0), (10, 8)), C.BlockSpec((10, 0), (24, 8))])),
        ("box3d_6x5x4_nh1", C.box3d(6, 5, 4, n_harm=1)),
    ]


def evaluate(cs):
    """The oracle's outputs on one case from the seeded start: sampled
    residual entries (compact interior order), the residual-norm history of
    3 RK iterations, and the force coefficients and J after them."""
    o = Oracle(cs)
    U = o.init_state(C.noise(cs), 0.01)
    R = o.unpack(o.residual(U, with_scale=False))
    idx = np.random.default_rng(99).choice(R.size, size=min(N_SAMPLE, R.size), replace=False)
    U3, norms = o.rk_smooth(U, 3)
    out = {"residual_index": [int(i) for i in np.sort(idx)],
           "residual": [float(R[i]) for i in np.sort(idx)],
           "norms_3it": [[float(x) for x in row] for row in norms]}
    if cs.n_bodies:
        coef, J = o.forces(U3)
        out["forces_3it"] = [[[float(x) for x in b] for b in s] for s in coef]
        out["J_3it"] = float(J)
    return out


CONVERGED_NAME = "converged_forces_ogrid32x8_viscous_nh1"
CONVERGED_ITERS = 24000


def converged_case():
    """Laminar pitching O-grid, 32 x 8 cells, N_H = 1, van Albada constant
    1e-12 (the reading used everywhere): small enough for the oracle to run
    the RK smoother to a steady periodic state (residual norms ~1e-13)."""
    return C.ogrid(32, 8, n_harm=1, viscous=True, pitch_deg=3.0)


def converged_forces(threads=None):
    """The oracle's force coefficients and J after CONVERGED_ITERS RK
    iterations from the freestream (the OpenMP build of the oracle: the same
    iterations bit for bit, on all host cores), with the last norms."""
    from oracle.hb_oracle import build_openmp
    build_openmp()
    cs = converged_case()
    o = Oracle(cs, openmp=True)
    U = o.init_state(np.zeros(C.interior_count(cs)), 0.0)
    n = threads or max(1, len(os.sched_getaffinity(0)))
    U, norms = o.rk_smooth_threads(U, CONVERGED_ITERS, n)
    coef, J = o.forces(U)
    return {"iterations": CONVERGED_ITERS, "last_norms": [float(x) for x in norms[-1]],
            "forces": [[[float(x) for x in b] for b in s] for s in coef], "J": float(J)}


def _write(name, out):
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        f.write("{\n" + ",\n".join(f'"{k}": {json.dumps(v)}' for k, v in out.items()) + "\n}\n")


def main():
    for name, cs in golden_cases():
        _write(name, evaluate(cs))
    _write(CONVERGED_NAME, converged_forces())


if __name__ == "__main__":
    main()
