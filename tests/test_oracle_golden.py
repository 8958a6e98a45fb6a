"""The oracle against its stored regression values: tests/golden/*.json,
written by tests/golden/make_golden.py from the oracle alone (the paper prints
no worked example).  Sampled residual entries, 3 RK iterations of residual
norms and the force coefficients after them, on small seeded members of the
benchmark families; any change to the oracle's arithmetic fails here until the
fixtures are rewritten by that script."""
import importlib.util
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


MAKER = _maker()


@pytest.mark.parametrize("name", [n for n, _ in MAKER.golden_cases()])
def test_oracle_reproduces_its_golden_values(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        ref = json.load(f)
    got = MAKER.evaluate(dict(MAKER.golden_cases())[name])
    assert got["residual_index"] == ref["residual_index"]
    for key in ref:
        if key == "residual_index":
            continue
        a, b = np.asarray(got[key], dtype=float), np.asarray(ref[key], dtype=float)
        scale = np.abs(b).max()
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13 * scale, err_msg=key)


def test_oracle_reproduces_its_converged_forces():
    """The converged-forces fixture (24,000 RK iterations of a small laminar
    O-grid; the OpenMP build of the oracle, bit for bit the plain one): the
    run reproduces it, and it is converged (last residual norms below 1e-12)."""
    with open(os.path.join(GOLDEN, MAKER.CONVERGED_NAME + ".json")) as f:
        ref = json.load(f)
    assert max(ref["last_norms"]) < 1e-12
    got = MAKER.converged_forces()
    np.testing.assert_allclose(np.asarray(got["forces"]), np.asarray(ref["forces"]), rtol=1e-11, atol=1e-15)
    assert abs(got["J"] - ref["J"]) <= 1e-13 * max(1.0, abs(ref["J"]))
