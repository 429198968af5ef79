"""The oracle against its stored results in tests/golden/ (written by
tests/golden/make_golden.py from oracle/ alone): a change of the oracle's
arithmetic shows here first.  Counts, coarse dimensions and CG iteration
counts must match exactly; eigenvalues to 1e-9 relative (absolute 1e-10 for
eigenvalues at rounding level, the kernels of floating subdomains)."""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


@pytest.mark.parametrize("name", sorted(make_golden.CASES))
def test_oracle_matches_stored_results(name):
    stored = json.load(open(os.path.join(HERE, "golden", name + ".json")))
    now = make_golden.compute(name)
    assert now["coarse_dims"] == stored["coarse_dims"]
    assert now["pcg"]["iterations_1e-8"] == stored["pcg"]["iterations_1e-8"]
    assert now["pcg"]["iterations_1e-12"] == stored["pcg"]["iterations_1e-12"]
    assert abs(now["pcg"]["x_norm_1e-12"] - stored["pcg"]["x_norm_1e-12"]) <= 1e-10 * stored["pcg"]["x_norm_1e-12"]
    for l, subs in stored["levels"].items():
        assert len(now["levels"][l]) == len(subs)
        for a, b in zip(now["levels"][l], subs):
            assert a["m"] == b["m"]
            la, lb = np.array(a["lam"]), np.array(b["lam"])
            assert la.shape == lb.shape
            assert np.all(np.abs(la - lb) <= np.maximum(1e-9 * np.abs(lb), 1e-10))
