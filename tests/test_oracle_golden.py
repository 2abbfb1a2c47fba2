"""Regression fixture of the FP64 oracle (tests/golden/oracle_regression.txt, written
by tests/golden/make_oracle_fixtures.py, which calls only oracle/): the oracle must
reproduce its stored values.  A change to the oracle's arithmetic that moves them is
regenerated with the script, and its commit names the passage that justifies it.
The oracle's independent pins are in test_oracle_pins.py."""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _fixture_module():
    spec = importlib.util.spec_from_file_location("make_oracle_fixtures",
                                                  os.path.join(HERE, "golden", "make_oracle_fixtures.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_oracle_reproduces_its_regression_fixture():
    stored = []
    with open(os.path.join(HERE, "golden", "oracle_regression.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            stored.append((parts[0], tuple(float(x) for x in parts[1:-1]), float(parts[-1])))
    now = _fixture_module().values()
    assert len(now) == len(stored) == 20
    for (k0, a0, v0), (k1, a1, v1) in zip(stored, now):
        assert k0 == k1 and np.allclose(a0, a1, rtol=1e-14, atol=0)
        # compilers may contract multiply-adds differently across hosts
        assert abs(v1 - v0) <= 1e-10 * abs(v0) + 1e-18, (k0, a0, v0, v1)
    assert any(k == "exact" and v > 0 for k, _, v in stored) and any(k == "band" for k, _, _ in stored)
