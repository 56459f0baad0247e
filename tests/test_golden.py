"""Regression fixtures of the oracle (tests/golden/, written by tests/golden/make_golden.py
from the oracle alone).

The paper prints no worked example with values for the sweep, so these files are not pins of
the oracle to the paper (tests/test_oracle_*.py hold those); they record the oracle's current
results so that a change to its arithmetic cannot pass unnoticed. The C oracle's chains must
reproduce them bit for bit; the numpy analysis, whose reductions may group sums differently
from one numpy build to another, to 1e-12 relative.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT

GOLDEN = os.path.join(ROOT, "tests", "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402


def read(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = vals
    return rows


def as_floats(vals):
    return np.array([float.fromhex(v) for v in vals])


@pytest.mark.parametrize("name,make", [("oracle_sc4_chain.txt", make_golden.sc4_chain),
                                       ("oracle_ising_chain.txt", make_golden.ising_chain)])
def test_oracle_chains_reproduce_their_fixtures_bit_for_bit(name, make):
    stored = read(name)
    rows = make()
    assert sorted(stored) == sorted(k for k, *_ in rows)
    for key, vals in rows:
        got, want = np.asarray(vals, dtype=np.float64), as_floats(stored[key])
        assert got.shape == want.shape and np.array_equal(got, want), (name, key)


def test_analysis_reproduces_its_fixture():
    stored = read("oracle_thermal.txt")
    rows = {r[0]: r for r in make_golden.thermal()}
    assert stored["names"] == rows["names"][2]
    np.testing.assert_allclose(rows["fields"][1], as_floats(stored["fields"]), rtol=1e-12, atol=0.0)


def test_fixtures_carry_their_provenance():
    for name in ("oracle_sc4_chain.txt", "oracle_ising_chain.txt", "oracle_thermal.txt"):
        with open(os.path.join(GOLDEN, name)) as f:
            head = f.readline() + f.readline()
        assert "Sec." in head and "make_golden.py" in head, name
    assert subprocess.run([sys.executable, "-m", "py_compile", os.path.join(GOLDEN, "make_golden.py")]).returncode == 0
