"""The oracle against its frozen outputs (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): path counts and flags
exact, fields to 1e-12 of the largest.  A change to the oracle's arithmetic
fails here until it is justified and the fixtures are rewritten."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402


@pytest.mark.parametrize("case", make_golden.cases(), ids=lambda c: c[0])
def test_oracle_reproduces_golden(oracle_mod, case):
    name, cite, sc = case
    path = os.path.join(HERE, "golden", name + ".txt")
    stored = np.loadtxt(path, comments="#", ndmin=2)
    r = oracle_mod.evaluate(sc)
    assert stored.shape[0] == sc.n_rx
    assert np.array_equal(stored[:, 1].astype(int), r.counts)
    assert np.array_equal(stored[:, 2].astype(np.uint32), r.flags)
    E = stored[:, 3:].reshape(sc.n_rx, len(sc.freqs), 3, 2)
    E = E[..., 0] + 1j * E[..., 1]
    got = np.transpose(r.E, (2, 0, 1))
    assert np.max(np.abs(got - E)) <= 1e-12 * np.max(np.abs(E))
    assert np.max(r.counts) > 0
