"""The oracle still reproduces its stored regression fixture (tests/golden/, written by
tests/golden/make_golden.py from oracle/ only).  A change to the oracle's arithmetic fails
here until the fixture is rewritten on purpose.  CPU only."""
import os
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden as mg  # noqa: E402


def test_oracle_matches_golden_fixture():
    stored = mg.read()
    now = mg.compute()
    assert set(stored) == set(now)
    for k, v in now.items():
        a, b = np.asarray(v, float), np.asarray(stored[k], float)
        assert a.shape == b.shape, k
        scale = np.abs(b).max()
        assert scale > 0, k
        assert np.abs(a - b).max() <= 1e-9 * scale, (k, np.abs(a - b).max() / scale)


def test_golden_fixture_is_consistent():
    """Internal relations of the stored values: the K(0,0) entry is -W0 (K = -W0 on the
    diagonal of the direct kernel's k = k' blocks for n = n', m = m'), the runs start from
    equilibrium, and the truncated runs stay close to the dense one."""
    g = mg.read()
    assert abs(g["K_entries"][0] + g["W0"][0]) < 1e-14 * g["W0"][0]
    assert g["P_full"][0] == 0.0 and g["occ_full"][0] == 0.0
    P = np.asarray(g["P_full"])
    for k in ("P_lowrank29", "P_channel9"):
        assert np.linalg.norm(np.asarray(g[k]) - P) < 0.2 * np.linalg.norm(P), k
