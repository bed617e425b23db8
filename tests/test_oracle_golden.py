"""The oracle (and the brute-force pin) against hand-derived closed forms in tests/golden/."""
import os

import numpy as np
import pytest

import oracle
from brute import brute_alpha_complex
from golden_io import fixtures, read_fixture


@pytest.mark.parametrize("path", fixtures(), ids=[os.path.basename(p) for p in fixtures()])
def test_oracle_matches_golden(path):
    atoms, alpha, expect = read_fixture(path)
    c = np.array([[float(a[0]), float(a[1]), float(a[2])] for a in atoms])
    r = np.array([float(a[3]) for a in atoms])
    ac = oracle.alpha_complex(c, r, alpha=float(alpha) if alpha is not None else 0.0, alpha_inf=alpha is None)
    got = {}
    for d in range(4):
        for i, t in enumerate(ac.simplices[d]):
            got[tuple(int(x) for x in t)] = (ac.f[d][i], bool(ac.attached[d][i]))
    assert set(got) == set(expect)
    for t, (f, att) in expect.items():
        assert got[t][1] == att, t
        assert got[t][0] == pytest.approx(float(f), rel=1e-15, abs=0), t


@pytest.mark.parametrize("path", fixtures(), ids=[os.path.basename(p) for p in fixtures()])
def test_brute_force_matches_golden(path):
    atoms, alpha, expect = read_fixture(path)
    P = [tuple(int(x * 1024) for x in a[:3]) for a in atoms]
    R = [int(a[3] * 1024) for a in atoms]
    A = None if alpha is None else int(alpha * 2**20)
    br = brute_alpha_complex(P, R, A)
    got = {t: v for d in range(4) for t, v in br[d].items()}
    assert set(got) == set(expect)
    for t, (f, att) in expect.items():
        assert got[t][0] / 2**20 == f, t
        assert got[t][1] == att, t
