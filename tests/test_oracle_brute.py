"""The oracle against the definition-level brute force (tests/brute.py) on small inputs.

Random positions, lattices with many exact ties (five co-orthospherical balls,
collinear and coplanar subsets, equal weights), alpha at 0, > 0, at a value
that some simplex attains exactly, and infinity.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from brute import brute_alpha_complex


def _case(kind, rng, n):
    if kind == "random":
        P = [tuple(int(v) for v in rng.integers(-3000, 3000, 3)) for _ in range(n)]
        R = [int(v) for v in rng.integers(800, 2500, n)]
    elif kind == "lattice":
        pts = set()
        while len(pts) < n:
            pts.add(tuple(int(v) * 1024 for v in rng.integers(-1, 2, 3)))
        P = sorted(pts, key=lambda p: rng.random())
        R = [int(rng.choice([1024, 1448])) for _ in range(n)]
    else:  # equal radii on a finer lattice
        pts = set()
        while len(pts) < n:
            pts.add(tuple(int(v) * 512 for v in rng.integers(-2, 3, 3)))
        P = sorted(pts, key=lambda p: rng.random())
        R = [700] * n
    return P, R


def _run_oracle(P, R, A):
    c = np.array(P, dtype=np.float64) / 1024.0
    r = np.array(R, dtype=np.float64) / 1024.0
    if A is None:
        return oracle.alpha_complex(c, r, alpha_inf=True)
    return oracle.alpha_complex(c, r, alpha=A / 2**20)


def _compare(P, R, A):
    ac = _run_oracle(P, R, A)
    br = brute_alpha_complex(P, R, A)
    for d in range(4):
        got = {tuple(int(x) for x in t): (ac.f[d][i], bool(ac.attached[d][i])) for i, t in enumerate(ac.simplices[d])}
        want = br[d]
        assert set(got) == set(want), f"dim {d}"
        for t, (size, att) in want.items():
            assert got[t][1] == att, (d, t)
            assert got[t][0] == pytest.approx(float(size / 2**20), rel=1e-14, abs=1e-300), (d, t)
    return br


@pytest.mark.parametrize("kind", ["random", "lattice", "equal"])
@pytest.mark.parametrize("seed", range(8))
def test_oracle_equals_brute_force(kind, seed):
    rng = np.random.default_rng(1000 * seed + len(kind))
    n = int(rng.integers(4, 11))
    P, R = _case(kind, rng, n)
    for A in (0, 300000, None):
        br = _compare(P, R, A)
    # alpha exactly at an attained integral Size: AC3 is inclusive (Section 2.4, "<=")
    sizes = sorted({v[0] for d in range(4) for v in br[d].values() if v[0].denominator == 1})
    if sizes:
        _compare(P, R, int(sizes[len(sizes) // 2]))


def test_empty_and_tiny_inputs():
    for n in range(0, 4):
        P = [(0, 0, 0), (2048, 0, 0), (0, 2048, 0)][:n]
        R = [1536] * n
        _compare(P, R, 0)
        _compare(P, R, None)


def test_coincident_centres_are_rejected():
    c = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    r = np.array([1.0, 1.0])
    with pytest.raises(oracle.OracleError) as e:
        oracle.alpha_complex(c, r)
    assert e.value.code == -2


def test_invalid_inputs_are_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.alpha_complex(np.array([[np.nan, 0, 0]]), np.array([1.0]))
    with pytest.raises(oracle.OracleError):
        oracle.alpha_complex(np.array([[0.0, 0, 0]]), np.array([0.0]))
