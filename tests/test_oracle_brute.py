"""The oracle against the definition-level brute force (tests/brute.py).

Random positions, lattices with many exact ties (co-orthospherical balls,
collinear and coplanar subsets, equal weights), alpha at 0, > 0, at a value
that some simplex attains exactly, and infinity. Small inputs (4-12 atoms, 100
seeds of each kind) and large ones (30-40 atoms, where every 4-subset is still
visited: C(40, 4) = 91,390 orthocentres). The integer-scaled brute force used
for the bulk is itself checked against the Fraction one on small inputs.
"""
import numpy as np
import pytest

import oracle
from brute import alpha_complexes_from_witnessed, brute_alpha_complex, witnessed_subsets


def _case(kind, rng, n):
    if kind == "random":
        P = [tuple(int(v) for v in rng.integers(-3000, 3000, 3)) for _ in range(n)]
        R = [int(v) for v in rng.integers(800, 2500, n)]
        return P, R
    if kind == "lattice":  # two radii on a unit lattice: many co-orthospherical quintuples
        span, step, radii = (1 if n <= 12 else 2), 1024, [1024, 1448]
    else:  # equal radii on a finer lattice: ties of the unweighted Delaunay kind
        span, step, radii = (2 if n <= 12 else 3), 512, [700]
    pts = set()
    while len(pts) < n:
        pts.add(tuple(int(v) * step for v in rng.integers(-span, span + 1, 3)))
    P = sorted(pts, key=lambda p: rng.random())
    R = [int(rng.choice(radii)) for _ in range(n)]
    return P, R


def _run_oracle(P, R, A):
    c = np.array(P, dtype=np.float64).reshape(-1, 3) / 1024.0
    r = np.array(R, dtype=np.float64) / 1024.0
    if A is None:
        return oracle.alpha_complex(c, r, alpha_inf=True)
    return oracle.alpha_complex(c, r, alpha=A / 2**20)


def _compare(P, R, A, want_all):
    ac = _run_oracle(P, R, A)
    for d in range(4):
        got = {tuple(int(x) for x in t): (ac.f[d][i], bool(ac.attached[d][i])) for i, t in enumerate(ac.simplices[d])}
        want = want_all[d]
        assert set(got) == set(want), f"dim {d}: {len(set(got) ^ set(want))} simplices differ at alpha {A}"
        for t, (size, att) in want.items():
            assert got[t][1] == att, (d, t, A)
            assert got[t][0] == pytest.approx(float(size / 2**20), rel=1e-14, abs=1e-300), (d, t, A)


def _check(P, R):
    """Oracle = brute force at alpha 0, 300000 quanta^2, infinity and an attained Size."""
    w = witnessed_subsets(P, R)
    alphas = [0, 300000, None]
    sizes = sorted({v for v in w.values() if v.denominator == 1})
    if sizes:  # alpha exactly at an attained integral Size: AC3 is inclusive (Section 2.4, "<=")
        alphas.append(int(sizes[len(sizes) // 2]))
    for A, want in zip(alphas, alpha_complexes_from_witnessed(w, alphas)):
        _compare(P, R, A, want)


@pytest.mark.parametrize("kind", ["random", "lattice", "equal"])
def test_integer_brute_force_equals_fraction_brute_force(kind):
    # the scaled-integer route and the Fraction route of the same definition agree
    for seed in range(10):
        rng = np.random.default_rng(500 + seed)
        P, R = _case(kind, rng, int(rng.integers(2, 10)))
        fast = alpha_complexes_from_witnessed(witnessed_subsets(P, R), [0, 300000, None])
        for A, f in zip([0, 300000, None], fast):
            assert f == brute_alpha_complex(P, R, A), (seed, A)


@pytest.mark.parametrize("kind", ["random", "lattice", "equal"])
@pytest.mark.parametrize("block", range(4))
def test_oracle_equals_brute_force(kind, block):
    # 25 seeds per block, 100 per kind, 4 to 12 atoms
    for seed in range(25 * block, 25 * block + 25):
        rng = np.random.default_rng(1000 * seed + len(kind))
        P, R = _case(kind, rng, int(rng.integers(4, 13)))
        _check(P, R)


@pytest.mark.parametrize("kind", ["random", "lattice", "equal"])
@pytest.mark.parametrize("n", [30, 40])
def test_oracle_equals_brute_force_large(kind, n):
    rng = np.random.default_rng(7 * n + len(kind))
    P, R = _case(kind, rng, n)
    _check(P, R)


def test_empty_and_tiny_inputs():
    for n in range(0, 4):
        P = [(0, 0, 0), (2048, 0, 0), (0, 2048, 0)][:n]
        R = [1536] * n
        for A in (0, None):
            _compare(P, R, A, brute_alpha_complex(P, R, A))


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
