"""The oracle's closed-form gradient against central differences of the definition.

L = sum_sigma w_sigma Size(sigma) with the combinatorics held fixed: Size(sigma) is
the OrthoSize of the simplex whose orthocentre is sigma's closest witness
(Section 2.3), chosen here by the brute force. The difference quotient is taken
in exact rationals on the definition (orthocentre by a linear solve, power
distance pi(p,b) = |p - p_b|^2 - r_b^2, Section 2.2), so it shares nothing with
the oracle's formula 2 lambda_k (p_k - c), -2 r_k lambda_k.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from brute import brute_alpha_complex, orthocentre, power


def _orthosize(P, W, tau):
    c = orthocentre(P, W, tau)
    return power(c, P, W, tau[0])


@pytest.mark.parametrize("seed", range(4))
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    n = 7
    Pq = [tuple(int(v) for v in rng.integers(-2500, 2500, 3)) for _ in range(n)]
    Rq = [int(v) for v in rng.integers(1200, 2400, n)]
    A = 2 * 2**20  # alpha = 2 A^2: plenty of simplices, some attached
    br = brute_alpha_complex(Pq, Rq, A, with_source=True)
    c = np.array(Pq, dtype=np.float64) / 1024
    r = np.array(Rq, dtype=np.float64) / 1024
    ac = oracle.alpha_complex(c, r, alpha=2.0)
    terms = []  # (weight, source tau)
    dldf = []
    for d in range(4):
        w = np.zeros(len(ac.simplices[d]))
        for i, t in enumerate(ac.simplices[d]):
            size, att, taus = br[d][tuple(int(x) for x in t)]
            if len(taus) == 1:
                w[i] = rng.normal()
                terms.append((Fraction(float(w[i])), taus[0]))
        dldf.append(w)
    assert any(len(t[1]) > 1 for t in terms)
    gc, gr = ac.gradient(dldf)

    P0 = [[Fraction(int(x), 1024) for x in p] for p in Pq]
    R0 = [Fraction(int(x), 1024) for x in Rq]
    h = Fraction(1, 1 << 26)

    def L(P, R):
        W = [x * x for x in R]
        return sum(w * _orthosize(P, W, tau) for w, tau in terms)

    for a in range(n):
        for ax in range(3):
            Pp = [list(p) for p in P0]
            Pm = [list(p) for p in P0]
            Pp[a][ax] += h
            Pm[a][ax] -= h
            fd = float((L(Pp, R0) - L(Pm, R0)) / (2 * h))
            assert gc[a, ax] == pytest.approx(fd, rel=1e-9, abs=1e-9)
        Rp = list(R0)
        Rm = list(R0)
        Rp[a] += h
        Rm[a] -= h
        fd = float((L(P0, Rp) - L(P0, Rm)) / (2 * h))
        assert gr[a] == pytest.approx(fd, rel=1e-9, abs=1e-9)
