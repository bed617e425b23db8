"""Brute-force alpha complex straight from the definitions, in exact rationals.

This is a pin for the oracle, not a second oracle: it shares nothing with
``oracle/alpha_oracle.c`` and takes a different route through the mathematics.

* Weighted Delaunay membership (Definition DT1/DT2, Section 2.3) and Size
  (Section 2.3) are evaluated over ALL k-subsets (k = 1..4): a subset tau is
  "witnessed at its orthocentre" when no other ball has strictly smaller power
  there. sigma belongs to the weighted Delaunay triangulation iff some tau
  containing sigma is witnessed at its orthocentre, and Size(sigma) is the
  smallest OrthoSize over those tau: the closest witness of sigma lies in the
  relative interior of a face of its (convex) witness region, and that face is
  the witness region of a coface tau whose orthocentre it then is.
* K_alpha = { sigma : Size(sigma) <= alpha } (Section 2.4).
* The orthocentre is found by solving linear systems in absolute coordinates:
  the equal-power planes 2 (p_k - p_0) . c = |p_k|^2 - |p_0|^2 - W_k + W_0,
  plus the plane of the triangle for triangles; the foot of the perpendicular
  for edges.
* Degeneracies (Section 2: symbolic perturbation) are resolved by perturbing
  every weight explicitly, W_k + delta^(k+1) with delta = 2^-delta_bits, and
  evaluating exactly with Fractions: no coefficient derivation is involved.
  Values (Size) are reported for the unperturbed weights.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations


def _solve3(M, b):
    """Gaussian elimination over Fractions; returns None if M is singular."""
    A = [[Fraction(M[i][j]) for j in range(3)] + [Fraction(b[i])] for i in range(3)]
    for col in range(3):
        piv = next((r for r in range(col, 3) if A[r][col] != 0), None)
        if piv is None:
            return None
        A[col], A[piv] = A[piv], A[col]
        for r in range(3):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [A[r][j] - f * A[col][j] for j in range(4)]
    return [A[i][3] / A[i][i] for i in range(3)]


def _sub(a, b):
    return [a[0] - b[0], a[1] - b[1], a[2] - b[2]]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def orthocentre(P, W, tau):
    """Point of equal power to the balls of tau that minimises that power; None if flat."""
    p0 = P[tau[0]]
    if len(tau) == 1:
        return [Fraction(x) for x in p0]
    rows, rhs = [], []
    for k in tau[1:]:
        rows.append([2 * (P[k][i] - p0[i]) for i in range(3)])
        rhs.append(_dot(P[k], P[k]) - _dot(p0, p0) - W[k] + W[tau[0]])
    if len(tau) == 2:
        q = _sub(P[tau[1]], p0)
        qq = _dot(q, q)
        if qq == 0:
            return None
        t = Fraction(rhs[0] - 2 * _dot(q, p0), 2 * qq)  # 2 q.(p0 + t q) = rhs
        return [p0[i] + t * q[i] for i in range(3)]
    if len(tau) == 3:
        nrm = _cross(_sub(P[tau[1]], p0), _sub(P[tau[2]], p0))
        if nrm == [0, 0, 0]:
            return None
        rows.append(nrm)
        rhs.append(_dot(nrm, p0))
    return _solve3(rows, rhs)


def power(c, P, W, k):
    d = [c[i] - P[k][i] for i in range(3)]
    return _dot(d, d) - W[k]


def brute_alpha_complex(P, R, A=None, delta_bits=160, with_source=False):
    """P: integer centres (quanta), R: integer radii (quanta), A: alpha in quanta^2 (None = infinity).

    Returns {d: {tuple: (size, attached)}} with exact Fraction sizes in quanta^2.
    With with_source=True the value is (size, attached, taus): the subsets tau whose
    orthocentre is the closest witness (the simplices Size is taken from).
    """
    n = len(P)
    W0 = [Fraction(r * r) for r in R]
    delta = Fraction(1, 1 << delta_bits)
    We = [W0[k] + delta ** (k + 1) for k in range(n)]
    witnessed = {}
    for k in range(1, 5):
        for tau in combinations(range(n), k):
            ce = orthocentre(P, We, tau)
            if ce is None:
                continue
            pw = power(ce, P, We, tau[0])
            if all(power(ce, P, We, x) > pw for x in range(n) if x not in tau):
                c0 = orthocentre(P, W0, tau)
                witnessed[tau] = power(c0, P, W0, tau[0])
    out = {0: {}, 1: {}, 2: {}, 3: {}}
    for k in range(1, 5):
        for sigma in combinations(range(n), k):
            s = set(sigma)
            vals = [(v, tau) for tau, v in witnessed.items() if s.issubset(tau)]
            if not vals:
                continue
            size = min(v for v, _ in vals)
            if A is None or size <= A:
                if with_source:
                    taus = [tau for v, tau in vals if v == size]
                    out[k - 1][sigma] = (size, sigma not in witnessed, taus)
                else:
                    out[k - 1][sigma] = (size, sigma not in witnessed)
    return out


def _det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def witnessed_subsets(P, R, delta_bits=160):
    """The same witnessed-at-orthocentre test as brute_alpha_complex, in scaled integers.

    Every perturbed weight W_k + delta^(k+1) is multiplied by S = delta^-n, which
    makes it an integer, and the orthocentre of the perturbed balls is kept as
    num / (den * S) with integer num (Cramer's rule on the scaled equal-power
    planes) and a small positive integer den. The power comparison against
    every other ball is then an integer sign, with the loop stopping at the
    first ball of smaller or equal power. Returns {tau: OrthoSize(tau)} for the
    witnessed subsets, OrthoSize as an exact Fraction of the unperturbed balls.
    """
    n = len(P)
    D = 1 << delta_bits
    S = D ** n
    W0 = [r * r for r in R]
    Ws = [W0[k] * S + D ** (n - k - 1) for k in range(n)]  # S * (W_k + delta^(k+1))
    sq = [_dot(p, p) for p in P]
    out = {}
    for k in range(1, 5):
        for tau in combinations(range(n), k):
            t0 = tau[0]
            p0 = P[t0]
            if k == 1:
                den, num = 1, [p0[i] * S for i in range(3)]
            elif k == 2:
                q = _sub(P[tau[1]], p0)
                qq = _dot(q, q)
                if qq == 0:
                    continue
                # 2 q.c = rhs on the line c = p0 + t q
                rhs = S * (sq[tau[1]] - sq[t0]) - Ws[tau[1]] + Ws[t0]
                tn = rhs - 2 * S * _dot(q, p0)
                den = 2 * qq
                num = [p0[i] * den * S + tn * q[i] for i in range(3)]
            else:
                rows = [[2 * (P[j][i] - p0[i]) for i in range(3)] for j in tau[1:]]
                rhs = [S * (sq[j] - sq[t0]) - Ws[j] + Ws[t0] for j in tau[1:]]
                if k == 3:
                    nrm = _cross(_sub(P[tau[1]], p0), _sub(P[tau[2]], p0))
                    rows.append(nrm)
                    rhs.append(S * _dot(nrm, p0))
                den = _det3(rows)
                if den == 0:
                    continue
                num = []
                for i in range(3):
                    m = [row[:] for row in rows]
                    for r_ in range(3):
                        m[r_][i] = rhs[r_]
                    num.append(_det3(m))
            if den < 0:
                den, num = -den, [-v for v in num]
            # (pi(c, x) - pi(c, t0)) * den * S with c = num / (den * S)
            ok = True
            for x in range(n):
                if x in tau:
                    continue
                dx = _sub(P[x], p0)
                if -2 * _dot(num, dx) + den * (S * (sq[x] - sq[t0]) - Ws[x] + Ws[t0]) <= 0:
                    ok = False
                    break
            if ok:
                c0 = orthocentre(P, [Fraction(w) for w in W0], tau)
                out[tau] = power(c0, P, [Fraction(w) for w in W0], t0)
    return out


def alpha_complexes_from_witnessed(witnessed, alphas):
    """K_alpha for each alpha of `alphas` (None = infinity), in brute_alpha_complex's format.

    Size(sigma) is the smallest OrthoSize over the witnessed supersets of sigma,
    gathered by visiting the (at most 15) non-empty subsets of each witnessed tau.
    """
    size = {}
    for tau, v in witnessed.items():
        for k in range(1, len(tau) + 1):
            for sigma in combinations(tau, k):
                if sigma not in size or v < size[sigma]:
                    size[sigma] = v
    res = []
    for A in alphas:
        out = {0: {}, 1: {}, 2: {}, 3: {}}
        for sigma, s in size.items():
            if A is None or s <= A:
                out[len(sigma) - 1][sigma] = (s, sigma not in witnessed)
        res.append(out)
    return res
