"""The pins are sensitive: copies of the oracle with a planted mistake must fail them.

Each mutation is a plausible slip (a sign, a dropped term, a strict bound, a
skipped step). It is applied to a temporary copy of ``oracle/alpha_oracle.c``,
compiled with gcc, and run against the golden fixtures, the quantisation cases
and the brute force; at least one comparison must fail. The real oracle is untouched.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from brute import brute_alpha_complex
from golden_io import fixtures, read_fixture

MUTATIONS = {
    "perturbation_sign_flipped": ("sign = coef[k] > 0 ? 1 : -1;", "sign = coef[k] > 0 ? -1 : 1;"),
    "test_ball_coefficient_positive": ("int sign = -1;", "int sign = 1;"),
    "a_k_drops_w0": ("- W[v[k + 1]] + w0;", "- W[v[k + 1]];"),
    "adjugate_2x2_sign": ("s->adj[0][1] = -G[0][1];", "s->adj[0][1] = G[0][1];"),
    "adjugate_3x3_transposed_index": ("s->adj[j][i] = G[r0][c0] * G[r1][c1] - G[r0][c1] * G[r1][c0];",
                                      "s->adj[j][i] = G[r0][c0] * G[r1][c1] - G[r1][c0] * G[r1][c1];"),
    "ac3_strict": ("return s->os_num <= (i128)pr->A * s->os_den;", "return s->os_num < (i128)pr->A * s->os_den;"),
    "attached_takes_max": ("if (fc < r->f[d][idx]) {", "if (fc > r->f[d][idx] || r->f[d][idx] == INFINITY) {"),
    "facets_not_inserted": ("for (int64_t t = 0; t < F->n; t++)\n        for (int k = 0; k <= d; k++) iv_push(&out, F->v[(d + 1) * t + k]);",
                            "for (int64_t t = 0; t < 0; t++)\n        for (int k = 0; k <= d; k++) iv_push(&out, F->v[(d + 1) * t + k]);"),
    "vertices_skip_ac2": ("int ok = simplex_geom(pr, v, c->d, &s) && ac2_holds(pr, v, c->d, &s);",
                          "int ok = simplex_geom(pr, v, c->d, &s) && (c->d == 0 || ac2_holds(pr, v, c->d, &s));"),
    "quantise_centre_half_away_from_zero": ("pr->P[3 * i + c] = (int64_t)nearbyint(x * 1024.0);",
                                            "pr->P[3 * i + c] = (int64_t)round(x * 1024.0);"),
    "quantise_alpha_half_away_from_zero": ("pr->A = (int64_t)nearbyint(alpha * 1048576.0);",
                                           "pr->A = (int64_t)round(alpha * 1048576.0);"),
    "quantise_radius_truncates": ("int64_t R = (int64_t)nearbyint(rr * 1024.0);", "int64_t R = (int64_t)(rr * 1024.0);"),
    "violation_ignores_ties": ("return sos_sign(v, s, x, qx) < 0;", "return 0;"),
}

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "alpha_oracle.c")).read()


def _brute_cases():
    rng = np.random.default_rng(7)
    cases = []
    for kind in range(3):
        for _ in range(3):
            n = int(rng.integers(5, 10))
            if kind == 0:
                P = [tuple(int(v) for v in rng.integers(-3000, 3000, 3)) for _ in range(n)]
                R = [int(v) for v in rng.integers(800, 2500, n)]
            else:
                step = 1024 if kind == 1 else 512
                span = 1 if kind == 1 else 2
                pts = set()
                while len(pts) < n:
                    pts.add(tuple(int(v) * step for v in rng.integers(-span, span + 1, 3)))
                P = sorted(pts, key=lambda p: rng.random())
                R = [int(rng.choice([1024, 1448]))] * n if kind == 2 else [int(rng.choice([1024, 1448])) for _ in range(n)]
            for A in (0, 300000, None):
                cases.append((P, R, A, brute_alpha_complex(P, R, A)))
    return cases


@pytest.fixture(scope="module")
def brute_cases():
    return _brute_cases()


def _agrees(lib_path, P, R, A, want):
    c = np.array(P, dtype=np.float64) / 1024.0
    r = np.array(R, dtype=np.float64) / 1024.0
    try:
        ac = oracle.alpha_complex(c, r, alpha=0.0 if A is None else A / 2**20, alpha_inf=A is None, lib_path=lib_path)
    except oracle.OracleError:
        return False
    for d in range(4):
        got = {tuple(int(x) for x in t): (ac.f[d][i], bool(ac.attached[d][i])) for i, t in enumerate(ac.simplices[d])}
        if set(got) != set(want[d]):
            return False
        for t, (size, att) in want[d].items():
            if got[t][1] != att or abs(got[t][0] - float(size / 2**20)) > 1e-12 * max(1.0, abs(float(size / 2**20))):
                return False
    return True


def _golden_agrees(lib_path):
    for path in fixtures():
        atoms, alpha, expect = read_fixture(path)
        P = [tuple(int(x * 1024) for x in a[:3]) for a in atoms]
        R = [int(a[3] * 1024) for a in atoms]
        A = None if alpha is None else int(alpha * 2**20)
        want = {d: {t: v for t, v in expect.items() if len(t) == d + 1} for d in range(4)}
        want = {d: {t: (f * 2**20, att) for t, (f, att) in want[d].items()} for d in range(4)}
        if not _agrees(lib_path, P, R, A, want):
            return False
    return True


def _quantisation_agrees(lib_path):
    """Rounding half to even at 1/1024 A (the cases of test_oracle_quantisation)."""
    try:
        for r, R in ((1.7, 1741), (1000.5 / 1024.0, 1000), (1001.5 / 1024.0, 1002)):
            ac = oracle.alpha_complex(np.array([[0.25, -3.5, 7.0]]), np.array([r]), 0.0, lib_path=lib_path)
            if len(ac.f[0]) != 1 or ac.f[0][0] != -(R * R) / 2.0**20:
                return False
        for x in (2048.5, -2048.5):
            ac = oracle.alpha_complex(np.array([[0.0, 0.0, 0.0], [x / 1024.0, 0.0, 0.0]]), np.array([1.0, 1.0]), 0.0,
                                      lib_path=lib_path)
            if ac.simplices[1].tolist() != [[0, 1]] or ac.f[1][0] != 0.0:
                return False
        ac = oracle.alpha_complex(np.array([[0.0, 0.0, 0.0], [2050.0 / 1024.0, 0.0, 0.0]]), np.array([1.0, 1.0]),
                                  2048.5 / 2.0**20, lib_path=lib_path)
        if len(ac.simplices[1]) != 0:
            return False
    except oracle.OracleError:
        return False
    return True


def test_unmutated_copy_passes(brute_cases, tmp_path):
    path = str(tmp_path / "orig.so")
    src = tmp_path / "orig.c"
    src.write_text(SRC)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", str(src), "-o", path, "-lm"])
    assert _golden_agrees(path)
    assert _quantisation_agrees(path)
    assert all(_agrees(path, P, R, A, want) for P, R, A, want in brute_cases)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, brute_cases, tmp_path):
    old, new = MUTATIONS[name]
    assert old in SRC, f"mutation anchor for {name} not found"
    src = tmp_path / "mut.c"
    src.write_text(SRC.replace(old, new, 1))
    path = str(tmp_path / "mut.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", str(src), "-o", path, "-lm"])
    caught = (not _golden_agrees(path) or not _quantisation_agrees(path)
              or not all(_agrees(path, P, R, A, want) for P, R, A, want in brute_cases))
    assert caught, f"planted mistake {name} passed every pin"
