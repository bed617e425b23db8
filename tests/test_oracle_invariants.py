"""Invariants of the alpha complex on the oracle's output for protein-like inputs.

* K_alpha is a simplicial complex (Section 2.1): every face of a simplex is in it.
* Size is monotone under faces (the witnesses of a coface are witnesses of the face).
* Size >= OrthoSize (Section 2.3); unattached simplices have Size == OrthoSize.
* A triangle has at most two tetrahedral cofaces in a triangulation.
* Every attached simplex takes the smallest Size of a coface one dimension up.
* Simplices per atom lie in the range of Table 1 (alpha = 0, van der Waals radii):
  932/260 = 3.6 up to 38796/4384 = 8.9 for the paper's molecules.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def globule2k():
    c, r = synth.workload("globule2k_vdw")
    return c, r, oracle.alpha_complex(c, r, 0.0)


@pytest.fixture(scope="module")
def globule3k_probe():
    c, r = synth.globule(77, 3000, probe=True)
    return c, r, oracle.alpha_complex(c, r, 0.0)


def _sets(ac):
    return [{tuple(int(x) for x in t): i for i, t in enumerate(ac.simplices[d])} for d in range(4)]


@pytest.mark.parametrize("which", ["globule2k", "globule3k_probe"])
def test_complex_invariants(which, request):
    c, r, ac = request.getfixturevalue(which)
    S = _sets(ac)
    for d in range(4):
        s = ac.simplices[d]
        if len(s):
            assert np.all(np.diff(s, axis=1) > 0), "tuples ascending"
            keys = [tuple(t) for t in s]
            assert keys == sorted(keys) and len(set(keys)) == len(keys), "sorted, unique"
    for d in range(1, 4):
        for t, i in S[d].items():
            for face in itertools.combinations(t, d):
                assert face in S[d - 1], ("closure", t, face)
                j = S[d - 1][face]
                assert ac.f[d - 1][j] <= ac.f[d][i], ("monotone", t, face)
    for d in range(4):
        assert np.all(ac.f[d] >= ac.orthosize[d] - 1e-12 * np.abs(ac.orthosize[d]))
        un = ~ac.attached[d]
        assert np.array_equal(ac.f[d][un], ac.orthosize[d][un])
        assert np.all(ac.f[d] <= 0.0)  # alpha = 0
    cof = {}
    for t in S[3]:
        for face in itertools.combinations(t, 3):
            cof[face] = cof.get(face, 0) + 1
    assert max(cof.values()) <= 2
    # attached simplices: Size = min over cofaces in the complex
    for d in range(3):
        best = {}
        for t, i in S[d + 1].items():
            for face in itertools.combinations(t, d + 1):
                best[face] = min(best.get(face, np.inf), ac.f[d + 1][i])
        for t, i in S[d].items():
            if ac.attached[d][i]:
                assert ac.f[d][i] == best[t]


def test_simplices_per_atom_in_table1_range(globule2k):
    c, r, ac = globule2k
    per_atom = sum(ac.counts()) / len(r)
    assert 3.5 <= per_atom <= 9.0


def test_threads_do_not_change_result(globule2k):
    c, r, ac = globule2k
    ac1 = oracle.alpha_complex(c, r, 0.0, threads=1)
    for d in range(4):
        assert np.array_equal(ac.simplices[d], ac1.simplices[d])
        assert np.array_equal(ac.f[d], ac1.f[d])


def test_concurrent_runs_equal_sequential_runs():
    # the oracle keeps no shared state: runs on several host threads at once (as the full-size
    # batch parity test makes them) give the lists and values of runs made one at a time
    from concurrent.futures import ThreadPoolExecutor

    mols = [synth.globule(1000 + m, 600 + 41 * m, probe=True) for m in range(16)]
    seq = [oracle.alpha_complex(c, r, 0.0, threads=2) for c, r in mols]

    def same(m):
        got = oracle.alpha_complex(*mols[m], 0.0, threads=2)
        return all(np.array_equal(got.simplices[d], seq[m].simplices[d]) and np.array_equal(got.f[d], seq[m].f[d])
                   and np.array_equal(got.attached[d], seq[m].attached[d]) for d in range(4))

    for _ in range(2):
        with ThreadPoolExecutor(8) as ex:
            assert all(ex.map(same, range(len(mols))))
