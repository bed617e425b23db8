"""Which precision level settles the predicates (Section 5.4: a floating-point
filter, then exact arithmetic where the filter cannot decide), counted by the
build and checked here.

* Lattice inputs are full of exact ties (co-orthospherical, coplanar and
  collinear subsets): their builds reach the exact integer level, and the
  results still equal the oracle's.
* In general position (a probe-radius globule) FP32 settles nearly every
  triangle and tetrahedron AC2 test, and the exact level is rare.
* The plain FP64 mode never counts an FP32 decision.
* The counts depend on the input only: two contexts built from the same atoms
  report the same figures.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_complex, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _lattice(seed):
    rng = np.random.default_rng(100 + seed)
    g = np.stack(np.meshgrid(*[np.arange(7)] * 3, indexing="ij"), -1).reshape(-1, 3)
    keep = rng.random(len(g)) < 0.8
    c = g[keep][rng.permutation(int(keep.sum()))] * (1.5 if seed % 2 else 2.0)
    r = rng.choice(np.array([1.25, 1.5]), len(c))
    return c.astype(np.float64), r


def _exact(st):
    return st["ac2_tests_tet"][2] + st["ac2_tests_tri"][2] + st["ac3_exact"]


@pytest.mark.parametrize("precision", [0, 1])
def test_lattice_reaches_exact_level(precision):
    exact = 0
    for seed in range(4):
        c, r = _lattice(seed)
        for alpha in (0.0, 0.5):
            gpu = run_gpu(c, r, alpha, precision=precision)
            assert_same_complex(gpu, oracle.alpha_complex(c, r, alpha))
            st = gpu.stats()
            exact += _exact(st)
            if precision == 1:
                assert st["ac2_tests_tet"][0] == 0 and st["ac2_tests_tri"][0] == 0
    assert exact > 0, "no lattice build reached the exact level"


def test_general_position_settles_in_fp32():
    c, r = synth.globule(61, 20000, probe=True)
    st = run_gpu(c, r, 0.0).stats()
    tet, tri = st["ac2_tests_tet"], st["ac2_tests_tri"]
    assert sum(tet) > 0 and sum(tri) > 0
    assert tet[0] >= 0.99 * sum(tet), tet
    assert tri[0] >= 0.99 * sum(tri), tri
    assert tet[2] + tri[2] <= 1e-4 * (sum(tet) + sum(tri)), (tet, tri)
    plain = run_gpu(c, r, 0.0, precision=1).stats()
    assert plain["ac2_tests_tet"][0] == 0 and plain["ac2_tests_tri"][0] == 0
    assert sum(plain["ac2_tests_tet"]) > 0


def test_counts_depend_on_input_only():
    c, r = synth.globule(62, 12000, probe=True)
    keys = ("ac2_tests_tet", "ac2_tests_tri", "ac2_tests_edge", "ac3_tests", "ac3_exact", "candidates", "simplices",
            "neighbour_pairs", "max_degree")
    a = run_gpu(c, r, 0.0).stats()
    b = run_gpu(c, r, 0.0).stats()
    assert {k: a[k] for k in keys} == {k: b[k] for k in keys}
