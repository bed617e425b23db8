"""The out-of-core build: slabs with halos, shares placed in host memory.

A chunked build must return exactly the lists of a build of the whole
molecule (rows, attached flags, filtration values) and of the oracle, for any
slab size: slabs thinner than the halo, cuts between equal-z lattice layers
(ties broken by input index), alpha > 0 and < 0, both precisions.
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_values

pytestmark = pytest.mark.gpu


def _whole(c, r, alpha, opt=None):
    import torch

    import paper_1908_05944_gb300 as ac

    return ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), alpha, opt).build()


def _assert_equal_to_whole(ch, whole):
    for d in range(4):
        t = whole.simplices(d).cpu().numpy()
        got = ch.simplices(d)
        assert got.shape == t.shape, f"dim {d}: {got.shape[0]} chunked vs {t.shape[0]} whole"
        assert np.array_equal(got, t), f"dim {d}: rows differ"
        assert np.array_equal(ch.attached(d), whole.attached(d).cpu().numpy()), f"dim {d}: attached flags differ"
        assert np.array_equal(ch.filtration_values(d), whole.filtration_values(d).cpu().numpy()), \
            f"dim {d}: values differ"


def _assert_equal_to_oracle(ch, ref):
    for d in range(4):
        assert np.array_equal(ch.simplices(d), ref.simplices[d]), f"dim {d}: rows differ from the oracle"
        assert np.array_equal(ch.attached(d).astype(bool), ref.attached[d])
        assert_values(ch.filtration_values(d), ref.f[d], f"dim {d}")


@pytest.mark.parametrize("max_core", [120, 700, 10 ** 6])
def test_chunked_equals_whole_and_oracle(max_core):
    import oracle
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(31, 3000, probe=True)
    ch = ac.ChunkedComplex(c, r, 0.0, max_core)
    st = ch.stats()
    thr, reach = ac.chunk_plan(c, r, 0.0, max_core)
    assert st["n_chunks"] == len(thr) - 1 and st["reach"] == reach
    assert st["core_max"] <= max_core and st["subset_total"] >= len(c)
    if max_core >= len(c):
        assert st["n_chunks"] == 1 and st["subset_total"] == len(c)
    _assert_equal_to_whole(ch, _whole(c, r, 0.0))
    _assert_equal_to_oracle(ch, oracle.alpha_complex(c, r, 0.0))


@pytest.mark.parametrize("alpha", [1.25, -0.8])
def test_chunked_other_alphas(alpha):
    import oracle
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(32, 2000, probe=False)
    ch = ac.ChunkedComplex(c, r, alpha, 250)
    assert ch.stats()["n_chunks"] >= 6
    _assert_equal_to_whole(ch, _whole(c, r, alpha))
    _assert_equal_to_oracle(ch, oracle.alpha_complex(c, r, alpha))


def test_chunked_lattice_ties():
    """Equal-z layers, every predicate tied: cuts between layers, one layer per slab."""
    import oracle
    import paper_1908_05944_gb300 as ac

    g = np.arange(6, dtype=np.float64) * 1.5
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(3)
    c = c[rng.permutation(len(c))]  # input order unrelated to the slabs
    r = np.full(len(c), 1.0)
    ch = ac.ChunkedComplex(c, r, 1.0, 36)
    assert ch.stats()["n_chunks"] == 6
    _assert_equal_to_whole(ch, _whole(c, r, 1.0))
    _assert_equal_to_oracle(ch, oracle.alpha_complex(c, r, 1.0))


def test_chunked_options_pass_through():
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(33, 1500, probe=True)
    for opt in (ac.options(precision=ac.AC_PRECISION_PLAIN_FP64), ac.options(filtration=ac.AC_FILTRATION_ORTHOSIZE)):
        ch = ac.ChunkedComplex(c, r, 0.0, 200, opt)
        _assert_equal_to_whole(ch, _whole(c, r, 0.0, opt))


def test_chunked_edge_cases():
    import torch

    import paper_1908_05944_gb300 as ac

    ch = ac.ChunkedComplex(np.zeros((0, 3)), np.zeros(0), 0.0, 100)
    assert all(ch.count(d) == 0 for d in range(4)) and ch.stats()["n_chunks"] == 0
    one = ac.ChunkedComplex(np.array([[1.0, 2.0, 3.0]]), np.array([1.5]), 0.0, 1)
    assert one.simplices(0).tolist() == [[0]] and one.filtration_values(0)[0] == -2.25
    c, r = synth.globule(34, 200, probe=True)
    with pytest.raises(ac.AlphacError) as e:
        ac.ChunkedComplex(c, r, 0.0, 50, ac.options(keep_candidates=True))
    assert e.value.code == ac.AC_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        ac.ChunkedComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0, 50)
    dup = c.copy()
    dup[17] = dup[4]
    with pytest.raises(ac.AlphacError) as e:
        ac.ChunkedComplex(dup, r, 0.0, 50)
    assert e.value.code == ac.AC_ERR_DEGENERATE
