"""Slab cuts of the out-of-core build (host logic, no GPU).

A chunked build cuts the molecule into z-slabs of at most max_core_atoms
atoms and builds each with a halo of width reach = 2 ceil(sqrt(max W + A))
quanta. These tests check the cut against its definition: the slabs partition
the atoms, respect the size bound (a slab is larger only when its atoms share
one z value), and every pair of atoms whose grown balls meet (brute force,
exact integers) lies within reach in z, so the halo holds every such partner.
"""
import numpy as np
import pytest

import synth


def _quantise(c, r, alpha):
    Z = np.rint(c[:, 2] * 1024.0).astype(np.int64)
    P = np.rint(c * 1024.0).astype(np.int64)
    W = np.rint(r * 1024.0).astype(np.int64) ** 2
    A = int(np.rint(alpha * 1048576.0))
    return Z, P, W, A


def _meeting_pairs(P, W, A):
    s = W + A
    i, j = np.triu_indices(len(P), 1)
    D = ((P[i] - P[j]) ** 2).sum(1)
    ok = (s[i] >= 0) & (s[j] >= 0)
    t = D - s[i] - s[j]
    meet = ok & ((t <= 0) | (t * t <= 4 * s[i] * s[j]))
    return i[meet], j[meet]


@pytest.mark.parametrize("alpha,max_core", [(0.0, 150), (1.0, 37), (-1.5, 400), (0.0, 5000)])
def test_plan_partitions_and_reach(alpha, max_core):
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(5, 1200, probe=True)
    thr, reach = ac.chunk_plan(c, r, alpha, max_core)
    Z, P, W, A = _quantise(c, r, alpha)
    H2 = int(W.max()) + A
    hq = 0
    while hq * hq < H2:
        hq += 1
    assert reach == 2 * hq
    assert np.all(np.diff(thr) > 0) and thr[0] == Z.min() and thr[-1] == Z.max() + 1
    slab = np.searchsorted(thr, Z, side="right") - 1
    assert slab.min() == 0 and slab.max() == len(thr) - 2
    sizes = np.bincount(slab, minlength=len(thr) - 1)
    assert sizes.min() > 0
    for k in np.nonzero(sizes > max_core)[0]:
        assert len(np.unique(Z[slab == k])) == 1, "an oversized slab must be a single z value"
    if max_core >= len(c):
        assert len(thr) == 2
    # every partner of an atom (grown balls meet) is within reach in z
    i, j = _meeting_pairs(P, W, A)
    assert len(i) > 0
    assert np.all(np.abs(Z[i] - Z[j]) <= reach)


def test_plan_with_equal_z_layers():
    """A lattice: whole z layers of equal Z; cuts fall between layers only."""
    import paper_1908_05944_gb300 as ac

    g = np.arange(6, dtype=np.float64) * 1.5
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = np.full(len(c), 1.0)
    thr, reach = ac.chunk_plan(c, r, 0.0, 40)  # 36 atoms per layer: one layer per slab
    Z = np.rint(c[:, 2] * 1024.0).astype(np.int64)
    assert len(thr) == 7 and set(thr[:-1]) == set(np.unique(Z))
    thr, _ = ac.chunk_plan(c, r, 0.0, 10)  # a layer exceeds the bound: still one layer per slab
    assert len(thr) == 7
    thr, _ = ac.chunk_plan(c, r, 0.0, 72)
    assert len(thr) == 4


def test_plan_errors():
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(6, 50, probe=False)
    with pytest.raises(ac.AlphacError) as e:
        ac.chunk_plan(c, r, 0.0, 0)
    assert e.value.code == ac.AC_ERR_INVALID_ARG
    bad = c.copy()
    bad[7, 1] = np.nan
    with pytest.raises(ac.AlphacError) as e:
        ac.chunk_plan(bad, r, 0.0, 10)
    assert e.value.code == ac.AC_ERR_INVALID_ARG and "atom 7" in str(e.value)
    big = r.copy()
    big[3] = 4.5
    with pytest.raises(ac.AlphacError) as e:
        ac.chunk_plan(c, big, 0.0, 10)
    assert e.value.code == ac.AC_ERR_RANGE
    thr, reach = ac.chunk_plan(np.zeros((0, 3)), np.zeros(0), 0.0, 10)
    assert len(thr) == 0 and reach == 0


def test_plan_large_input_matches_greedy_cut():
    """150k atoms (the plan runs on several host threads): the cut equals a plain greedy cut over
    the distinct z values, and the first bad atom is reported whatever range it falls in."""
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(7, 150000, probe=True)
    max_core = 20000
    thr, _ = ac.chunk_plan(c, r, 0.0, max_core)
    Z = np.rint(c[:, 2] * 1024.0).astype(np.int64)
    vals, counts = np.unique(Z, return_counts=True)
    want = [vals[0]]
    run = 0
    for v, h in zip(vals, counts):
        if run > 0 and run + h > max_core:
            want.append(v)
            run = 0
        run += h
    want.append(vals[-1] + 1)
    assert np.array_equal(thr, np.array(want))
    bad = c.copy()
    bad[140001, 0] = np.inf
    bad[90001, 2] = np.nan
    with pytest.raises(ac.AlphacError) as e:
        ac.chunk_plan(bad, r, 0.0, max_core)
    assert "atom 90001" in str(e.value)


def test_plan_coordinate_range():
    """Coordinates must quantise below 2^30 quanta (|x| < 2^20 A), so any two differ by less than 2^31."""
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(6, 50, probe=False)
    for edge in (1048575.0, -1048575.0, 1048576.0 - 1.0 / 1024.0):
        ok = c.copy()
        ok[3, 0] = edge  # 2^30 - 1024 and 2^30 - 1 quanta: accepted
        ac.chunk_plan(ok, r, 0.0, 10)
    for edge in (1048576.0, -1048576.0, 1048576.0 - 1.0 / 4096.0):
        bad = c.copy()
        bad[3, 2] = edge  # 2^30 quanta after rounding: refused
        with pytest.raises(ac.AlphacError) as e:
            ac.chunk_plan(bad, r, 0.0, 10)
        assert e.value.code == ac.AC_ERR_RANGE and "atom 3" in str(e.value)
